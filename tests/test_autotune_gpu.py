"""The schedule autotuner through the C ABI: it keeps a schedule the volume supports, the volume
decodes bit-exactly with it, and the choice is at least as fast as the default when re-timed."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_36898_gb300 as vc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vc._lib_handle()


@pytest.mark.parametrize("log2b,coder", [(5, 1), (4, 0)])
def test_autotune_keeps_a_supported_fast_schedule(log2b, coder):
    V = synth.fill(synth.small(dims=(256, 256, 128), seed=60 + log2b, grid=16, diameter=20.0, bg=0.1))
    enc = vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=coder)
    vol = vc.Volume(enc)
    try:
        n = vol.n_bricks
        e = vol.b
        ids = torch.arange(n, dtype=torch.int32, device="cuda")
        cache = torch.zeros(n * e ** 3, dtype=torch.int32, device="cuda")
        st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        sched, mode, ms = vc.vc_volume_autotune(vol.handle, ids.data_ptr(), n, ids.data_ptr(), cache.data_ptr(), 0,
                                                st.data_ptr(), s, reps=2)
        assert int(st[0]) == 0 and ms > 0
        assert mode in (vc.VC_MODE_GRID, vc.VC_MODE_BATCHED)
        assert vc.vc_volume_get_schedule(vol.handle) == sched
        cache.zero_()
        vol.decode(ids, ids, cache, 0, mode, st)
        torch.cuda.synchronize()
        assert int(st[0]) == 0
        out = cache.cpu().numpy().view(np.uint32).reshape(n, e, e, e)
        for i in np.random.default_rng(0).choice(n, 12, replace=False):
            assert np.array_equal(out[i], oracle.decode_brick(enc, int(i), 0))
    finally:
        vol.release()
