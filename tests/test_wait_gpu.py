"""The bounded device-side wait of the batched schedule's prefetch, made to run out: a wait on an
mbarrier that nothing arrives at (no copy bound to it) gives up after its wall-clock budget,
reports VC_ERR_TIMEOUT through the status buffer, and leaves the context usable (a decode that
follows matches the oracle)."""
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


@pytest.mark.parametrize("budget_us", [2000, 20000])
def test_wait_runs_out_and_reports_timeout(budget_us):
    st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
    vc.vc_selftest_bounded_wait(budget_us, st.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    w = st.cpu().numpy().view(np.uint32)
    assert int(st[0]) == vc.VC_ERR_TIMEOUT
    waited_ns = int(w[2]) | (int(w[3]) << 32)
    assert budget_us * 1000 <= waited_ns < budget_us * 1000 + 50_000_000
    # the context is still usable
    V = synth.fill(synth.small(dims=(40, 24, 20), seed=3))
    enc = oracle.encode_volume(V, 3, coder=oracle.CODER_RANS)
    vol = vc.Volume(enc)
    try:
        n = vol.n_bricks
        ids = torch.arange(n, dtype=torch.int32, device="cuda")
        cache = torch.zeros(n * 8 ** 3, dtype=torch.int32, device="cuda")
        st.zero_()
        vc.vc_decode_bricks(vol.handle, ids.data_ptr(), n, ids.data_ptr(), cache.data_ptr(), 0, vc.VC_MODE_BATCHED,
                            st.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert int(st[0]) == 0
        got = cache.cpu().numpy().view(np.uint32).reshape(n, -1)
        for b in range(n):
            assert np.array_equal(got[b], oracle.decode_brick(enc, b).reshape(-1))
    finally:
        vol.release()


def test_wait_arguments_checked():
    st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
    for bad in (0, 10_000_001):
        with pytest.raises(vc.VCError):
            vc.vc_selftest_bounded_wait(bad, st.data_ptr())
