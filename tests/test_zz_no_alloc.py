"""vc_decode_bricks_noalloc (statically reserved workspace) against vc_decode_bricks, through the C ABI.

Collected last on purpose: it must pass both alone and after every other GPU test has run in the
same process (other volumes loaded, the stream-ordered pool warm)."""
import numpy as np
import pytest

import synth
import paper_2609_36898_gb300 as vc

pytestmark = pytest.mark.gpu

VC_NOALLOC_WS_BYTES = 32 << 20


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _ws_stride(max_sym: int) -> int:
    return 16 * (((max_sym + 1) // 2 + 15) // 16) + 16


@pytest.mark.parametrize("coder", [1, 0])
@pytest.mark.parametrize("mode", ["grid", "batched"])
def test_noalloc_matches_decode_bricks_twice_in_a_row(torch, coder, mode):
    V = synth.fill(synth.small(), (0, 0, 0), (128, 128, 128))
    enc = vc.vc_encode_volume(V, 5, op_mask=0x7F, coder=coder)
    vol = vc.Volume(enc)
    n = vol.n_bricks
    e3 = vol.b ** 3
    m = vc.MODES[mode]
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(7 + coder)
    for call in range(2):  # two calls in a row: the shared workspace is reused
        ids_np = rng.permutation(n).astype(np.uint32)
        ids = torch.from_numpy(ids_np.view(np.int32)).cuda()
        slots = torch.arange(n, dtype=torch.int32, device="cuda")
        ref = torch.full((n * e3,), -1, dtype=torch.int32, device="cuda")
        got = torch.full((n * e3,), -1, dtype=torch.int32, device="cuda")
        st_ref = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
        st_got = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
        vc.vc_decode_bricks(vol.handle, ids.data_ptr(), n, slots.data_ptr(), ref.data_ptr(), 0, m,
                            st_ref.data_ptr(), stream.cuda_stream)
        vc.vc_decode_bricks_noalloc(vol.handle, ids.data_ptr(), n, slots.data_ptr(), got.data_ptr(), 0, m,
                                    st_got.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        assert int(st_ref[0]) == 0 and int(st_got[0]) == 0, (st_ref.tolist(), st_got.tolist())
        assert torch.equal(ref, got), f"call {call}: noalloc output differs"
        # and both equal the input volume (lossless)
        out = got.cpu().numpy().view(np.uint32).reshape(n, vol.b, vol.b, vol.b)
        nb = 128 // vol.b
        for i in (0, n // 2, n - 1):
            bid = int(ids_np[i])
            bx, by, bz = bid % nb, (bid // nb) % nb, bid // (nb * nb)
            b = vol.b
            assert np.array_equal(out[i], V[bz * b:(bz + 1) * b, by * b:(by + 1) * b, bx * b:(bx + 1) * b])
    vol.release()


def test_noalloc_rejects_requests_beyond_its_workspace(torch):
    V = synth.fill(synth.small(), (0, 0, 0), (64, 64, 64))
    enc = vc.vc_encode_volume(V, 5, op_mask=0x7F, coder=1)
    vol = vc.Volume(enc)
    info = vc.vc_volume_info_get(vol.handle)
    stride = _ws_stride(int(info.max_sym))
    n_max = VC_NOALLOC_WS_BYTES // stride
    ids = torch.zeros(n_max + 1, dtype=torch.int32, device="cuda")
    cache = torch.zeros((n_max + 1) * vol.b ** 3, dtype=torch.int32, device="cuda")
    st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(vc.VCError) as ex:
        vc.vc_decode_bricks_noalloc(vol.handle, ids.data_ptr(), n_max + 1, ids.data_ptr(), cache.data_ptr(), 0,
                                    vc.VC_MODE_GRID, st.data_ptr(), s)
    assert ex.value.code == vc.VC_ERR_ARG
    # the largest accepted size decodes (every item is brick 0 into its own slot)
    slots = torch.arange(n_max, dtype=torch.int32, device="cuda")
    vc.vc_decode_bricks_noalloc(vol.handle, ids.data_ptr(), n_max, slots.data_ptr(), cache.data_ptr(), 0,
                                vc.VC_MODE_GRID, st.data_ptr(), s)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    first = cache[: vol.b ** 3]
    last = cache[(n_max - 1) * vol.b ** 3: n_max * vol.b ** 3]
    assert torch.equal(first, last)
    # the pipelined schedule allocates, so it is refused here
    with pytest.raises(vc.VCError):
        vc.vc_decode_bricks_noalloc(vol.handle, ids.data_ptr(), 1, slots.data_ptr(), cache.data_ptr(), 0,
                                    vc.VC_MODE_PIPELINED, st.data_ptr(), s)
    vol.release()
