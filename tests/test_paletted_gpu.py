"""Cache paletting on the GPU, through the C ABI: every slot holds packed palette indices (Methods,
"Cache paletting"); unpacked and looked up in each brick's palette they give exactly the oracle's
labels, at every level of detail and with the grid, batched and per-brick schedules."""
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


def unpack(words: np.ndarray, n: int, bits: int, per: int) -> np.ndarray:
    v = np.arange(n)
    w = words[v // per].astype(np.uint64)
    return ((w >> (bits * (v % per)).astype(np.uint64)) & ((1 << bits) - 1)).astype(np.int64)


@pytest.mark.parametrize("log2b,coder,diameter", [(5, 1, 14.0), (4, 0, 6.0), (3, 1, 20.0)])
def test_paletted_slots_decode_to_the_oracle_labels(log2b, coder, diameter):
    V = synth.fill(synth.small(dims=(128, 96, 64), seed=70 + log2b, grid=16, diameter=diameter, bg=0.2))
    enc = vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=coder)
    vol = vc.Volume(enc)
    try:
        n = vol.n_bricks
        max_pal = int(oracle.header(enc)["max_pal"])
        for lod in range(0, min(3, log2b) + 1):
            e = vol.b >> lod
            words, bits, per = vc.vc_volume_slot_words(vol.handle, lod, True)
            want_bits = max(1, int(np.ceil(np.log2(max_pal)))) if max_pal > 1 else 1
            assert bits == want_bits and per == 32 // bits and words == -(-e ** 3 // per)
            assert vc.vc_volume_slot_words(vol.handle, lod, False)[0] == e ** 3
            ids = torch.arange(n, dtype=torch.int32, device="cuda")
            for mode in ("grid", "batched", "plain"):
                cache = torch.full((n * words,), -1, dtype=torch.int32, device="cuda")
                st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
                vol.decode(ids, ids, cache, lod, vc.MODES[mode] | vc.VC_MODE_PALETTED, st)
                torch.cuda.synchronize()
                assert int(st[0]) == 0
                out = cache.cpu().numpy().view(np.uint32).reshape(n, words)
                for i in range(0, n, max(1, n // 9)):
                    pal = oracle.brick_record(enc, i)["palette"]
                    idx = unpack(out[i], e ** 3, bits, per)
                    assert idx.max() < len(pal)
                    assert np.array_equal(pal[idx].reshape(e, e, e), oracle.decode_brick(enc, i, lod)), (mode, lod, i)
        with pytest.raises(vc.VCError):  # the pipelined schedule writes labels only
            cache = torch.zeros(n * 32768, dtype=torch.int32, device="cuda")
            vol.decode(ids, ids, cache, 0, vc.VC_MODE_PIPELINED | vc.VC_MODE_PALETTED, st)
    finally:
        vol.release()
