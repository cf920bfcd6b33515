"""rANS runs on the GPU (K independently coded runs per record, K warps per brick at full
resolution, one warp walking the runs at coarse levels of detail) against the oracle: every brick
at every level of detail in every schedule, for K = 2, 4, 8 and brick sizes 8^3 to 64^3; the
coarsest labels read past the runs' states; the detail split (coarse records re-coded in runs);
the frame cache (the symbol kernel with a device-side count); corrupt run starts rejected at load
and a corrupt word inside a run reported for exactly its item."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_36898_gb300 as vc  # noqa: E402
from test_decode_gpu import MODES, gpu_decode, oracle_bricks  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vc._lib_handle()


def _vol(b, seed):
    return synth.fill(synth.small(dims=(3 * b - 5, 2 * b + 3, b + 6), seed=seed, grid=max(4, b // 2),
                                  diameter=max(3.0, b / 2.5), bg=0.2))


@pytest.mark.parametrize("log2b,K,flags", [(3, 2, 0), (4, 4, 2), (5, 2, 0), (5, 4, 0), (5, 8, 1), (6, 4, 0)])
def test_runs_every_brick_every_lod_every_schedule(log2b, K, flags):
    V = _vol(1 << log2b, 70 + log2b + K)
    enc = vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=1, flags=flags | oracle.runs_flag(K))
    n = oracle.header(enc)["n_bricks"]
    ids = np.arange(n)
    for lod in range(log2b + 1):
        ref = oracle_bricks(enc, ids, lod)
        for mode in MODES:
            if log2b == 6 and mode == "plain" and lod > 1:
                continue  # one launch per brick of 64^3: the other schedules cover these levels
            out, st = gpu_decode(enc, ids, lod, mode)
            assert st[0] == 0, (mode, lod, st)
            assert np.array_equal(out, ref), (mode, lod)


@pytest.mark.parametrize("K", [2, 8])
def test_runs_coarsest_labels_and_split(K):
    V = _vol(32, 90 + K)
    enc = vc.vc_encode_volume(V, 5, op_mask=0x7F, coder=1, flags=oracle.runs_flag(K))
    n = oracle.header(enc)["n_bricks"]
    vol = vc.Volume(enc)
    try:
        ids = torch.arange(n, dtype=torch.int32, device="cuda")
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
        vc.vc_coarsest_labels(vol.handle, ids.data_ptr(), n, out.data_ptr(), st.data_ptr(), 0)
        torch.cuda.synchronize()
        assert int(st[0]) == 0
        want = np.array([oracle.decode_brick(enc, i, 5).reshape(-1)[0] for i in range(n)], np.uint32)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), want)
    finally:
        vol.release()
    sv = vc.Volume(enc, split=True)
    try:
        for lod in range(6):
            e = 32 >> lod
            ids = torch.arange(n, dtype=torch.int32, device="cuda")
            cache = torch.full((n * e ** 3,), -1, dtype=torch.int32, device="cuda")
            st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
            for mode in ("grid", "batched"):
                sv.decode(ids, ids, cache, lod=lod, mode=mode, status=st)
                torch.cuda.synchronize()
                assert int(st[0]) == 0, (lod, mode)
                got = cache.cpu().numpy().view(np.uint32).reshape(n, e, e, e)
                assert np.array_equal(got, oracle_bricks(enc, range(n), lod)), (lod, mode)
    finally:
        sv.release()


def test_runs_frame_cache():
    """The frame cache's decode stage (item count on the device) on a volume of 4 runs per record."""
    from test_frame_gpu import _run
    V = synth.fill(synth.small(dims=(96, 80, 64), seed=71, grid=16, diameter=14.0, bg=0.03))
    enc = oracle.encode_volume(V, 4, coder=oracle.CODER_RANS, flags=oracle.runs_flag(4))
    _run(enc, dict(max_lod=2, cap=1 << 22, per_frame=120, free_cap=1 << 20), frames=5)


def test_runs_corrupt_starts_and_words():
    V = _vol(16, 5)
    enc = vc.vc_encode_volume(V, 4, op_mask=0x7F, coder=1, flags=oracle.runs_flag(4))
    h = oracle.header(enc)
    rec_off = (128 + 4 * (h["n_bricks"] + 1) + 15) & ~15
    lib = oracle._load()
    b = next(i for i in range(h["n_bricks"]) if oracle.brick_record(enc, i)["n_sym"] > 300)
    r = oracle.brick_record(enc, b)
    S = r["n_sym"]
    hw = int(lib.oracle_head_words(1, oracle.runs_flag(4), S))
    Q = 32 * -(-S // 128)
    nr = -(-S // Q)
    at = rec_off + 4 * r["offset_words"] + 16 + 4 * (hw - (nr - 1))  # the run starts
    bad = enc.copy()
    bad[at: at + 4] = np.asarray([r["coded_bytes"] // 2 + 1], "<u4").view(np.uint8)  # past the words
    with pytest.raises(vc.VCError) as ex:
        vc.Volume(bad)
    assert ex.value.code == vc.VC_ERR_FORMAT
    # a flipped word inside run 1: the oracle and the GPU report that brick (at full resolution)
    w0 = int(np.frombuffer(enc[at: at + 4].tobytes(), "<u4")[0])
    words_at = rec_off + 4 * r["offset_words"] + 16 + 4 * hw + 4 * r["n_pal"]
    bad = enc.copy()
    bad[words_at + 2 * w0] ^= 0x5A
    assert oracle.decode_brick_status(bad, b) == oracle.ERR_CORRUPT
    ids = [b - 1, b, b + 1] if b > 0 else [b, b + 1]
    for mode in ("grid", "batched", "pipelined"):
        _, st = gpu_decode(bad, ids, 0, mode)
        assert st[0] == vc.VC_ERR_CORRUPT and ids[st[1]] == b, (mode, st)
