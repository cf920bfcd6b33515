"""GPU parity: libvc.so's CUDA decoder against the CPU oracle, through the C ABI.

Bit-exact on every brick (integer work): every brick size 2..32, both coders, every operation
subset, every level of detail, all three schedules; brute-force enumerated legal streams;
corrupt records (each rule of the format) must raise VC_ERR_CORRUPT for exactly that item; the
512^3 workload the benchmark times is checked at full size against the generator's voxels (the
encoding is lossless) and against the oracle on sampled bricks.
"""
import random

import numpy as np
import pytest

import oracle
import synth
from streams import (OP_ADV, OP_DELTA, OP_LAST, OP_NY, OP_PARENT, StreamEnumerator, load_golden, padded_brick)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_36898_gb300 as vc  # noqa: E402

MODES = ["plain", "grid", "batched", "pipelined"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vc._lib_handle()


def gpu_decode(enc: np.ndarray, ids, lod=0, mode="batched", slots=None, expect_status=0, cache_slots=None):
    """Decodes bricks `ids` into slots 0..n-1 (or `slots`); returns (n, e, e, e) labels and status."""
    vol = vc.Volume(enc, device=0)
    try:
        ids_t = torch.as_tensor(np.asarray(ids, dtype=np.int64), dtype=torch.int64).to(torch.int32).cuda()
        n = ids_t.numel()
        e = vol.edge(lod)
        if slots is None:
            slots = np.arange(n)
        slots_t = torch.as_tensor(np.asarray(slots, dtype=np.int64)).to(torch.int32).cuda()
        nslots = int(max(slots)) + 1 if n else 1
        cache = torch.full((nslots * e ** 3,), -1, dtype=torch.int32, device="cuda")
        status = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
        vol.decode(ids_t, slots_t, cache, lod=lod, mode=mode, status=status)
        torch.cuda.synchronize()
        st = status.cpu().numpy()
        out = cache.cpu().numpy().view(np.uint32).reshape(nslots, e, e, e)
        return out, st
    finally:
        vol.release()


def oracle_bricks(enc, ids, lod=0):
    return np.stack([oracle.decode_brick(enc, int(i), lod) for i in ids])


@pytest.fixture(scope="module")
def small_volume():
    return synth.fill(synth.small(dims=(40, 24, 20), seed=7, diameter=10.0, bg=0.2))


@pytest.mark.parametrize("log2b", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("coder", [0, 1])
def test_parity_every_brick_every_lod(small_volume, log2b, coder):
    enc = oracle.encode_volume(small_volume, log2b, coder=coder)
    n = oracle.header(enc)["n_bricks"]
    ids = np.arange(n)
    for lod in range(log2b + 1):
        ref = oracle_bricks(enc, ids, lod)
        for mode in MODES:
            out, st = gpu_decode(enc, ids, lod, mode)
            assert st[0] == 0, (mode, lod, st)
            assert np.array_equal(out, ref), (mode, lod)


@pytest.mark.parametrize("mask", [1 << 4, (1 << 4) | 1, (1 << 4) | 0b1111, 0x7F & ~(1 << OP_DELTA),
                                  0x7F & ~(1 << OP_LAST), 0x7F])
def test_parity_operation_subsets(small_volume, mask):
    for coder in (0, 1):
        for flags in (0, 1):
            enc = oracle.encode_volume(small_volume, 4, op_mask=mask, coder=coder, flags=flags)
            ids = np.arange(oracle.header(enc)["n_bricks"])
            out, st = gpu_decode(enc, ids, 0, "batched")
            assert st[0] == 0
            assert np.array_equal(out, oracle_bricks(enc, ids))


def test_parity_workload_64cube():
    V = synth.fill(synth.c1())
    for coder in (0, 1):
        enc = oracle.encode_volume(V, 5, coder=coder)
        for mode in MODES:
            out, st = gpu_decode(enc, range(8), 0, mode)
            assert st[0] == 0
            for i in range(8):
                assert np.array_equal(out[i], padded_brick(V, 32, i))


def _bricks_of(V, b):
    nz, ny, nx = (s // b for s in V.shape)
    return V.reshape(nz, b, ny, b, nx, b).transpose(0, 2, 4, 1, 3, 5).reshape(-1, b, b, b)


@pytest.mark.parametrize("coder", [0, 1])
def test_parity_full_size_512cube_batched(coder):
    """The benchmark's workload at full size: all 4096 bricks, batched schedule."""
    spec = synth.c2()
    V = synth.fill(spec)
    enc = vc.vc_encode_volume(V, 5, coder=coder)
    ids = np.arange(4096)
    out, st = gpu_decode(enc, ids, 0, "batched")
    assert st[0] == 0
    assert np.array_equal(out, _bricks_of(V, 32))
    rng = np.random.default_rng(0)
    for i in rng.choice(4096, size=24, replace=False):
        assert np.array_equal(out[i], oracle.decode_brick(enc, int(i)))
    # the same volume encoded by the oracle decodes identically (sampled bricks)
    sub = V[:64, :64, :]
    enc2 = oracle.encode_volume(sub, 5, coder=coder)
    out2, st2 = gpu_decode(enc2, np.arange(64), 0, "grid")
    assert st2[0] == 0 and np.array_equal(out2, _bricks_of(sub, 32))


@pytest.mark.parametrize("mode", ["auto", "grid", "batched"])
def test_parity_full_size_512cube_bench_path(mode):
    """The benchmark's exact configuration at full size: the 512^3 volume (rANS, 32^3 bricks, all
    operations), all 4096 bricks in one call, ids = slots = 0..4095, with the schedule the library's
    autotuner picks on that very request ("auto": the grid schedule on GB300 with the size-aware
    order, 256 threads) and with the grid and batched schedules fixed; every brick against the
    generator's voxels and sampled bricks against the oracle."""
    spec = synth.c2()
    V = synth.fill(spec)
    enc = vc.vc_encode_volume(V, 5, op_mask=0x7F, coder=1)
    want = _bricks_of(V, 32)
    vol = vc.Volume(enc, device=0)
    try:
        n = vol.n_bricks
        assert n == 4096
        ids = torch.arange(n, dtype=torch.int32, device="cuda")
        cache = torch.full((n * 32 ** 3,), -1, dtype=torch.int32, device="cuda")
        st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        if mode == "auto":
            _, m, _ = vc.vc_volume_autotune(vol.handle, ids.data_ptr(), n, ids.data_ptr(), cache.data_ptr(), 0,
                                            st.data_ptr(), s, reps=1)
            torch.cuda.synchronize()
            st.zero_()
            cache.fill_(-1)
        else:
            m = vc.MODES[mode]
        for call in range(2):
            vc.vc_decode_bricks(vol.handle, ids.data_ptr(), n, ids.data_ptr(), cache.data_ptr(), 0, m, st.data_ptr(), s)
            torch.cuda.synchronize()
            assert int(st[0]) == 0, st.tolist()
            out = cache.cpu().numpy().view(np.uint32).reshape(n, 32, 32, 32)
            bad = np.flatnonzero((out != want).reshape(n, -1).any(axis=1))
            assert bad.size == 0, f"{mode} call {call}: {bad.size} bricks differ, first {bad[:8].tolist()}"
        for i in np.random.default_rng(3).choice(n, size=16, replace=False):
            assert np.array_equal(out[i], oracle.decode_brick(enc, int(i)))
    finally:
        vol.release()


def test_random_order_duplicates_and_scattered_slots(small_volume):
    enc = oracle.encode_volume(small_volume, 3, coder=1)
    n = oracle.header(enc)["n_bricks"]
    rng = np.random.default_rng(1)
    ids = rng.integers(0, n, size=300)
    slots = rng.permutation(1000)[:300]
    for mode in MODES:
        out, st = gpu_decode(enc, ids, 0, mode, slots=slots)
        assert st[0] == 0
        for i, s in zip(ids, slots):
            assert np.array_equal(out[s], oracle.decode_brick(enc, int(i)))


@pytest.mark.parametrize("coder", [0, 1])
def test_large_request_runs_longest_first_with_the_same_result(coder):
    """Requests of 1024 items or more run in size-aware order (longest record first) in the grid
    and batched schedules: duplicates, scattered slots and an out-of-range id (reported with its
    own item index) give the same result as in request order."""
    V = synth.fill(synth.small(dims=(128, 128, 96), seed=21, grid=16, diameter=12.0, bg=0.2))
    enc = vc.vc_encode_volume(V, 4, op_mask=0x7F, coder=coder)
    n = oracle.header(enc)["n_bricks"]  # 384 bricks of 16^3, of varied record sizes
    rng = np.random.default_rng(5)
    ids = rng.integers(0, n, size=1500)
    ids[777] = n + 3
    slots = rng.permutation(2000)[:1500]
    ref = oracle_bricks(enc, np.arange(n), 0)
    for mode in ("grid", "batched", "plain"):
        out, st = gpu_decode(enc, ids, 0, mode, slots=slots)
        assert st[0] == vc.VC_ERR_ARG and st[1] == 777, (mode, st)
        for k in range(0, 1500, 7):
            if k != 777:
                assert np.array_equal(out[slots[k]], ref[ids[k]]), (mode, k)


def test_empty_request_is_noop(small_volume):
    enc = oracle.encode_volume(small_volume, 3)
    vol = vc.Volume(enc)
    try:
        z = torch.zeros(1, dtype=torch.int32, device="cuda")
        st = torch.zeros(4, dtype=torch.int32, device="cuda")
        vc.vc_decode_bricks(vol.handle, z.data_ptr(), 0, z.data_ptr(), z.data_ptr(), 0, 2, st.data_ptr(), 0)
        torch.cuda.synchronize()
        assert st.cpu()[0] == 0
    finally:
        vol.release()


def test_out_of_range_brick_id_reports_arg(small_volume):
    enc = oracle.encode_volume(small_volume, 3)
    n = oracle.header(enc)["n_bricks"]
    for mode in MODES:
        out, st = gpu_decode(enc, [0, 1, n + 5, 2], 0, mode)
        assert st[0] == vc.VC_ERR_ARG and st[1] == 2
        assert np.array_equal(out[0], oracle.decode_brick(enc, 0))
        assert np.array_equal(out[3], oracle.decode_brick(enc, 2))


def test_host_entry_point_matches_device_path(small_volume):
    """Pageable output goes through a device staging buffer and a copy; pinned (mapped) output is
    written by the decode kernels directly. Both give the oracle's labels, in every schedule."""
    enc = oracle.encode_volume(small_volume, 4, coder=1)
    n = oracle.header(enc)["n_bricks"]
    vol = vc.Volume(enc)
    try:
        ids = np.arange(n, dtype=np.uint32)[::-1].copy()
        for lod in (0, 1):
            e = 16 >> lod
            ref = oracle_bricks(enc, ids, lod)
            for pinned in (False, True):
                for mode in (vc.VC_MODE_BATCHED, vc.VC_MODE_GRID, vc.VC_MODE_PIPELINED):
                    if pinned:
                        buf = torch.full((n * e ** 3,), -1, dtype=torch.int32, pin_memory=True)
                        labels = buf.numpy().view(np.uint32).reshape(n, e, e, e)
                    else:
                        labels = np.full((n, e, e, e), 0xFFFFFFFF, dtype=np.uint32)
                    st = vc.vc_decode_bricks_host(vol.handle, ids, lod, mode, labels)
                    assert st == 0
                    assert np.array_equal(labels, ref), (lod, pinned, mode)
    finally:
        vol.release()


def test_garbage_coded_words_in_every_record_are_reported_not_faulted():
    """Random bytes in place of every record's coded words (headers, states and palettes intact):
    every brick decodes from garbage symbols, whose parse claims node and stop-0 counts no brick of
    the volume has (rank lists cut, node counts beyond the layout, neighbour chains through cells
    left unset). Every schedule and three levels of detail report VC_ERR_CORRUPT without a fault,
    and the intact volume decodes to the oracle afterwards in the same context."""
    V = synth.fill(synth.small(dims=(128, 128, 96), seed=12, grid=16, diameter=19.0, bg=0.1))
    enc = vc.vc_encode_volume(V, 5, op_mask=0x7F, coder=1)
    h = oracle.header(enc)
    n = h["n_bricks"]
    rec_off = (128 + 4 * (n + 1) + 15) & ~15
    lib = oracle._load()
    rng = np.random.default_rng(8)
    bad = enc.copy()
    for i in range(n):
        r = oracle.brick_record(enc, i)
        hw = int(lib.oracle_head_words(1, 0, r["n_sym"]))
        at = rec_off + 4 * r["offset_words"] + 16 + 4 * hw + 4 * r["n_pal"]
        bad[at: at + r["coded_bytes"]] = rng.integers(0, 256, r["coded_bytes"], dtype=np.uint8)
    for lod in (0, 1, 2):
        for mode in ("grid", "batched", "pipelined"):
            _, st = gpu_decode(bad, np.arange(n), lod, mode)
            assert st[0] == vc.VC_ERR_CORRUPT, (lod, mode, st)
    torch.cuda.synchronize()
    out, st = gpu_decode(enc, np.arange(n), 0, "grid")
    assert st[0] == 0
    assert np.array_equal(out, oracle_bricks(enc, np.arange(n), 0))


# ------------------------------------------------------------------ brute force

def _tiny_bricks():
    rng = np.random.default_rng(11)
    out = []
    for b in (2, 4):
        for n_labels in (1, 2, 3):
            for _ in range(3):
                if b == 2:
                    B = rng.integers(1, n_labels + 1, size=(2, 2, 2)).astype(np.uint32)
                else:
                    B = np.repeat(np.repeat(np.repeat(rng.integers(1, n_labels + 1, size=(2, 2, 2)), 2, 0), 2, 1), 2, 2)
                    B = B.astype(np.uint32)
                    B[rng.integers(0, 4), rng.integers(0, 4), rng.integers(0, 4)] = rng.integers(1, n_labels + 1)
                out.append(B)
    return out


@pytest.mark.parametrize("coder", [0, 1])
def test_brute_force_streams_decode_on_gpu(coder):
    rng = random.Random(5)
    for B in _tiny_bricks():
        L = B.shape[0].bit_length() - 1
        en = StreamEnumerator(B)
        streams = en.count_and_enumerate(limit=2000) if B.shape[0] == 2 else None
        if streams is None:
            streams = [en.sample(rng) for _ in range(300)]
        enc = oracle.pack_bricks(L, streams, coder=coder)
        for mode in ("grid", "batched"):
            out, st = gpu_decode(enc, np.arange(len(streams)), 0, mode)
            assert st[0] == 0
            assert (out == B[None]).all()
        # every level of detail agrees with the oracle replay of the same streams
        for lod in range(1, L + 1):
            out, st = gpu_decode(enc, np.arange(len(streams)), lod, "batched")
            assert st[0] == 0
            assert np.array_equal(out, oracle_bricks(enc, range(len(streams)), lod))


# ------------------------------------------------------------------ corruption

def _corrupt_cases():
    g = load_golden("brick4_x1_neighbours.txt")
    sym = [int(s) for s in g["symbols"]]
    pal = [int(p) for p in g["palette"]]
    cases = []
    s = list(sym); s[5] = 7; cases.append((s, pal, 0, 0x7F, 0))
    cases.append((sym, pal, 0, 0x7F & ~(1 << OP_NY), 0))
    s = list(sym); s[0] = OP_PARENT; cases.append((s, pal, 0, 0x7F, 0))
    s = list(sym); s[0] = OP_LAST; cases.append((s, pal, 0, 0x7F, 0))
    s = list(sym); s[12] = OP_NY; cases.append((s, pal, 0, 0x7F, 0))
    s = list(sym); s[2] = OP_ADV; cases.append((s, pal, 0, 0x7F, 0))
    cases.append((sym, pal + [7], 0, 0x7F, 0))
    s = list(sym); s[10] = OP_LAST | 8; cases.append((s, pal, 0, 0x7F, 0))
    cases.append((sym + [0], pal, 0, 0x7F, 0))
    cases.append((sym[:-1], pal, 0, 0x7F, 0))
    cases.append((sym, pal, 1, 0x7F, 0))
    s = list(sym[:10]) + [OP_DELTA, 3] + sym[11:]; cases.append((s, pal, 1, 0x7F, 0))
    s = list(sym[:10]) + [OP_DELTA, 0] + sym[11:]; cases.append((s, pal, 1, 0x7F, 0))
    s = list(sym[:10]) + [OP_DELTA] + [8] * 7 + [1] + sym[11:]; cases.append((s, pal, 1, 0x7F, 0))
    s = list(sym[:-1]) + [OP_DELTA, 9]; cases.append((s, pal, 1, 0x7F, 0))
    cases.append((sym, pal, 0, 0x7F, 1))
    return sym, pal, cases


@pytest.mark.parametrize("coder", [0, 1])
def test_corrupt_records_flagged_per_item(coder):
    sym, pal, cases = _corrupt_cases()
    for s, p, nd, mask, flags in cases:
        assert oracle.decode_brick_status(oracle.pack_single_brick(2, s, p, nd, op_mask=mask, flags=flags,
                                                                   coder=coder), 0) == oracle.ERR_CORRUPT
        # a valid brick, the corrupt one, a valid brick
        good = (sym, pal, 0)
        enc = oracle.pack_bricks(2, [good, (s, p, nd), good], op_mask=mask, coder=coder, flags=flags)
        if mask != 0x7F or flags:
            # the good stream itself violates the restricted mask / flags: use only the corrupt one
            enc = oracle.pack_bricks(2, [(s, p, nd)], op_mask=mask, coder=coder, flags=flags)
            for mode in MODES:
                _, st = gpu_decode(enc, [0], 0, mode)
                assert st[0] == vc.VC_ERR_CORRUPT and st[1] == 0, (s, mode)
            continue
        for mode in MODES:
            out, st = gpu_decode(enc, [0, 1, 2], 0, mode)
            assert st[0] == vc.VC_ERR_CORRUPT and st[1] == 1, (s, p, nd, mode, st)
            ref = oracle.decode_brick(enc, 0)
            assert np.array_equal(out[0], ref) and np.array_equal(out[2], ref)


def test_rans_corrupt_words_flagged():
    g = load_golden("brick4_x1_neighbours.txt")
    sym = [int(s) for s in g["symbols"]] * 1
    pal = [int(p) for p in g["palette"]]
    enc = oracle.pack_single_brick(2, sym, pal, 0, coder=1)
    rec = oracle.brick_record(enc, 0)
    rec_off = (128 + 8 + 15) & ~15
    # an initial state below 2^16 is invalid
    bad = enc.copy()
    bad[rec_off + 16: rec_off + 20] = 0
    assert oracle.decode_brick_status(bad, 0) == oracle.ERR_CORRUPT
    _, st = gpu_decode(bad, [0], 0, "batched")
    assert st[0] == vc.VC_ERR_CORRUPT
    assert rec["n_sym"] == len(sym)


def _many_label_volume(n_labels_per_brick_edge: int, edge: int, seed: int) -> np.ndarray:
    """A volume whose bricks hold many distinct labels: small cubes of side n with unique ids."""
    rng = np.random.default_rng(seed)
    s = n_labels_per_brick_edge
    cells = rng.permutation(np.arange(1, (edge // s) ** 3 + 1, dtype=np.uint32) * 2654435761 % 4294967291 + 1)
    grid = cells.reshape(edge // s, edge // s, edge // s).astype(np.uint32)
    return np.repeat(np.repeat(np.repeat(grid, s, 0), s, 1), s, 2)


@pytest.mark.parametrize("coder", [0, 1])
def test_parity_16bit_index_grids(coder):
    """Bricks with more than 251 labels take the 16-bit index grids: 2^3 cubes of distinct labels
    give 4096 labels per 32^3 brick; every brick, every level of detail, every schedule."""
    V = _many_label_volume(2, 64, 3)
    V[:, :, :8] = 7  # a few repeated labels and a constant slab too
    enc = vc.vc_encode_volume(V, 5, op_mask=0x7F, coder=coder)
    assert oracle.header(enc)["max_pal"] >= 252
    ids = np.arange(oracle.header(enc)["n_bricks"])
    for lod in (0, 1, 3, 5):
        ref = oracle_bricks(enc, ids, lod)
        for mode in MODES:
            out, st = gpu_decode(enc, ids, lod, mode)
            assert st[0] == 0, (mode, lod, st)
            assert np.array_equal(out, ref), (mode, lod)


@pytest.mark.parametrize("log2b", [3, 4])
def test_parity_all_distinct_worst_case(log2b):
    """Every voxel its own label: the largest palettes and streams a brick of this size can have."""
    b = 1 << log2b
    V = _many_label_volume(1, 2 * b, 11)
    for coder in (0, 1):
        enc = vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=coder)
        ids = np.arange(oracle.header(enc)["n_bricks"])
        out, st = gpu_decode(enc, ids, 0, "grid")
        assert st[0] == 0
        assert np.array_equal(out, oracle_bricks(enc, ids, 0))


@pytest.mark.parametrize("log2b,coder", [(4, 0), (5, 1), (6, 1), (3, 0)])
def test_coarsest_labels_straight_from_the_encoding(log2b, coder):
    """vc_coarsest_labels reads each brick's first palette entry without decoding: it equals the
    single label of a decode at lod = L (the top of the mode hierarchy), for every brick; an id out
    of range reports VC_ERR_ARG for its item."""
    V = synth.fill(synth.small(dims=(160, 96, 80), seed=40 + log2b, grid=16, diameter=18.0, bg=0.3))
    enc = vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=coder)
    n = oracle.header(enc)["n_bricks"]
    vol = vc.Volume(enc)
    try:
        ids_np = np.concatenate([np.arange(n), np.arange(n)[::-1]]).astype(np.uint32)
        ids = torch.from_numpy(ids_np.view(np.int32)).cuda()
        out = torch.full((ids_np.size,), -1, dtype=torch.int32, device="cuda")
        st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
        vc.vc_coarsest_labels(vol.handle, ids.data_ptr(), ids_np.size, out.data_ptr(), st.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert int(st[0]) == 0
        got = out.cpu().numpy().view(np.uint32)
        want = np.array([oracle.decode_brick(enc, int(i), log2b).reshape(-1)[0] for i in ids_np], dtype=np.uint32)
        assert np.array_equal(got, want)
        bad = torch.tensor([0, n + 1, 1], dtype=torch.int32, device="cuda")
        vc.vc_coarsest_labels(vol.handle, bad.data_ptr(), 3, out.data_ptr(), st.data_ptr(), 0)
        torch.cuda.synchronize()
        assert int(st[0]) == vc.VC_ERR_ARG and int(st[1]) == 1 and int(out[1]) == 0
    finally:
        vol.release()


@pytest.mark.parametrize("coder", [0, 1])
def test_parity_short_delta_variant(small_volume, coder):
    """Limited delta (flags bit 1: one 4-bit entry per delta operation holding delta - 1,
    2 <= delta <= 16): every brick, several levels of detail, every schedule, on a volume whose
    palettes need re-appended labels and on the small workload; a hand-packed brick that reaches
    delta = 16; delta operations without their entry or with an invalid one (entry 0, or delta
    beyond the palette cursor) are flagged for exactly their item."""
    from test_oracle import reuse_volume
    F = oracle.FLAG_SHORT_DELTA
    for V, log2b in ((reuse_volume(), 3), (reuse_volume(), 5), (small_volume, 4)):
        enc = vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=coder, flags=F)
        n = oracle.header(enc)["n_bricks"]
        ids = np.arange(n)
        for lod in (0, 1, log2b):
            ref = oracle_bricks(enc, ids, lod)
            for mode in MODES:
                out, st = gpu_decode(enc, ids, lod, mode)
                assert st[0] == 0, (mode, lod, st)
                assert np.array_equal(out, ref), (log2b, mode, lod)
    sym, pal, _ = _corrupt_cases()
    good = (sym, pal, 0)
    for s in (list(sym[:-1]) + [OP_DELTA], list(sym[:10]) + [OP_DELTA, 9] + sym[11:],
              list(sym[:10]) + [OP_DELTA, 0] + sym[11:], list(sym[:10]) + [OP_DELTA, 2] + sym[11:]):
        enc = oracle.pack_bricks(2, [good, (s, pal, 1), good], coder=coder, flags=F)
        assert oracle.decode_brick_status(enc, 1) == oracle.ERR_CORRUPT
        for mode in MODES:
            out, st = gpu_decode(enc, [0, 1, 2], 0, mode)
            assert st[0] == vc.VC_ERR_CORRUPT and st[1] == 1, (s, mode, st)
    legal = list(sym[:10]) + [OP_DELTA, 1] + sym[11:]
    pal16 = [1000 + 13 * i for i in range(17)]
    sym16 = [OP_ADV] * 17 + [OP_DELTA, 15] + [0] * 55  # delta 16 re-reads palette[1]
    enc = oracle.pack_bricks(2, [good, (legal, pal, 1), (sym16, pal16, 1)], coder=coder, flags=F)
    ref = oracle_bricks(enc, [0, 1, 2], 0)
    assert int(ref[2].reshape(4, 4, 4)[0, 0, 2]) == pal16[1]
    for mode in MODES:
        out, st = gpu_decode(enc, [0, 1, 2], 0, mode)
        assert st[0] == 0 and np.array_equal(out, ref), mode
