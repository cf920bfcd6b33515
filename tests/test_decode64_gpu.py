"""GPU parity for 64^3 bricks (L = 6), through the C ABI.

A 64^3 brick's working set (node operations, cursor masks, level grids, the 64^3 index grid) is
beyond a thread block's shared memory, so these bricks are decoded by persistent blocks that keep
its large parts in global scratch slices and the rest in shared memory. Bit-exact against the CPU oracle on every brick of ragged volumes,
both coders, every schedule and thread count, several levels of detail, 8- and 16-bit index
grids, cache paletting, the allocation-free entry point, the serving runtime with graph-launched
batches, and per-item error reporting.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_36898_gb300 as vc  # noqa: E402

MODES = ["plain", "grid", "batched", "pipelined"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vc._lib_handle()


@pytest.fixture(scope="module")
def ragged():
    """160 x 96 x 80 voxels: 3 x 2 x 2 bricks of 64^3, each axis with a partial last brick."""
    return synth.fill(synth.small(dims=(160, 96, 80), seed=64, grid=16, diameter=20.0, bg=0.3))


def _many_label_volume(side: int, edge: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    cells = rng.permutation(np.arange(1, (edge // side) ** 3 + 1, dtype=np.uint64) * 2654435761 % 4294967291 + 1)
    grid = cells.reshape(edge // side, edge // side, edge // side).astype(np.uint32)
    return np.repeat(np.repeat(np.repeat(grid, side, 0), side, 1), side, 2)


def decode(vol, ids, lod=0, mode="batched", slots=None, paletted=False):
    n = len(ids)
    ids_t = torch.as_tensor(np.asarray(ids, dtype=np.int64)).to(torch.int32).cuda()
    slots = np.arange(n) if slots is None else np.asarray(slots)
    slots_t = torch.as_tensor(slots.astype(np.int64)).to(torch.int32).cuda()
    if paletted:
        words = vc.vc_volume_slot_words(vol.handle, lod, True)[0]
    else:
        words = vol.edge(lod) ** 3
    nslots = int(slots.max()) + 1
    cache = torch.full((nslots * words,), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
    m = vc.MODES[mode] | (vc.VC_MODE_PALETTED if paletted else 0)
    vol.decode(ids_t, slots_t, cache, lod, m, st)
    torch.cuda.synchronize()
    return cache.cpu().numpy().view(np.uint32).reshape(nslots, words), st.cpu().numpy()


def oracle_bricks(enc, ids, lod):
    return np.stack([oracle.decode_brick(enc, int(i), lod) for i in ids])


@pytest.mark.parametrize("coder", [0, 1])
def test_b64_parity_every_brick_every_schedule(ragged, coder):
    enc = vc.vc_encode_volume(ragged, 6, op_mask=0x7F, coder=coder)
    vol = vc.Volume(enc)
    try:
        info = vc.vc_volume_info_get(vol.handle)
        assert info.brick_size == 64 and 0 < info.smem_bytes <= 227 * 1024  # the small regions only
        assert vc.vc_volume_get_schedule(vol.handle)[0] == 1024
        ids = np.arange(vol.n_bricks)
        for lod in (0, 1, 2, 4, 6):
            ref = oracle_bricks(enc, ids, lod)
            e = 64 >> lod
            for mode in MODES:
                out, st = decode(vol, ids, lod, mode)
                assert st[0] == 0, (mode, lod, st)
                assert np.array_equal(out.reshape(-1, e, e, e), ref), (mode, lod)
    finally:
        vol.release()


@pytest.mark.parametrize("threads,blocks_per_sm", [(256, 0), (256, 1), (1024, 2), (512, 3)])
def test_b64_thread_counts_and_grid_sizes(ragged, threads, blocks_per_sm):
    enc = vc.vc_encode_volume(ragged, 6, op_mask=0x7F, coder=1)
    vol = vc.Volume(enc)
    try:
        vc.vc_volume_set_schedule(vol.handle, threads, 1, blocks_per_sm)
        # duplicates and scattered slots: 30 items over 12 bricks
        rng = np.random.default_rng(threads + blocks_per_sm)
        ids = rng.integers(0, vol.n_bricks, size=30)
        slots = rng.permutation(40)[:30]
        out, st = decode(vol, ids, 0, "batched", slots=slots)
        assert st[0] == 0
        ref = oracle_bricks(enc, np.arange(vol.n_bricks), 0).reshape(vol.n_bricks, -1)
        for i, s in zip(ids, slots):
            assert np.array_equal(out[s], ref[i])
    finally:
        vol.release()


@pytest.fixture(scope="module")
def dense():
    """128 x 128 x 64 voxels of ~19-voxel cells: 4 bricks of 64^3 with up to ~98k nodes each, too
    many for every region of a brick to fit one block's shared memory."""
    return synth.fill(synth.small(dims=(128, 128, 64), seed=66, grid=16, diameter=19.0, bg=0.1))


@pytest.mark.parametrize("threads", [1024, 512, 256])
def test_b64_scratch_layout_with_regions_in_shared_memory(dense, threads):
    """Bricks beyond the all-in-shared-memory layout keep their large regions in a scratch slice,
    and the shared memory a block leaves over takes some of them back (1024 threads: children and
    node operations; 512: delta values; 256: none): every brick, label and packed-index output,
    levels 0 and 1, grid and batched schedules, 1 and 4 rANS runs, against the oracle."""
    for flags in (0, oracle.runs_flag(4)):
        enc = vc.vc_encode_volume(dense, 6, op_mask=0x7F, coder=1, flags=flags)
        n = oracle.header(enc)["n_bricks"]
        assert max(len(oracle.brick_nodes(enc, i)) for i in range(n)) > 60000
        vol = vc.Volume(enc)
        try:
            vc.vc_volume_set_schedule(vol.handle, threads, 1, 0)
            for lod in (0, 1):
                ref = oracle_bricks(enc, range(n), lod)
                for mode in ("grid", "batched"):
                    out, st = decode(vol, list(range(n)), lod, mode)
                    assert st[0] == 0, (threads, flags, lod, mode, st)
                    assert np.array_equal(out.reshape(ref.shape), ref), (threads, flags, lod, mode)
            out, st = decode(vol, list(range(n)), 0, "grid", paletted=True)
            assert st[0] == 0
            _, bits, per = vc.vc_volume_slot_words(vol.handle, 0, True)
            v = np.arange(64 ** 3)
            for i in range(n):
                pal = oracle.brick_record(enc, i)["palette"]
                w = out[i][v // per].astype(np.uint64)
                idx = ((w >> (bits * (v % per)).astype(np.uint64)) & ((1 << bits) - 1)).astype(np.int64)
                assert np.array_equal(pal[idx].reshape(64, 64, 64), oracle.decode_brick(enc, i, 0)), (threads, flags, i)
        finally:
            vol.release()


@pytest.mark.parametrize("which", ["ragged", "dense"])
def test_b64_garbage_coded_words_are_reported_not_faulted(which, ragged, dense):
    """Random bytes in place of every record's coded words (headers, states, run starts and
    palettes intact), in both layouts (everything in shared memory; a scratch slice with some
    regions in shared memory) and with 1 and 4 rANS runs: every schedule at levels 0 and 1
    reports VC_ERR_CORRUPT without a fault, and the intact volume decodes to the oracle afterwards."""
    V = ragged if which == "ragged" else dense
    lib = oracle._load()
    rng = np.random.default_rng(9)
    for flags in (0, oracle.runs_flag(4)):
        enc = vc.vc_encode_volume(V, 6, op_mask=0x7F, coder=1, flags=flags)
        n = oracle.header(enc)["n_bricks"]
        rec_off = (128 + 4 * (n + 1) + 15) & ~15
        bad = enc.copy()
        for i in range(n):
            r = oracle.brick_record(enc, i)
            hw = int(lib.oracle_head_words(1, flags, r["n_sym"]))
            at = rec_off + 4 * r["offset_words"] + 16 + 4 * hw + 4 * r["n_pal"]
            bad[at: at + r["coded_bytes"]] = rng.integers(0, 256, r["coded_bytes"], dtype=np.uint8)
        vol = vc.Volume(bad)
        try:
            for lod in (0, 1):
                for mode in ("grid", "batched"):
                    _, st = decode(vol, list(range(n)), lod, mode)
                    assert st[0] == vc.VC_ERR_CORRUPT, (which, flags, lod, mode, st)
        finally:
            vol.release()
        good = vc.Volume(enc)
        try:
            out, st = decode(good, list(range(n)), 0, "grid")
            assert st[0] == 0
            assert np.array_equal(out.reshape(n, 64, 64, 64), oracle_bricks(enc, range(n), 0))
        finally:
            good.release()


@pytest.mark.parametrize("coder", [0, 1])
def test_b64_16bit_index_grids(coder):
    """2^3 cubes of distinct labels: 32768 labels per 64^3 brick (16-bit grids, palettes read from
    the encoding), plus a constant slab."""
    V = _many_label_volume(2, 128, 5)
    V[:, :, :16] = 9
    enc = vc.vc_encode_volume(V, 6, op_mask=0x7F, coder=coder)
    assert oracle.header(enc)["max_pal"] >= 252
    vol = vc.Volume(enc)
    try:
        ids = np.arange(vol.n_bricks)
        for lod in (0, 1, 3):
            ref = oracle_bricks(enc, ids, lod)
            e = 64 >> lod
            for mode in ("grid", "plain"):
                out, st = decode(vol, ids, lod, mode)
                assert st[0] == 0, (mode, lod, st)
                assert np.array_equal(out.reshape(-1, e, e, e), ref), (mode, lod)
    finally:
        vol.release()


def test_b64_palettes_beyond_16_bits_are_refused():
    """Every voxel its own label gives 262144-entry palettes: more than 16-bit index grids hold."""
    V = _many_label_volume(1, 64, 6)
    enc = vc.vc_encode_volume(V, 6, op_mask=0x7F, coder=0)
    with pytest.raises(vc.VCError) as ex:
        vc.vc_load_compressed(enc, 0, 0)
    assert ex.value.code == vc.VC_ERR_UNSUPPORTED


@pytest.mark.parametrize("coder", [0, 1])
def test_b64_paletted_slots(ragged, coder):
    enc = vc.vc_encode_volume(ragged, 6, op_mask=0x7F, coder=coder)
    vol = vc.Volume(enc)
    try:
        ids = np.arange(vol.n_bricks)
        for lod in (0, 2):
            e = 64 >> lod
            words, bits, per = vc.vc_volume_slot_words(vol.handle, lod, True)
            out, st = decode(vol, ids, lod, "batched", paletted=True)
            assert st[0] == 0
            v = np.arange(e ** 3)
            for i in ids:
                pal = oracle.brick_record(enc, int(i))["palette"]
                w = out[i][v // per].astype(np.uint64)
                idx = ((w >> (bits * (v % per)).astype(np.uint64)) & ((1 << bits) - 1)).astype(np.int64)
                assert np.array_equal(pal[idx].reshape(e, e, e), oracle.decode_brick(enc, int(i), lod)), (lod, i)
    finally:
        vol.release()


def test_b64_corrupt_brick_is_flagged_alone(ragged):
    enc = vc.vc_encode_volume(ragged, 6, op_mask=0x7F, coder=0)
    h = oracle.header(enc)
    bad = enc.copy()
    # brick 1's first symbol (the root) becomes the invalid operation 7
    starts = np.frombuffer(enc[128:128 + 4 * (h["n_bricks"] + 1)].tobytes(), dtype="<u4")
    rec_off = (128 + 4 * (h["n_bricks"] + 1) + 15) & ~15
    r = rec_off + 4 * int(starts[1])
    n_pal = int(np.frombuffer(enc[r:r + 4].tobytes(), dtype="<u4")[0])
    c = r + 16 + 4 * n_pal
    bad[c] = (bad[c] & 0xF0) | 7
    assert oracle.decode_brick_status(bad, 1) == oracle.ERR_CORRUPT
    assert oracle.decode_brick_status(bad, 0) == 0
    vol = vc.Volume(bad)
    try:
        for mode in MODES:
            out, st = decode(vol, [0, 1, 2], 0, mode)
            assert st[0] == vc.VC_ERR_CORRUPT and st[1] == 1, (mode, st)
            assert np.array_equal(out[0].reshape(64, 64, 64), oracle.decode_brick(enc, 0, 0))
            assert np.array_equal(out[2].reshape(64, 64, 64), oracle.decode_brick(enc, 2, 0))
        out, st = decode(vol, [0, 99], 0, "batched")
        assert st[0] == vc.VC_ERR_ARG and st[1] == 1
    finally:
        vol.release()


def test_b64_noalloc_matches_decode(ragged):
    enc = vc.vc_encode_volume(ragged, 6, op_mask=0x7F, coder=1)
    vol = vc.Volume(enc)
    try:
        n = vol.n_bricks
        ids = torch.arange(n, dtype=torch.int32, device="cuda")
        ref = torch.full((n * 64 ** 3,), -1, dtype=torch.int32, device="cuda")
        got = torch.full((n * 64 ** 3,), -1, dtype=torch.int32, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        for mode in (vc.VC_MODE_GRID, vc.VC_MODE_BATCHED):
            st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
            st2 = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
            vc.vc_decode_bricks(vol.handle, ids.data_ptr(), n, ids.data_ptr(), ref.data_ptr(), 0, mode, st.data_ptr(), s)
            vc.vc_decode_bricks_noalloc(vol.handle, ids.data_ptr(), n, ids.data_ptr(), got.data_ptr(), 0, mode,
                                        st2.data_ptr(), s)
            torch.cuda.synchronize()
            assert int(st[0]) == 0 and int(st2[0]) == 0
            assert torch.equal(ref, got)
        want = oracle_bricks(enc, np.arange(n), 0)
        assert np.array_equal(got.cpu().numpy().view(np.uint32).reshape(n, 64, 64, 64), want)
    finally:
        vol.release()


def test_b64_server_graph_batches(ragged):
    encs = [vc.vc_encode_volume(ragged, 6, op_mask=0x7F, coder=c) for c in (1, 0)]
    srv = vc.vc_server_create(64 << 20, 0, max_batch_items=16, flags=vc.VC_SERVER_GRAPHS)
    hs = []
    try:
        for enc in encs:
            h = vc.vc_load_compressed(enc, 0, 0)
            hs.append(h)
            vc.vc_server_add_volume(srv, h)
        ptr, nbytes = vc.vc_server_cache(srv)

        class _H:
            __cuda_array_interface__ = {"shape": (nbytes // 4,), "typestr": "<i4", "data": (ptr, False), "version": 3}
        cache = torch.as_tensor(_H(), device="cuda")
        rng = np.random.default_rng(64)
        for k in range(6):
            vi = k % 2
            bricks = rng.choice(12, size=8, replace=False).astype(np.uint32)
            lods = rng.integers(0, 3, size=8).astype(np.uint32)
            rid = vc.vc_submit_bricks(srv, vi, bricks, lods)
            assert vc.vc_wait(srv, rid, 60000) == vc.VC_REQ_DONE
            _, offs = vc.vc_poll(srv, rid, 8)
            for b, l, o in zip(bricks, lods, offs):
                e = 64 >> int(l)
                got = cache[int(o) // 4:int(o) // 4 + e ** 3].cpu().numpy().view(np.uint32).reshape(e, e, e)
                assert np.array_equal(got, oracle.decode_brick(encs[vi], int(b), int(l))), (k, b, l)
            vc.vc_request_release(srv, rid)
        st = vc.vc_server_stats_get(srv)
        assert st.requests_failed == 0 and st.graph_launches == st.batches
    finally:
        vc.vc_release(srv)
        for h in hs:
            vc.vc_release(h)
