"""The serving runtime on the GPU, through the C ABI: requests decode into the server's cache
bit-exactly as the oracle does; a request's result is the same alone and in a mix of concurrent
requests (continuous batching, shared batches, evictions in between); admission waits for cache
memory; a corrupt brick fails its request without touching the others' results."""
import threading

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_36898_gb300 as vc  # noqa: E402

MiB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vc._lib_handle()


@pytest.fixture(scope="module")
def volumes():
    """Three volumes of different brick sizes and coders (the server serves them side by side)."""
    out = []
    for shape, log2b, coder, seed in (((128, 128, 128), 5, 1, 11), ((96, 64, 64), 4, 0, 12), ((64, 64, 64), 3, 1, 13)):
        spec = synth.small(dims=shape[::-1], seed=seed, grid=16, diameter=14.0, bg=0.15)
        V = synth.fill(spec)
        enc = vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=coder)
        out.append((V, enc, log2b))
    return out


def read_bricks(srv, offsets, edges):
    """Copies each brick (u32, x fastest) out of the server's cache."""
    ptr, nbytes = vc.vc_server_cache(srv)
    cache = _cache_view(ptr, nbytes)
    res = []
    for off, e in zip(offsets, edges):
        w0 = int(off) // 4
        res.append(cache[w0:w0 + e ** 3].cpu().numpy().view(np.uint32).reshape(e, e, e).copy())
    return res


_views = {}


def _cache_view(ptr, nbytes):
    """A torch view of device memory owned by the server (no copy)."""
    key = (ptr, nbytes)
    if key not in _views:
        class _Holder:
            __cuda_array_interface__ = {"shape": (nbytes // 4,), "typestr": "<i4", "data": (ptr, False), "version": 3}
        _views[key] = torch.as_tensor(_Holder(), device="cuda")
    return _views[key]


def make_server(volumes, cache_bytes, **kw):
    srv = vc.vc_server_create(cache_bytes, 0, **kw)
    vols = []
    for V, enc, log2b in volumes:
        h = vc.vc_load_compressed(enc, 0, torch.cuda.current_stream().cuda_stream)
        vols.append(h)
        vc.vc_server_add_volume(srv, h)
    return srv, vols


def close_server(srv, vols):
    vc.vc_release(srv)
    for h in vols:
        vc.vc_release(h)
    _views.clear()


def expected(volumes, vi, brick, lod):
    return oracle.decode_brick(volumes[vi][1], int(brick), int(lod))


def run_request(srv, vi, bricks, lods, log2b):
    rid = vc.vc_submit_bricks(srv, vi, bricks, lods)
    st = vc.vc_wait(srv, rid, 60000)
    assert st == vc.VC_REQ_DONE
    st, offs = vc.vc_poll(srv, rid, len(bricks))
    edges = [(1 << log2b) >> int(l) for l in lods]
    return rid, read_bricks(srv, offs, edges)


def test_request_alone_matches_oracle(volumes):
    srv, vols = make_server(volumes, 256 * MiB)
    try:
        rng = np.random.default_rng(1)
        for vi, (V, enc, log2b) in enumerate(volumes):
            nb = oracle.header(enc)["n_bricks"]
            bricks = rng.choice(nb, size=min(nb, 40), replace=False).astype(np.uint32)
            lods = rng.integers(0, min(3, log2b) + 1, size=bricks.size).astype(np.uint32)
            rid, got = run_request(srv, vi, bricks, lods, log2b)
            for g, b, l in zip(got, bricks, lods):
                assert np.array_equal(g, expected(volumes, vi, b, l)), (vi, b, l)
            info = vc.vc_request_info_get(srv, rid)
            assert info.n_bricks == bricks.size and info.t_done_ns >= info.t_admit_ns >= info.t_submit_ns
            vc.vc_request_release(srv, rid)
        # the same request again: every brick is a hit and nothing is decoded
        before = vc.vc_server_stats_get(srv)
        V, enc, log2b = volumes[0]
        rid = vc.vc_submit_bricks(srv, 0, np.arange(5, dtype=np.uint32), None)
        vc.vc_wait(srv, rid)
        vc.vc_request_release(srv, rid)
        rid = vc.vc_submit_bricks(srv, 0, np.arange(5, dtype=np.uint32), None)
        vc.vc_wait(srv, rid)
        assert vc.vc_request_info_get(srv, rid).hits == 5
        vc.vc_request_release(srv, rid)
        after = vc.vc_server_stats_get(srv)
        assert after.requests_done >= before.requests_done + 2
    finally:
        close_server(srv, vols)


def test_result_is_the_same_alone_and_in_a_mix(volumes):
    rng = np.random.default_rng(5)
    V, enc, log2b = volumes[0]
    nb = oracle.header(enc)["n_bricks"]
    probe = rng.choice(nb, size=24, replace=False).astype(np.uint32)
    probe_lods = rng.integers(0, 3, size=probe.size).astype(np.uint32)

    srv, vols = make_server(volumes, 256 * MiB)
    try:
        _, alone = run_request(srv, 0, probe, probe_lods, log2b)
    finally:
        close_server(srv, vols)

    # a small cache (evictions), small batches and several client threads, each holding one
    # request at a time
    srv, vols = make_server(volumes, 8 * MiB, max_batch_items=64, max_inflight=2)
    errors = []
    results = {}

    def client(tid):
        r = np.random.default_rng(100 + tid)
        try:
            for k in range(12):
                vi = int(r.integers(len(volumes)))
                Vv, encv, lb = volumes[vi]
                nbv = oracle.header(encv)["n_bricks"]
                bricks = r.choice(nbv, size=int(r.integers(1, min(nbv, 48))), replace=False).astype(np.uint32)
                lods = r.integers(0, min(2, lb) + 1, size=bricks.size).astype(np.uint32)
                if tid == 0 and k == 5:  # the probe request, in the middle of the mix
                    prid = vc.vc_submit_bricks(srv, 0, probe, probe_lods)
                    assert vc.vc_wait(srv, prid, 60000) == vc.VC_REQ_DONE
                    _, offs = vc.vc_poll(srv, prid, probe.size)
                    results["probe"] = read_bricks(srv, offs, [(1 << log2b) >> int(l) for l in probe_lods])
                    vc.vc_request_release(srv, prid)
                rid = vc.vc_submit_bricks(srv, vi, bricks, lods)
                assert vc.vc_wait(srv, rid, 60000) == vc.VC_REQ_DONE
                _, offs = vc.vc_poll(srv, rid, bricks.size)
                got = read_bricks(srv, offs, [(1 << lb) >> int(l) for l in lods])
                for g, b, l in zip(got[:4], bricks[:4], lods[:4]):
                    if not np.array_equal(g, expected(volumes, vi, b, l)):
                        errors.append((tid, k, vi, int(b), int(l)))
                vc.vc_request_release(srv, rid)
        except Exception as e:  # surfaced below
            errors.append(repr(e))

    try:
        threads = [threading.Thread(target=client, args=(t,)) for t in range(6)]
        for t in threads:
            t.start()
        for t in threads:
            t.join(120)
        assert not errors, errors[:5]
        assert "probe" in results
        for a, b in zip(alone, results["probe"]):
            assert np.array_equal(a, b)
        st = vc.vc_server_stats_get(srv)
        assert st.evictions > 0 and st.batches > 1 and st.requests_failed == 0
    finally:
        close_server(srv, vols)


def test_admission_waits_for_cache_memory(volumes):
    V, enc, log2b = volumes[0]  # b = 32: 128 KiB per finest brick
    srv, vols = make_server(volumes[:1], 6 * MiB, max_class=5)  # 48 bricks
    try:
        a = vc.vc_submit_bricks(srv, 0, np.arange(40, dtype=np.uint32))
        assert vc.vc_wait(srv, a, 60000) == vc.VC_REQ_DONE
        b = vc.vc_submit_bricks(srv, 0, np.arange(40, 64, dtype=np.uint32))  # 24 bricks, 8 free
        with pytest.raises(vc.VCError) as ex:
            vc.vc_wait(srv, b, 300)
        assert ex.value.code == vc.VC_ERR_TIMEOUT
        assert vc.vc_poll(srv, b)[0] == vc.VC_REQ_WAITING
        vc.vc_request_release(srv, a)  # frees 40 bricks' worth of evictable memory
        assert vc.vc_wait(srv, b, 60000) == vc.VC_REQ_DONE
        _, offs = vc.vc_poll(srv, b, 24)
        got = read_bricks(srv, offs, [32] * 24)
        for g, brick in zip(got, range(40, 64)):
            assert np.array_equal(g, expected(volumes, 0, brick, 0))
        assert vc.vc_server_stats_get(srv).evictions >= 16
        with pytest.raises(vc.VCError) as ex:  # larger than the whole cache: never admissible
            vc.vc_submit_bricks(srv, 0, np.arange(49, dtype=np.uint32))
        assert ex.value.code == vc.VC_ERR_BUSY
        vc.vc_request_release(srv, b)
    finally:
        close_server(srv, vols)


def test_corrupt_brick_fails_its_request(volumes):
    V, enc, log2b = volumes[1]  # plain coder: flip an operation nibble to the invalid code 7
    bad = enc.copy()
    h = oracle.header(enc)
    rec = oracle.brick_record(enc, 3)
    rec_off = (128 + 4 * (h["n_bricks"] + 1) + 15) & ~15
    coded = rec_off + 4 * (rec["offset_words"] + 4 + rec["n_pal"])
    # first coded byte of brick 3's stream: both nibbles become 7 (an invalid operation)
    bad[coded] = 0x77
    assert oracle.decode_brick_status(bad, 3, 0) == oracle.ERR_CORRUPT
    srv, vols = make_server([(V, bad, log2b)], 64 * MiB)
    try:
        r_bad = vc.vc_submit_bricks(srv, 0, np.array([3, 4], dtype=np.uint32))
        with pytest.raises(vc.VCError) as ex:
            vc.vc_wait(srv, r_bad, 60000)
        assert ex.value.code == vc.VC_ERR_CORRUPT
        assert vc.vc_request_info_get(srv, r_bad).state == vc.VC_REQ_FAILED
        vc.vc_request_release(srv, r_bad)
        ok = vc.vc_submit_bricks(srv, 0, np.array([4, 5], dtype=np.uint32))
        assert vc.vc_wait(srv, ok, 60000) == vc.VC_REQ_DONE
        _, offs = vc.vc_poll(srv, ok, 2)
        got = read_bricks(srv, offs, [1 << log2b] * 2)
        for g, b in zip(got, (4, 5)):
            assert np.array_equal(g, expected([(V, enc, log2b)], 0, b, 0))
        assert h["n_bricks"] > 5
        vc.vc_request_release(srv, ok)
    finally:
        close_server(srv, vols)


def test_graph_launched_batches_match_the_oracle(volumes):
    """With VC_SERVER_GRAPHS every batch is one CUDA graph; batches of a repeated shape update the
    graph in place. Results are the same bricks as without graphs."""
    srv, vols = make_server(volumes, 64 * MiB, max_batch_items=32, flags=vc.VC_SERVER_GRAPHS)
    try:
        rng = np.random.default_rng(9)
        for k in range(10):
            vi = k % len(volumes)
            V, enc, log2b = volumes[vi]
            nb = oracle.header(enc)["n_bricks"]
            bricks = rng.choice(nb, size=min(nb, 20), replace=False).astype(np.uint32)
            lods = np.zeros(bricks.size, dtype=np.uint32)
            rid, got = run_request(srv, vi, bricks, lods, log2b)
            for g, b in zip(got[:5], bricks[:5]):
                assert np.array_equal(g, expected(volumes, vi, b, 0))
            vc.vc_request_release(srv, rid)
        st = vc.vc_server_stats_get(srv)
        assert st.graph_launches == st.batches and st.batches >= 10
        assert st.graph_instantiations < st.graph_launches  # later batches updated an existing graph
        assert st.requests_failed == 0
    finally:
        close_server(srv, vols)


def test_waiting_request_reads_the_coarsest_level_from_the_encoding():
    """A request that cannot be admitted yet (the cache is full of another request's pinned bricks)
    gets each brick's coarsest level of detail straight from the encoding (Methods, "Memory
    management"): the oracle's decode at lod = L, brick by brick; once the other request is
    released it is admitted and decodes to the oracle's finest level."""
    spec = synth.small(dims=(64, 64, 64), seed=21, grid=16, diameter=12.0, bg=0.2)
    V = synth.fill(spec)
    enc = vc.vc_encode_volume(V, 4, op_mask=0x7F, coder=1)
    block = 4 * 16 ** 3
    srv = vc.vc_server_create(8 * block, 0, min_class=2, max_class=4)
    h = vc.vc_load_compressed(enc, 0, torch.cuda.current_stream().cuda_stream)
    try:
        vi = vc.vc_server_add_volume(srv, h)
        first = vc.vc_submit_bricks(srv, vi, np.arange(0, 8, dtype=np.uint32))
        assert vc.vc_wait(srv, first, 60000) == vc.VC_REQ_DONE
        ids = np.array([9, 17, 33, 8, 63, 40, 12, 50], dtype=np.uint32)
        waiting = vc.vc_submit_bricks(srv, vi, ids)
        assert vc.vc_poll(srv, waiting)[0] == vc.VC_REQ_WAITING
        labels = torch.full((ids.size,), -1, dtype=torch.int32, device="cuda")
        st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
        s = torch.cuda.current_stream()
        vc.vc_request_coarsest(srv, waiting, labels.data_ptr(), st.data_ptr(), s.cuda_stream)
        torch.cuda.synchronize()
        assert int(st[0]) == 0
        want = np.array([oracle.decode_brick(enc, int(i), 4).reshape(-1)[0] for i in ids], dtype=np.uint32)
        assert np.array_equal(labels.cpu().numpy().view(np.uint32), want)
        assert vc.vc_poll(srv, waiting)[0] == vc.VC_REQ_WAITING
        vc.vc_request_release(srv, first)
        assert vc.vc_wait(srv, waiting, 60000) == vc.VC_REQ_DONE
        offsets = vc.vc_poll(srv, waiting, ids.size)[1]
        got = read_bricks(srv, offsets, [16] * ids.size)
        for g, i in zip(got, ids):
            assert np.array_equal(g, oracle.decode_brick(enc, int(i)))
        vc.vc_request_release(srv, waiting)
    finally:
        vc.vc_release(srv)
        vc.vc_release(h)
        _views.clear()
