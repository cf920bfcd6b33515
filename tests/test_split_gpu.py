"""Detail split on the GPU, through the C ABI: a volume loaded with vc_load_compressed_split keeps
only its coarse levels in device memory; decodes at lod >= 1 read them, decodes at lod = 0 read the
whole records from pinned host memory mapped into the device. Every brick at every level of detail
equals the oracle's decode of the original encoding, in every schedule, through the host entry
point, the allocation-free entry point and the serving runtime."""
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


def decode(vol, ids, lod, mode, paletted=False):
    n = len(ids)
    ids_t = torch.as_tensor(np.asarray(ids, dtype=np.int64)).to(torch.int32).cuda()
    words = vc.vc_volume_slot_words(vol.handle, lod, True)[0] if paletted else vol.edge(lod) ** 3
    cache = torch.full((n * words,), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
    vol.decode(ids_t, torch.arange(n, dtype=torch.int32, device="cuda"), cache, lod,
               vc.MODES[mode] | (vc.VC_MODE_PALETTED if paletted else 0), st)
    torch.cuda.synchronize()
    return cache.cpu().numpy().view(np.uint32).reshape(n, words), st.cpu().numpy()


@pytest.mark.parametrize("log2b,coder,flags", [(5, 1, 0), (5, 0, 0), (3, 1, 2), (4, 0, 1), (6, 1, 0)])
def test_split_volume_every_lod_every_schedule(log2b, coder, flags):
    V = synth.fill(synth.small(dims=(160, 96, 80), seed=30 + log2b, grid=16, diameter=14.0, bg=0.25))
    enc = vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=coder, flags=flags)
    full = vc.Volume(enc)
    vol = vc.Volume(enc, split=True)
    try:
        info, finfo = vc.vc_volume_info_get(vol.handle), vc.vc_volume_info_get(full.handle)
        assert info.split == 1 and finfo.split == 0
        assert info.host_bytes >= enc.size and finfo.host_bytes == 0
        assert info.device_bytes < finfo.device_bytes  # the finest level stays on the host
        n = vol.n_bricks
        ids = np.arange(n)
        for lod in sorted({0, 1, 2, log2b}):
            e = vol.edge(lod)
            ref = np.stack([oracle.decode_brick(enc, i, lod) for i in ids]).reshape(n, -1)
            for mode in MODES:
                out, st = decode(vol, ids, lod, mode)
                assert st[0] == 0, (lod, mode, st)
                assert np.array_equal(out, ref), (lod, mode)
        # packed palette indices at the finest level (read from the host records)
        out, st = decode(vol, ids, 0, "batched", paletted=True)
        assert st[0] == 0
        words, bits, per = vc.vc_volume_slot_words(vol.handle, 0, True)
        v = np.arange(vol.b ** 3)
        for i in ids[:: max(1, n // 5)]:
            pal = oracle.brick_record(enc, int(i))["palette"]
            idx = ((out[i][v // per].astype(np.uint64) >> (bits * (v % per)).astype(np.uint64)) & ((1 << bits) - 1))
            assert np.array_equal(pal[idx.astype(np.int64)].reshape(vol.b, vol.b, vol.b), oracle.decode_brick(enc, int(i), 0))
        # the coarsest level of detail from the device copy
        ids_t = torch.arange(n, dtype=torch.int32, device="cuda")
        lab = torch.zeros(n, dtype=torch.int32, device="cuda")
        st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
        vc.vc_coarsest_labels(vol.handle, ids_t.data_ptr(), n, lab.data_ptr(), st.data_ptr(), 0)
        torch.cuda.synchronize()
        assert int(st[0]) == 0
        assert np.array_equal(lab.cpu().numpy().view(np.uint32),
                              np.array([oracle.decode_brick(enc, int(i), log2b).reshape(-1)[0] for i in ids], np.uint32))
    finally:
        vol.release()
        full.release()


def test_split_volume_host_entry_noalloc_and_server():
    V = synth.fill(synth.small(dims=(128, 128, 64), seed=77, grid=16, diameter=12.0, bg=0.2))
    enc = vc.vc_encode_volume(V, 5, op_mask=0x7F, coder=1)
    n = oracle.header(enc)["n_bricks"]
    h = vc.vc_load_compressed_split(enc, 0, 0)
    srv = vc.vc_server_create(32 << 20, 0, max_batch_items=64, flags=vc.VC_SERVER_GRAPHS)
    try:
        # host entry point at the finest level
        ids = np.arange(n, dtype=np.uint32)[::-1].copy()
        labels = np.zeros(n * 32 ** 3, dtype=np.uint32)
        assert vc.vc_decode_bricks_host(h, ids, 0, vc.VC_MODE_BATCHED, labels, 0) == 0
        for k in range(0, n, 5):
            assert np.array_equal(labels[k * 32 ** 3:(k + 1) * 32 ** 3].reshape(32, 32, 32),
                                  oracle.decode_brick(enc, int(ids[k]), 0))
        # allocation-free entry point, finest and coarser levels
        ids_t = torch.from_numpy(ids.view(np.int32)).cuda()
        for lod in (0, 2):
            e = 32 >> lod
            cache = torch.full((n * e ** 3,), -1, dtype=torch.int32, device="cuda")
            st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
            vc.vc_decode_bricks_noalloc(h, ids_t.data_ptr(), n, torch.arange(n, dtype=torch.int32, device="cuda").data_ptr(),
                                        cache.data_ptr(), lod, vc.VC_MODE_GRID, st.data_ptr(), 0)
            torch.cuda.synchronize()
            assert int(st[0]) == 0
            got = cache.cpu().numpy().view(np.uint32).reshape(n, e, e, e)
            for k in range(0, n, 7):
                assert np.array_equal(got[k], oracle.decode_brick(enc, int(ids[k]), lod))
        # serving: mixed levels of detail, graph-launched batches
        vc.vc_server_add_volume(srv, h)
        ptr, nbytes = vc.vc_server_cache(srv)

        class _H:
            __cuda_array_interface__ = {"shape": (nbytes // 4,), "typestr": "<i4", "data": (ptr, False), "version": 3}
        cache = torch.as_tensor(_H(), device="cuda")
        rng = np.random.default_rng(8)
        for _ in range(4):
            bricks = rng.choice(n, size=12, replace=False).astype(np.uint32)
            lods = rng.integers(0, 3, size=12).astype(np.uint32)
            rid = vc.vc_submit_bricks(srv, 0, bricks, lods)
            assert vc.vc_wait(srv, rid, 60000) == vc.VC_REQ_DONE
            _, offs = vc.vc_poll(srv, rid, 12)
            for b, l, o in zip(bricks, lods, offs):
                e = 32 >> int(l)
                got = cache[int(o) // 4:int(o) // 4 + e ** 3].cpu().numpy().view(np.uint32).reshape(e, e, e)
                assert np.array_equal(got, oracle.decode_brick(enc, int(b), int(l)))
            vc.vc_request_release(srv, rid)
        assert vc.vc_server_stats_get(srv).requests_failed == 0
    finally:
        vc.vc_release(srv)
        vc.vc_release(h)
