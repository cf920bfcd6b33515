"""The frame cache (vc_frame_*) on the GPU against the frame cache oracle (oracle/frame_cache.py)
frame by frame: the marks (from the request stage's brick rays, or from the renderer's rays) give
the visible bricks, the camera oracle their levels; every frame's counts (requested, freed,
resident, assigned per level, top, dead labels, free-stack entries, pending reset) equal the
oracle's; resident bricks keep their regions; the newly cached bricks of a level are that many of
its requested bricks; every region is aligned, inside the buffer and disjoint from the others; and
every cached brick's labels equal the CSGV oracle's decode at its level. Cameras move between
frames; small caches force top overflow, defragmentation resets, full free stacks and the
per-frame limit."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import frame_cache as fm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_36898_gb300 as vc  # noqa: E402

NONE = fm.NONE


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vc._lib_handle()


class _Dev:
    """Zero-copy torch view of library-owned device memory (CUDA array interface)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (int(ptr), False), "version": 3}


def _host(ptr: int, n: int, typestr: str, dtype) -> np.ndarray:
    torch.cuda.synchronize()
    return torch.as_tensor(_Dev(ptr, n, typestr), device="cuda").cpu().numpy().view(dtype).copy()


def _read(view, with_cache=True):
    n = view.n_bricks
    offsets = _host(view.offsets, n, "<i8", np.uint64)
    lods = _host(view.lods, n, "|u1", np.uint8)
    cache = _host(view.cache, int(view.cache_words), "<i4", np.uint32) if with_cache else None
    return offsets, lods, cache


def _orbit(i, f, dims, W, H, fov=0.6):
    """Camera i of frame f: near for three frames, then far for three (the levels switch), its
    target wandering around the centre."""
    c = np.asarray(dims, np.float64) / 2
    a = 1.3 * i + 0.5 * f
    r = (0.8 if (f // 3) % 2 == 0 else 2.2) * max(dims) + 7.0 * i
    pos = (c[0] + r * math.cos(a), c[1] + 0.3 * r, c[2] + r * math.sin(a))
    tgt = (c[0] + 25 * math.sin(0.9 * f + i), c[1], c[2] + 20 * math.cos(0.7 * f))
    look = tuple(float(tgt[k] - pos[k]) for k in range(3))
    return (tuple(float(x) for x in pos), look, (0.0, 1.0, 0.0), fov, W, H)


def _want(enc, cams, max_lod, visible):
    """Per brick: the finest level over the cameras for visible bricks, NONE otherwise."""
    w = np.full(visible.size, NONE, np.uint8)
    if not visible.any():
        return w
    lv = np.min(np.stack([oracle.brick_lods(enc, *c, max_lod=max_lod) for c in cams]), axis=0)
    w[visible] = lv[visible]
    return w


def _brick_marks(enc, cams):
    n = oracle.header(enc)["n_bricks"]
    vis = np.zeros(n, bool)
    for c in cams:
        ids, _ = oracle.camera_bricks(enc, *c)
        vis[ids] = True
    return vis


def _check_frame(enc, L, cfg, state, want, prev, now, stats, decoded_cache):
    """Compares one GPU frame with the oracle's; returns the oracle state for the next frame."""
    r = fm.update(state, want, L=L, **cfg)
    off0, lod0 = prev
    off, lod, cache = now
    assert stats.last_requested == len(r["requested"])
    assert stats.last_freed == len(r["freed"])
    assert stats.last_resident == len(r["resident"])
    assert stats.last_decoded == sum(r["assign_n"])
    assert stats.last_unassigned == len(r["requested"]) - sum(r["assign_n"])
    assert (stats.top_words, stats.dead_words, bool(stats.reset_pending)) == (r["top"], r["dead"], r["reset_pending"])
    for lev in range(L + 1):
        assert stats.free_entries[lev] == min(r["free_n"][lev], cfg["free_cap"]), lev
    # resident bricks keep their regions (unless this frame reset the cache)
    if not r["in_reset"]:
        res = r["resident"]
        assert np.array_equal(lod[res], lod0[res]) and np.array_equal(off[res], off0[res])
    else:
        assert len(r["resident"]) == 0
    # newly cached bricks per level: assign_n of that level's requests
    new = np.zeros(lod.size, bool)
    new[r["requested"]] = lod[r["requested"]] != NONE
    for lev in range(L + 1):
        got = np.flatnonzero(new & (lod == lev))
        assert got.size == r["assign_n"][lev], (lev, got.size, r["assign_n"][lev])
        assert np.isin(got, r["requested_at"][lev]).all()
    cached = lod != NONE
    assert np.array_equal(cached, np.isin(np.arange(lod.size), np.concatenate([r["resident"], np.flatnonzero(new)])))
    assert (off[~cached] == np.uint64(2 ** 64 - 1)).all()
    # regions: aligned, inside [0, top), disjoint
    ids = np.flatnonzero(cached)
    sz = np.array([fm.region(L, int(lod[b])) for b in ids], np.uint64)
    o = off[ids]
    assert (o % sz == 0).all() and (o + sz <= np.uint64(r["top"])).all()
    order = np.argsort(o)
    assert (o[order][1:] >= (o + sz)[order][:-1]).all()
    # labels
    for b in ids:
        k = int(lod[b])
        if (b, k) not in decoded_cache:
            decoded_cache[(b, k)] = oracle.decode_brick(enc, int(b), k).reshape(-1)
        want_l = decoded_cache[(b, k)]
        assert np.array_equal(cache[int(off[b]):int(off[b]) + want_l.size], want_l), (b, k)
    return fm.next_state(r, lod)


def _run(enc, cfg, frames, marks="bricks", ncam=2, W=64, H=48, materials=None):
    h = oracle.header(enc)
    L, n = h["log2b"], h["n_bricks"]
    vol = vc.vc_load_compressed(enc)
    fc = vc.vc_frame_cache_create(vol, cfg["cap"] * 4, cfg["per_frame"], cfg["free_cap"])
    try:
        view = vc.vc_frame_cache_view_get(fc)
        assert view.n_bricks == n and view.max_bricks_per_frame == min(cfg["per_frame"], n)
        status = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        state = fm.empty_state(n, L)
        prev = (np.full(n, 2 ** 64 - 1, np.uint64), np.full(n, NONE, np.uint8))
        decoded = {}
        resets = 0
        for f in range(frames):
            cams = [_orbit(i, f, h["dims"], W, H) for i in range(ncam)]
            vcams = [vc.make_camera(*c) for c in cams]
            if marks == "bricks":
                vc.vc_frame_mark_cameras(fc, vcams, s)
                visible = _brick_marks(enc, cams)
            else:  # the renderer's rays of the first camera, on the cache as it stands
                off_d, lod_d, cache_d = prev[0], prev[1], _read(view)[2]
                lab = torch.zeros(W * H, dtype=torch.int32, device="cuda")
                vc.vc_render(vol, view.offsets, view.lods, view.cache, vcams[0], materials, lab.data_ptr(), stream=s,
                             mode=vc.VC_SHADE_SHADOW, frame=f, marks_ptr=view.marks, request_depth=1)
                vis_o = np.zeros(n, np.uint8)
                got_lab = oracle.render(enc, off_d, lod_d, cache_d, *cams[0], materials=materials, mode=1, frame=f,
                                        visible=vis_o, request_depth=1)[0]
                marks_gpu = _host(view.marks, (n + 31) // 32, "<i4", np.uint32)
                bits = (marks_gpu[np.arange(n) >> 5] >> (np.arange(n) & 31).astype(np.uint32)) & 1
                assert np.array_equal(bits.astype(bool), vis_o.astype(bool)), f
                assert np.array_equal(lab.cpu().numpy().view(np.uint32).reshape(H, W), got_lab), f
                visible = vis_o.astype(bool)
                cams = cams[:1]
                vcams = vcams[:1]
            want = _want(enc, cams, cfg["max_lod"], visible)
            vc.vc_frame_update(fc, vcams, cfg["max_lod"], status.data_ptr(), s)
            stats = vc.vc_frame_stats_get(fc, s)
            assert int(status[0]) == 0, status.cpu().tolist()
            now = _read(view)
            state = _check_frame(enc, L, cfg, state, want, prev, now, stats, decoded)
            prev = (now[0], now[1])
            resets = int(stats.resets)
        return resets, vc.vc_frame_stats_get(fc, s)
    finally:
        vc.vc_release(fc)
        vc.vc_release(vol)


@pytest.fixture(scope="module")
def vol16():
    V = synth.fill(synth.small(dims=(96, 80, 64), seed=71, grid=16, diameter=14.0, bg=0.03))
    return oracle.encode_volume(V, 4, coder=oracle.CODER_RANS)


def test_frames_with_room_for_everything(vol16):
    cfg = dict(max_lod=2, cap=1 << 22, per_frame=120, free_cap=1 << 20)
    resets, st = _run(vol16, cfg, frames=6)
    assert resets == 0 and st.frames == 6 and st.bricks_decoded > 0 and st.level_switches > 0


def test_tight_cache_overflows_resets_and_dead_regions(vol16):
    # 60,000 labels: 14 level-0 regions of 4096; stacks of 3 entries; 24 bricks per frame
    cfg = dict(max_lod=2, cap=60000, per_frame=24, free_cap=3)
    resets, st = _run(vol16, cfg, frames=10)
    assert st.bricks_unassigned > 0 and resets >= 1


def test_plain_coder_and_single_level(vol16):
    V = synth.fill(synth.small(dims=(64, 64, 48), seed=72, grid=16, diameter=12.0, bg=0.3))
    enc = oracle.encode_volume(V, 4, coder=oracle.CODER_PLAIN)
    cfg = dict(max_lod=0, cap=1 << 20, per_frame=1000, free_cap=8)
    _run(enc, cfg, frames=4)


def test_b64_bricks():
    V = synth.fill(synth.small(dims=(128, 128, 64), seed=73, grid=24, diameter=20.0, bg=0.3))
    enc = oracle.encode_volume(V, 6, coder=oracle.CODER_RANS)
    cfg = dict(max_lod=3, cap=1 << 20, per_frame=4, free_cap=8)
    _run(enc, cfg, frames=4, ncam=1)


def test_renderer_marks_drive_the_cache(vol16):
    mats = np.array([[0.9, 0.3, 0.2, 1.0], [0.2, 0.7, 0.4, 1.0], [0.3, 0.4, 0.9, 0.5], [0.8, 0.8, 0.1, 1.0]],
                    np.float32)
    cfg = dict(max_lod=2, cap=1 << 22, per_frame=120, free_cap=1 << 20)
    _, st = _run(vol16, cfg, frames=5, marks="render", W=64, H=48, materials=mats)
    assert st.bricks_decoded > 0


def test_arguments_checked(vol16):
    vol = vc.vc_load_compressed(vol16)
    try:
        with pytest.raises(vc.VCError):
            vc.vc_frame_cache_create(vol, 0)
        fc = vc.vc_frame_cache_create(vol, 1 << 20)
        try:
            st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
            cam = vc.make_camera((-50, 40, 30), (1, 0, 0), (0, 1, 0), 0.8, 16, 16)
            with pytest.raises(vc.VCError):
                vc.vc_frame_update(fc, [], 2, st.data_ptr())
            with pytest.raises(vc.VCError):
                vc.vc_frame_update(fc, [cam], 2, 0)
            with pytest.raises(vc.VCError):
                vc.vc_frame_update(fc, [cam] * 257, 2, st.data_ptr())
            bad = vc.make_camera((-50, 40, 30), (1, 0, 0), (0, 1, 0), 0.8, 0, 16)
            with pytest.raises(vc.VCError):
                vc.vc_frame_mark_cameras(fc, [bad])
        finally:
            vc.vc_release(fc)
    finally:
        vc.vc_release(vol)
