"""vc_render on the GPU against the rendering oracle, bit for bit: labels, depths, entered faces and
colours of every pixel, for bricks decoded at mixed levels of detail (and some not decoded), opaque,
semi-transparent and hidden materials, the four shading modes, several frames with and without
jitter, cameras outside and inside the volume. The GPU side decodes its bricks with the library;
the oracle side takes the CSGV oracle's decodes of the same bricks."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_36898_gb300 as vc  # noqa: E402

NOT_DECODED = 2 ** 64 - 1


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vc._lib_handle()


MATERIALS = np.array([[0.9, 0.3, 0.2, 1.0], [0.2, 0.7, 0.4, 1.0], [0.3, 0.4, 0.9, 0.4], [0.8, 0.8, 0.1, 1.0],
                      [0.5, 0.5, 0.5, 0.0], [0.6, 0.2, 0.7, 1.0], [0.1, 0.9, 0.9, 0.7]], np.float32)


def _setup(V, log2b, seed):
    enc = vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=1)
    vol = vc.Volume(enc)
    n, b = vol.n_bricks, vol.b
    rng = np.random.default_rng(seed)
    lods = rng.choice([0, 1, 2, 255], size=n, p=[0.55, 0.2, 0.15, 0.1]).astype(np.uint8)
    offsets = np.full(n, NOT_DECODED, np.uint64)
    groups, base = {}, 0
    for k in (0, 1, 2):
        ids = np.flatnonzero(lods == k)
        e3 = (b >> k) ** 3
        offsets[ids] = base + np.arange(ids.size, dtype=np.uint64) * e3
        groups[k] = (ids, base, e3)
        base += ids.size * e3
    cache = torch.zeros(max(1, base), dtype=torch.int32, device="cuda")
    st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for k, (ids, gb, e3) in groups.items():
        if ids.size == 0:
            continue
        ids_t = torch.from_numpy(ids.astype(np.int32)).cuda()
        slots = torch.arange(ids.size, dtype=torch.int32, device="cuda")
        sub = cache[gb:gb + ids.size * e3]
        vc.vc_decode_bricks(vol.handle, ids_t.data_ptr(), ids.size, slots.data_ptr(), sub.data_ptr(), k, vc.VC_MODE_BATCHED,
                            st.data_ptr(), s)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    # the oracle's cache: the CSGV oracle's decodes at the same offsets
    ocache = np.zeros(max(1, base), np.uint32)
    for i in range(n):
        if lods[i] != 255:
            cells = oracle.decode_brick(enc, i, int(lods[i])).reshape(-1)
            ocache[int(offsets[i]):int(offsets[i]) + cells.size] = cells
    return enc, vol, lods, offsets, cache, ocache


def _gpu_render(vol, offsets, lods, cache, cam_args, **kw):
    pos, look, up, fov, W, H = cam_args
    cam = vc.make_camera(pos, look, up, fov, W, H)
    off_t = torch.from_numpy(offsets.view(np.int64)).cuda()
    lod_t = torch.from_numpy(lods).cuda()
    lab = torch.zeros(H * W, dtype=torch.int32, device="cuda")
    dep = torch.zeros(H * W, dtype=torch.float32, device="cuda")
    face = torch.zeros(H * W, dtype=torch.uint8, device="cuda")
    rgb = torch.zeros(H * W * 3, dtype=torch.float32, device="cuda")
    vc.vc_render(vol.handle, off_t.data_ptr(), lod_t.data_ptr(), cache.data_ptr(), cam, MATERIALS, lab.data_ptr(),
                 dep.data_ptr(), face.data_ptr(), rgb.data_ptr(), torch.cuda.current_stream().cuda_stream, **kw)
    torch.cuda.synchronize()
    return (lab.cpu().numpy().view(np.uint32).reshape(H, W), dep.cpu().numpy().reshape(H, W),
            face.cpu().numpy().reshape(H, W), rgb.cpu().numpy().reshape(H, W, 3))


CAMERAS = [((-60.0, 130.0, -80.0), (70.0, -90.0, 110.0), (0.0, 1.0, 0.0), 0.8, 40, 30),
           ((150.0, 20.0, 40.0), (-1.0, 0.15, 0.1), (0.0, 0.0, 1.0), 1.1, 33, 21),
           ((40.0, 30.0, 20.0), (0.4, 0.2, 1.0), (0.0, 1.0, 0.0), 1.3, 24, 24)]  # inside the volume


@pytest.mark.parametrize("log2b", [4, 5])
def test_render_matches_the_oracle_bit_for_bit(log2b):
    V = synth.fill(synth.small(dims=(96, 80, 64), seed=40 + log2b, grid=16, diameter=14.0, bg=0.45))
    enc, vol, lods, offsets, cache, ocache = _setup(V, log2b, 7 + log2b)
    try:
        for ci, cam in enumerate(CAMERAS):
            for mode, frame, jitter in ((0, 0, False), (1, 1, False), (2, 2, True), (3, 3, True), (3, 4, False)):
                kw = dict(mode=mode, frame=frame, jitter=jitter, max_bounces=12, light_dir=(0.4, 0.7, -0.5),
                          ambient=0.2, ao_radius=12.0, sky=1.5)
                got = _gpu_render(vol, offsets, lods, cache, cam, **kw)
                want = oracle.render(enc, offsets, lods, ocache, *cam, materials=MATERIALS, **kw)
                for name, g, w in zip(("labels", "depth", "face", "rgb"), got, want):
                    assert np.array_equal(g.view(np.uint8), np.ascontiguousarray(w).view(np.uint8)), (
                        log2b, ci, mode, frame, name, int((g != w).sum()))
                assert (got[0] != 0).sum() > 0
    finally:
        vol.release()


def test_render_arguments_checked():
    V = synth.fill(synth.small(dims=(32, 32, 32), seed=3))
    enc = vc.vc_encode_volume(V, 4, op_mask=0x7F, coder=1)
    vol = vc.Volume(enc)
    try:
        off = torch.zeros(vol.n_bricks, dtype=torch.int64, device="cuda")
        lod = torch.zeros(vol.n_bricks, dtype=torch.uint8, device="cuda")
        cache = torch.zeros(vol.n_bricks * 16 ** 3, dtype=torch.int32, device="cuda")
        cam = vc.make_camera((-10, 16, 16), (1, 0, 0), (0, 1, 0), 0.8, 8, 8)
        for bad in (dict(mode=9), dict(mode=3, max_bounces=0), dict(mode=3, max_bounces=33), dict(mode=2, ao_radius=0.0),
                    dict(light_dir=(0.0, 0.0, 0.0))):
            with pytest.raises(vc.VCError):
                vc.vc_render(vol.handle, off.data_ptr(), lod.data_ptr(), cache.data_ptr(), cam, MATERIALS, **bad)
        with pytest.raises(vc.VCError):
            vc.vc_render(vol.handle, off.data_ptr(), lod.data_ptr(), cache.data_ptr(), cam, np.zeros((0, 4), np.float32))
    finally:
        vol.release()


@pytest.mark.parametrize("subsample", [1, 2, 4])
def test_stratified_frames_and_postprocessing_match_the_oracle(subsample):
    """Stratified subsets (one pixel of each s x s block per frame) render exactly the oracle's pixels;
    the post-processing (accumulation, G-buffer, À-trous passes, upsampling, tone map) over s^2 + 1
    frames gives the oracle's image within one unit per channel (exp and pow are the only operations
    whose last bits may differ between the GPU and the host C library)."""
    V = synth.fill(synth.small(dims=(64, 64, 48), seed=55, grid=16, diameter=16.0, bg=0.4))
    enc, vol, lods, offsets, cache, ocache = _setup(V, 4, 9)
    try:
        pos, look, up, fov, W, H = (-40.0, 90.0, -60.0), (70.0, -60.0, 90.0), (0.0, 1.0, 0.0), 0.9, 48, 36
        cam = vc.make_camera(pos, look, up, fov, W, H)
        off_t = torch.from_numpy(offsets.view(np.int64)).cuda()
        lod_t = torch.from_numpy(lods).cuda()
        lab = torch.zeros(H * W, dtype=torch.int32, device="cuda")
        dep = torch.zeros(H * W, dtype=torch.float32, device="cuda")
        face = torch.zeros(H * W, dtype=torch.uint8, device="cuda")
        rgb = torch.zeros(H * W * 3, dtype=torch.float32, device="cuda")
        state = torch.zeros(vc.vc_post_state_bytes(W, H), dtype=torch.uint8, device="cuda")
        rgba = torch.zeros(H * W, dtype=torch.int32, device="cuda")
        o_out = (np.zeros((H, W), np.uint32), np.zeros((H, W), np.float32), np.zeros((H, W), np.uint8),
                 np.zeros((H, W, 3), np.float32))
        o_state = oracle.post_state(W, H)
        s = torch.cuda.current_stream().cuda_stream
        for f in range(subsample * subsample + 1):
            kw = dict(mode=vc.VC_SHADE_AO, frame=f, jitter=False, ao_radius=10.0, sky=1.2, subsample=subsample)
            vc.vc_render(vol.handle, off_t.data_ptr(), lod_t.data_ptr(), cache.data_ptr(), cam, MATERIALS, lab.data_ptr(),
                         dep.data_ptr(), face.data_ptr(), rgb.data_ptr(), s, **kw)
            oracle.render(enc, offsets, lods, ocache, pos, look, up, fov, W, H, materials=MATERIALS, out=o_out, **kw)
            pk = dict(iterations=3, subsample=subsample, frame=f, reset=f == 0, phi_rho=8.0, phi_d=1.0, exposure=1.3,
                      gamma=2.2)
            vc.vc_postprocess(vol.handle, W, H, lab.data_ptr(), dep.data_ptr(), face.data_ptr(), rgb.data_ptr(),
                              state.data_ptr(), rgba.data_ptr(), MATERIALS, pos, stream=s, **pk)
            want = oracle.post(o_state, (64, 64, 48), o_out[0], o_out[1], o_out[2], o_out[3], MATERIALS, pos, **pk)
            torch.cuda.synchronize()
            assert np.array_equal(lab.cpu().numpy().view(np.uint32).reshape(H, W), o_out[0]), f
            assert np.array_equal(rgb.cpu().numpy().reshape(H, W, 3).view(np.uint32), o_out[3].view(np.uint32)), f
            got = rgba.cpu().numpy().view(np.uint32).reshape(H, W)
            gb = np.stack([(got >> (8 * k)) & 255 for k in range(4)], -1).astype(np.int64)
            wb = np.stack([(want >> (8 * k)) & 255 for k in range(4)], -1).astype(np.int64)
            assert np.abs(gb - wb).max() <= 1, (f, int(np.abs(gb - wb).max()))
            assert (gb == wb).all(axis=-1).mean() > 0.95
    finally:
        vol.release()


@pytest.mark.parametrize("mode,depth", [(0, 0), (1, 0), (1, 1), (2, 1), (3, 1), (3, 2), (3, 5)])
def test_visibility_marks_match_the_oracle(mode, depth):
    """The bricks the rays of path depth <= request_depth access (one bit per brick), for every
    shading mode, equal the oracle's, and the image is unchanged by marking."""
    V = synth.fill(synth.small(dims=(96, 80, 64), seed=45, grid=16, diameter=14.0, bg=0.45))
    enc, vol, lods, offsets, cache, ocache = _setup(V, 4, 11)
    try:
        n = vol.n_bricks
        marks = torch.zeros((n + 31) // 32, dtype=torch.int32, device="cuda")
        for ci, cam in enumerate(CAMERAS):
            marks.zero_()
            kw = dict(mode=mode, frame=ci + 1, jitter=True, max_bounces=8, ao_radius=10.0)
            got = _gpu_render(vol, offsets, lods, cache, cam, marks_ptr=marks.data_ptr(), request_depth=depth, **kw)
            vis = np.zeros(n, np.uint8)
            want = oracle.render(enc, offsets, lods, ocache, *cam, materials=MATERIALS, visible=vis, request_depth=depth,
                                 **kw)
            m = marks.cpu().numpy().view(np.uint32)
            bits = (m[np.arange(n) >> 5] >> (np.arange(n) & 31).astype(np.uint32)) & 1
            assert np.array_equal(bits.astype(bool), vis.astype(bool)), (mode, depth, ci, int((bits != vis).sum()))
            assert vis.sum() > 0
            for g, w in zip(got, want):
                assert np.array_equal(g.view(np.uint8), np.ascontiguousarray(w).view(np.uint8))
    finally:
        vol.release()
