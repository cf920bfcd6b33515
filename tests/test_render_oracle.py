"""Pins of the rendering oracle (oracle/render_oracle.c) against what geometry and the shading
definitions fix on their own (Methods, "Volcanite rendering"): axis-aligned rays hit the first
opaque voxel of their voxel column at its exact face distance; general rays agree with a
double-precision brute-force intersection of the ray with every voxel box; coarse levels of detail
and undecoded bricks are seen as their cells; local, shadow, ambient-occlusion and path-traced
shading reduce to closed forms on planes, open half spaces and closed boxes; semi-transparent
materials composite front to back; the jitter stays inside (-1, 1) pixel."""
import numpy as np
import pytest

import oracle

NOT_DECODED = np.uint64(2 ** 64 - 1)


def encode(V, log2b=2):
    return oracle.encode_volume(np.ascontiguousarray(V, dtype=np.uint32), log2b, coder=1)


def layout(enc, lods):
    """Per brick the oracle's decode at its level of detail, packed one after the other."""
    h = oracle.header(enc)
    n = h["n_bricks"]
    offsets = np.zeros(n, np.uint64)
    parts, at = [], 0
    for i in range(n):
        if lods[i] == 255:
            offsets[i] = NOT_DECODED
            continue
        cells = oracle.decode_brick(enc, i, int(lods[i])).reshape(-1)
        offsets[i] = at
        parts.append(cells)
        at += cells.size
    cache = np.concatenate(parts) if parts else np.zeros(1, np.uint32)
    return offsets, np.asarray(lods, np.uint8), cache


def opaque_materials(n=4, rgb=(0.8, 0.6, 0.4)):
    return np.array([[rgb[0], rgb[1], rgb[2], 1.0]] * n, np.float32)


def render(enc, lods, cam, mats, **kw):
    offsets, lods8, cache = layout(enc, lods)
    return oracle.render(enc, offsets, lods8, cache, *cam, materials=mats, **kw)


def column_camera(x, y, z0=-10.0):
    """One pixel looking along +z through the centre of voxel column (x, y)."""
    return ((x + 0.5, y + 0.5, z0), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0), 0.5, 1, 1)


def random_volume(seed, shape=(16, 12, 20), p_zero=0.85, nlab=5):
    rng = np.random.default_rng(seed)
    V = rng.integers(1, nlab + 1, size=shape).astype(np.uint32)
    V[rng.random(shape) < p_zero] = 0
    return V


def test_axis_aligned_rays_hit_the_first_voxel_of_their_column():
    V = random_volume(1)
    enc = encode(V)
    n = oracle.header(enc)["n_bricks"]
    mats = opaque_materials()
    nz, ny, nx = V.shape
    for y in range(ny):
        for x in range(nx):
            lab, depth, face, _ = render(enc, [0] * n, column_camera(x, y), mats)
            col = np.flatnonzero(V[:, y, x])
            if col.size == 0:
                assert lab[0, 0] == 0 and np.isinf(depth[0, 0]) and face[0, 0] == 0
            else:
                z = int(col[0])
                assert lab[0, 0] == V[z, y, x]
                assert depth[0, 0] == np.float32(10 + z)  # exact: unit steps from t = 10
                assert face[0, 0] == 5  # entered through the voxel's -z side


def _brute_force(V, o, d):
    """First nonzero voxel along o + t d (double precision, slab test per voxel) and its entry t."""
    nz, ny, nx = V.shape
    z, y, x = np.nonzero(V)
    lo = np.stack([x, y, z], 1).astype(np.float64)
    hi = lo + 1.0
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (lo - o) / d
        t2 = (hi - o) / d
    tmin = np.nanmax(np.where(np.isfinite(t1) | np.isfinite(t2), np.minimum(t1, t2), -np.inf), axis=1)
    tmax = np.nanmin(np.where(np.isfinite(t1) | np.isfinite(t2), np.maximum(t1, t2), np.inf), axis=1)
    inside = (np.abs(d) > 0) | ((o >= lo) & (o < hi))
    ok = inside.all(axis=1) & (tmin < tmax) & (tmax > 0)
    if not ok.any():
        return 0, np.inf, np.inf
    idx = np.flatnonzero(ok)
    order = np.argsort(tmin[idx])
    best = idx[order[0]]
    gap = tmin[idx[order[1]]] - tmin[best] if order.size > 1 else np.inf
    return int(V[z[best], y[best], x[best]]), float(tmin[best]), gap


def test_general_rays_match_a_brute_force_intersection():
    V = random_volume(2, shape=(20, 18, 22), p_zero=0.93)
    enc = encode(V)
    n = oracle.header(enc)["n_bricks"]
    W, H = 24, 18
    pos, look, up, fov = (-9.0, 31.0, -14.0), (15.0, -18.0, 24.0), (0.0, 1.0, 0.0), 0.9
    lab, depth, face, _ = oracle.render(enc, *layout(enc, [0] * n), pos, look, up, fov, W, H, opaque_materials())
    # the same camera model in double precision
    f = np.asarray(look, np.float64) / np.linalg.norm(look)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    t = np.tan(fov / 2)
    checked = 0
    for py in range(H):
        for px in range(W):
            sx = ((px + 0.5) * 2 / W - 1) * t * W / H
            sy = (1 - (py + 0.5) * 2 / H) * t
            d = f + sx * r + sy * u
            d /= np.linalg.norm(d)
            want, tw, gap = _brute_force(V, np.asarray(pos, np.float64), d)
            if gap < 1e-3:  # the ray passes (nearly) through an edge: either voxel is right
                continue
            assert lab[py, px] == want, (px, py)
            if want:
                assert abs(depth[py, px] - tw) < 1e-3 * max(1.0, tw)
            checked += 1
    assert checked > 0.8 * W * H


def test_coarse_levels_and_undecoded_bricks_are_seen_as_their_cells():
    V = random_volume(3, shape=(16, 16, 16), p_zero=0.5, nlab=3)
    enc = encode(V)  # 4^3 bricks
    nbx = 4
    n = oracle.header(enc)["n_bricks"]
    mats = opaque_materials()
    for lod in (1, 2):
        for y in range(16):
            for x in range(0, 16, 3):
                lab, depth, face, _ = render(enc, [lod] * n, column_camera(x, y), mats)
                # the column through the level-lod cells of the bricks along z
                col = []
                for bz in range(4):
                    bid = (x // 4) + nbx * ((y // 4) + nbx * bz)
                    g = oracle.decode_brick(enc, bid, lod)
                    e = 4 >> lod
                    cx, cy = (x % 4) >> lod, (y % 4) >> lod
                    for cz in range(e):
                        col += [int(g[cz, cy, cx])] * (1 << lod)
                first = next((z for z, l in enumerate(col) if l), None)
                if first is None:
                    assert lab[0, 0] == 0
                else:
                    assert lab[0, 0] == col[first] and depth[0, 0] == np.float32(10 + first)
    # not decoded: one cell per brick holding its first palette entry
    for y in range(0, 16, 2):
        for x in range(0, 16, 2):
            lab, depth, face, _ = render(enc, [255] * n, column_camera(x, y), mats)
            col = []
            for bz in range(4):
                bid = (x // 4) + nbx * ((y // 4) + nbx * bz)
                col += [int(oracle.brick_record(enc, bid)["palette"][0])] * 4
            first = next((z for z, l in enumerate(col) if l), None)
            want = 0 if first is None else col[first]
            assert lab[0, 0] == want


def _plane(z=6, shape=(16, 16, 16), label=3):
    V = np.zeros(shape, np.uint32)
    V[z:, :, :] = label
    return V


def test_local_and_shadow_shading_closed_forms():
    V = _plane()
    enc = encode(V)
    n = oracle.header(enc)["n_bricks"]
    mats = opaque_materials(rgb=(0.5, 0.25, 1.0))
    light = np.array([0.2, -0.3, -0.9])
    lu = (light / np.linalg.norm(light)).astype(np.float32)
    nl = max(0.0, float(-lu[2]))  # face -z: normal (0, 0, -1)
    for mode in (0, 1):
        lab, depth, face, rgb = render(enc, [0] * n, column_camera(7, 7), mats, mode=mode, light_dir=tuple(light),
                                       ambient=0.25)
        shade = np.float32(0.25) + np.float32(0.75) * np.float32(nl)
        assert face[0, 0] == 5 and depth[0, 0] == 16.0
        assert np.allclose(rgb[0, 0], np.array([0.5, 0.25, 1.0], np.float32) * shade, rtol=0, atol=1e-6)
    # an occluder between the surface and the light: the shadow ray is blocked, only ambient stays
    V2 = V.copy()
    V2[2:4, :, :] = 2  # a slab in front of the plane, with a hole for the view ray
    V2[2:4, 7, 7] = 0
    enc2 = encode(V2)
    lab, depth, face, rgb = render(enc2, [0] * n, column_camera(7, 7), mats, mode=1, light_dir=tuple(light),
                                   ambient=0.25)
    assert lab[0, 0] == 3
    assert np.allclose(rgb[0, 0], np.array([0.5, 0.25, 1.0], np.float32) * np.float32(0.25), atol=1e-6)


def test_ambient_occlusion_and_path_tracing_open_and_closed():
    mats = opaque_materials(rgb=(0.9, 0.5, 0.3))
    # open half space in front of a plane: every occlusion ray and every first bounce escapes
    V = _plane()
    enc = encode(V)
    n = oracle.header(enc)["n_bricks"]
    for frame in range(6):
        _, _, _, rgb = render(enc, [0] * n, column_camera(5, 9), mats, mode=2, frame=frame, ao_radius=30.0, sky=2.0)
        assert np.allclose(rgb[0, 0], np.array([0.9, 0.5, 0.3], np.float32) * np.float32(2.0), atol=1e-6)
        _, _, _, rgb = render(enc, [0] * n, column_camera(5, 9), mats, mode=3, frame=frame, max_bounces=8, sky=2.0)
        assert np.allclose(rgb[0, 0], np.array([0.9, 0.5, 0.3], np.float32) * np.float32(2.0), atol=1e-6)
    # the camera inside a closed box: every ray hits a wall right away
    V = np.full((16, 16, 16), 4, np.uint32)
    V[4:12, 4:12, 4:12] = 0
    enc = encode(V)
    cam = ((8.0, 8.0, 6.0), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0), 1.2, 5, 4)
    for frame in range(3):
        _, _, _, rgb = render(enc, [0] * n, cam, mats, mode=2, frame=frame, ao_radius=30.0, sky=2.0)
        assert (rgb == 0).all()
        _, _, _, rgb = render(enc, [0] * n, cam, mats, mode=3, frame=frame, max_bounces=32, sky=2.0)
        assert (rgb == 0).all()  # no path can reach the sky


def test_semi_transparent_slab_composites_in_front_of_a_surface():
    V = _plane(z=9, label=3)
    V[4:6, :, :] = 2  # a semi-transparent slab two voxels thick (entered once)
    enc = encode(V)
    n = oracle.header(enc)["n_bricks"]
    # materials by label: find which material index each label maps to, by probing opacities
    light = (0.0, 0.0, -1.0)  # facing the -z faces: shade = ambient + (1 - ambient) = 1
    for sigma in (0.25, 0.5, 0.75):
        mats = np.array([[0.2, 0.4, 0.6, sigma]] * 4, np.float32)
        # label 3 must be opaque: give every material opacity sigma, then test with the plane label
        # in its own material by making the slab label the only semi-transparent one
        lab, depth, face, rgb = render(enc, [0] * n, column_camera(3, 3), mats, light_dir=light, ambient=0.25)
        # every material semi-transparent: slab then plane, both composited, no opaque hit
        assert lab[0, 0] == 0
        s = np.float32(sigma)
        T1 = np.float32(1) - s
        want = s * np.array([0.2, 0.4, 0.6], np.float32) + (T1 * s) * np.array([0.2, 0.4, 0.6], np.float32)
        assert np.allclose(rgb[0, 0], want, atol=1e-6)


def test_jitter_stays_inside_the_pixel_and_centres_on_it():
    V = _plane()
    enc = encode(V)
    n = oracle.header(enc)["n_bricks"]
    mats = opaque_materials()
    # a wide view of the plane: the depth of the centre pixel moves with the jitter
    cam = ((8.0, 8.0, -10.0), (0.3, 0.2, 1.0), (0.0, 1.0, 0.0), 0.3, 1, 1)
    base = render(enc, [0] * n, cam, mats)[1][0, 0]
    offs = []
    for frame in range(64):
        d = render(enc, [0] * n, cam, mats, jitter=True, frame=frame)[1][0, 0]
        offs.append(d - base)
    offs = np.array(offs)
    assert np.ptp(offs) > 0 and abs(offs.mean()) < 0.25 * np.abs(offs).max()
