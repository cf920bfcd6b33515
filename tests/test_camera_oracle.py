"""Pins of the camera request oracle (oracle/camera_oracle.c) against closed forms and a
double-precision brute-force traversal; no GPU."""
import math

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def vol16():
    V = synth.fill(synth.small(dims=(128, 96, 80), seed=21, grid=16, diameter=18.0, bg=0.35))
    return V, oracle.encode_volume(V, 4, coder=0)


def brick_flags(V, b):
    """(nbz, nby, nbx) arrays: has background (label 0), has a visible label (!= 0) — from the voxels."""
    nz, ny, nx = (s // b for s in V.shape)
    blk = V.reshape(nz, b, ny, b, nx, b).transpose(0, 2, 4, 1, 3, 5).reshape(nz, ny, nx, -1)
    return (blk == 0).any(-1), (blk != 0).any(-1)


def test_axis_ray_requests_its_column_up_to_the_first_opaque_brick(vol16):
    V, enc = vol16
    b = 16
    has_bg, has_fg = brick_flags(V, b)
    nbz, nby, nbx = has_bg.shape
    for bx, by in ((0, 0), (3, 2), (7, 5), (4, 1)):
        pos = ((bx + 0.5) * b, (by + 0.5) * b, -40.0)
        ids, lods = oracle.camera_bricks(enc, pos, (0, 0, 1), (0, 1, 0), 0.5, 1, 1)
        want = []
        for z in range(nbz):
            if has_fg[z, by, bx]:
                want.append(bx + nbx * (by + nby * z))
            if not has_bg[z, by, bx]:
                break
        assert ids.tolist() == want, (bx, by)
    # looking back along -z from behind the volume: the same column from the other end
    bx, by = 3, 2
    ids, _ = oracle.camera_bricks(enc, ((bx + 0.5) * b, (by + 0.5) * b, V.shape[0] + 33.0), (0, 0, -1), (0, 1, 0),
                                  0.5, 1, 1)
    want = []
    for z in reversed(range(nbz)):
        if has_fg[z, by, bx]:
            want.append(bx + nbx * (by + nby * z))
        if not has_bg[z, by, bx]:
            break
    assert ids.tolist() == sorted(want)


def test_lod_closed_form(vol16):
    V, enc = vol16
    b, H, fov = 16, 64, 0.7
    # one pixel row straight down the x axis; brick centres at known distances
    for dist in (10.0, 30.0, 70.0, 150.0, 400.0, 1000.0):
        pos = (-dist + 0.5 * b, 0.5 * b, 0.5 * b)
        ids, lods = oracle.camera_bricks(enc, pos, (1, 0, 0), (0, 1, 0), fov, 1, H, max_lod=4)
        first = np.where(ids == 0)[0]
        if first.size == 0:
            continue
        k = int(lods[first[0]])
        w = dist * 2 * math.tan(fov / 2) / H  # pixel footprint in voxels at the brick centre
        want = 0
        while want < 4 and 4 ** (want + 1) <= w * w * (1 + 1e-6):
            want += 1
        assert k == want, (dist, k, want)


def brute_force(V, b, pos, d, has_bg, has_fg, eps=1e-6):
    """Bricks one ray passes, by an exact-arithmetic-style traversal in double precision (cell by
    cell: the next crossing is the nearest face), stopping after the first opaque brick. Returns
    (requested ids, ambiguous) where ambiguous is True when the ray enters the grid on an edge or
    passes within eps of an edge or corner of the brick grid (float and double may then take
    different, equally valid, cells)."""
    nbz, nby, nbx = has_bg.shape
    n = np.array([nbx, nby, nbz], dtype=np.float64)
    o = np.asarray(pos, np.float64) / b
    d = np.asarray(d, np.float64) / b
    if np.any((d == 0) & ((o < 0) | (o >= n))):
        return set(), False
    with np.errstate(divide="ignore", invalid="ignore"):
        ta = np.where(d != 0, (0 - o) / d, -np.inf)
        tb = np.where(d != 0, (n - o) / d, np.inf)
    t0, t1 = max(0.0, np.minimum(ta, tb).max()), np.maximum(ta, tb).min()
    if not t0 < t1:
        return set(), False
    p = o + t0 * d
    cell = np.clip(np.floor(p), 0, n - 1).astype(np.int64)
    frac = p - np.floor(p)
    amb = int((np.minimum(frac, 1 - frac) < eps).sum()) >= 2
    out = set()
    while True:
        x, y, z = (int(v) for v in cell)
        if has_fg[z, y, x]:
            out.add(x + nbx * (y + nby * z))
        if not has_bg[z, y, x]:
            break
        with np.errstate(divide="ignore", invalid="ignore"):
            nxt = np.where(d > 0, (cell + 1 - o) / d, np.where(d < 0, (cell - o) / d, np.inf))
        order = np.argsort(nxt, kind="stable")
        if nxt[order[1]] - nxt[order[0]] < eps * max(1.0, abs(nxt[order[0]])):
            amb = True
        a = order[0]
        if nxt[a] >= t1:
            break
        cell[a] += 1 if d[a] > 0 else -1
        if cell[a] < 0 or cell[a] >= n[a]:
            break
    return out, amb


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_matches_brute_force_traversal(vol16, seed):
    V, enc = vol16
    b = 16
    has_bg, has_fg = brick_flags(V, b)
    rng = np.random.default_rng(seed)
    W, H, fov = 12, 9, 0.8
    centre = np.array(V.shape[::-1], np.float64) / 2
    for _ in range(3):
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        pos = centre + axis * rng.uniform(150, 300)
        dirv = centre - pos + rng.normal(size=3) * 10
        up = np.cross(dirv, rng.normal(size=3))
        ids, _ = oracle.camera_bricks(enc, pos, dirv, up, fov, W, H)
        got = set(ids.tolist())
        # the same frame and pixel directions, in double precision
        f = dirv / np.linalg.norm(dirv)
        r = np.cross(f, up)
        r /= np.linalg.norm(r)
        u = np.cross(r, f)
        t = math.tan(fov / 2)
        want, loose, n_amb = set(), set(), 0
        for py in range(H):
            for px in range(W):
                sx = ((px + 0.5) * 2 / W - 1) * t * W / H
                sy = (1 - (py + 0.5) * 2 / H) * t
                w, a = brute_force(V, b, pos.astype(np.float32), f + sx * r + sy * u, has_bg, has_fg)
                if a:  # an edge or corner crossing: either neighbour is a valid float result
                    n_amb += 1
                    loose |= w
                else:
                    want |= w
        assert n_amb <= W * H // 10
        assert want <= got, sorted(want - got)[:10]
        # bricks only the oracle has must come from rays whose double-precision path was ambiguous,
        # and lie next to a brick such a ray passed
        extra = got - want - loose
        nbx, nby = has_bg.shape[2], has_bg.shape[1]
        near = set()
        for i in loose:
            x, y, z = i % nbx, (i // nbx) % nby, i // (nbx * nby)
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        near.add((x + dx) + nbx * ((y + dy) + nby * (z + dz)))
        assert extra <= near, sorted(extra)[:10]
        assert len(want) > 0


def test_camera_inside_volume_and_sorted_output(vol16):
    V, enc = vol16
    ids, lods = oracle.camera_bricks(enc, (60.0, 50.0, 40.0), (1, 0.2, 0.1), (0, 0, 1), 1.2, 32, 24)
    assert len(ids) > 0
    assert np.all(np.diff(ids.astype(np.int64)) > 0)
    assert lods.max() <= 4
    has_bg, has_fg = brick_flags(V, 16)
    assert all(has_fg.reshape(-1)[ids])  # only bricks with a visible label are requested
