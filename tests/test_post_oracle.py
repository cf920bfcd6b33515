"""Pins of the post-processing oracle (oracle/post_oracle.c) against what the definitions fix on
their own (Methods, "Post-processing"): with no passes the output is the tone-mapped mean of the
accumulated samples; a uniform surface stays uniform under any number of passes (the weights are
normalised); the filter does not mix pixels of different normals; it lowers the variance of noise on
one surface without moving its mean; the accumulation averages frames; and pixels not rendered yet
take the colour of a rendered pixel at the smallest distance (checked against brute force)."""
import numpy as np

import oracle

MATS = np.array([[0.8, 0.4, 0.2, 1.0], [0.2, 0.6, 0.9, 1.0]], np.float32)
DIMS = (64, 64, 64)
CAM = (32.0, 32.0, -100.0)


def tone(x, exposure=1.0, gamma=2.2):
    x = np.asarray(x, np.float64) * exposure
    y = np.clip(x * (2.51 * x + 0.03) / (x * (2.43 * x + 0.59) + 0.14), 0, 1) ** (1 / gamma)
    return np.floor(y * 255 + 0.5).astype(np.int64)


def unpack(rgba):
    return np.stack([(rgba >> (8 * k)) & 255 for k in range(3)], -1).astype(np.int64)


def frame_inputs(H, W, label=5, face=5, depth=110.0, rgb=(0.3, 0.5, 0.7)):
    labels = np.full((H, W), label, np.uint32)
    faces = np.full((H, W), face, np.uint8)
    depths = np.full((H, W), depth, np.float32)
    cols = np.broadcast_to(np.asarray(rgb, np.float32), (H, W, 3)).copy()
    return labels, depths, faces, cols


def test_no_passes_is_the_tone_mapped_sample():
    H, W = 7, 9
    rng = np.random.default_rng(0)
    labels, depths, faces, _ = frame_inputs(H, W)
    rgb = rng.random((H, W, 3)).astype(np.float32) * 2
    st = oracle.post_state(W, H)
    out = oracle.post(st, DIMS, labels, depths, faces, rgb, MATS, CAM, iterations=0, reset=True)
    assert np.abs(unpack(out) - tone(rgb)).max() <= 1
    assert ((out >> 24) == 255).all()


def test_uniform_surface_stays_uniform_and_frames_average():
    H, W = 12, 10
    labels, depths, faces, rgb = frame_inputs(H, W, rgb=(0.4, 0.1, 0.9))
    st = oracle.post_state(W, H)
    for it in (0, 1, 3, 5):
        out = oracle.post(st, DIMS, labels, depths, faces, rgb, MATS, CAM, iterations=it, reset=True)
        assert len(np.unique(out)) == 1 and np.abs(unpack(out)[0, 0] - tone([0.4, 0.1, 0.9])).max() <= 1
    # two frames of different colours average to their mean
    st = oracle.post_state(W, H)
    oracle.post(st, DIMS, labels, depths, faces, rgb * 0 + 0.2, MATS, CAM, iterations=0, reset=True)
    out = oracle.post(st, DIMS, labels, depths, faces, rgb * 0 + 0.6, MATS, CAM, iterations=0)
    assert np.abs(unpack(out) - tone([0.4, 0.4, 0.4])).max() <= 1


def test_edges_between_normals_are_kept():
    H, W = 10, 16
    labels, depths, faces, rgb = frame_inputs(H, W)
    faces[:, W // 2:] = 1  # right half faces -x instead of -z
    rgb[:, W // 2:] = (0.9, 0.9, 0.1)
    st = oracle.post_state(W, H)
    out = unpack(oracle.post(st, DIMS, labels, depths, faces, rgb, MATS, CAM, iterations=4, reset=True))
    assert np.abs(out[:, :W // 2] - tone([0.3, 0.5, 0.7])).max() <= 1
    assert np.abs(out[:, W // 2:] - tone([0.9, 0.9, 0.1])).max() <= 1


def test_noise_on_one_surface_is_smoothed_with_its_mean_kept():
    H, W = 40, 40
    labels, depths, faces, _ = frame_inputs(H, W)
    rng = np.random.default_rng(3)
    noisy = (0.3 + 0.2 * rng.standard_normal((H, W, 1))).clip(0.0, 1.0).astype(np.float32).repeat(3, -1)
    st = oracle.post_state(W, H)
    raw = unpack(oracle.post(st, DIMS, labels, depths, faces, noisy, MATS, CAM, iterations=0, reset=True))
    out = unpack(oracle.post(st, DIMS, labels, depths, faces, noisy, MATS, CAM, iterations=3, reset=True))
    inner = (slice(8, -8), slice(8, -8), 0)
    assert out[inner].std() < 0.5 * raw[inner].std()
    # the filter averages linear colours: its output sits at the tone-mapped mean of the samples
    assert abs(out[inner].mean() - tone([noisy[8:-8, 8:-8, 0].mean()])[0]) < 3


def test_unrendered_pixels_take_a_nearest_rendered_pixel():
    H, W = 24, 30
    labels, depths, faces, _ = frame_inputs(H, W)
    # distinct depths: the depth weight keeps every rendered pixel's own colour (phi_d large)
    depths = (100.0 + np.arange(H * W, dtype=np.float32).reshape(H, W) * 0.9).astype(np.float32)
    rgb = np.stack(list(np.meshgrid(np.linspace(0.05, 0.95, W), np.linspace(0.05, 0.95, H))) + [np.full((H, W), 0.5)],
                   -1).astype(np.float32)
    for s in (2, 4):
        st = oracle.post_state(W, H)
        out = oracle.post(st, DIMS, labels, depths, faces, rgb, MATS, CAM, iterations=5, subsample=s, frame=0,
                          reset=True, phi_d=50.0)
        rendered = np.array([[oracle_subset(px, py, s, 0) for px in range(W)] for py in range(H)])
        ry, rx = np.nonzero(rendered)
        off = st["off1"] if 5 & 1 else st["off0"]
        for py in range(H):
            for px in range(W):
                if rendered[py, px]:
                    continue
                o = int(off[py * W + px])
                dx = (o & 0xFFFF) - (0x10000 if o & 0x8000 else 0)
                dy = o >> 16
                qx, qy = px + int(dx), py + int(dy)
                assert rendered[qy, qx]
                best = ((rx - px) ** 2 + (ry - py) ** 2).min()
                assert int(dx) ** 2 + int(dy) ** 2 == best, (s, px, py)
                assert out[py, px] == out[qy, qx]


def oracle_subset(px, py, s, f):
    """The stratified subset rule (render_oracle.c), through the oracle library."""
    import ctypes
    lib = oracle._load()
    lib.oracle_subset_pixel.argtypes = [ctypes.c_uint32] * 4
    lib.oracle_subset_pixel.restype = ctypes.c_int
    return bool(lib.oracle_subset_pixel(px, py, s, f))
