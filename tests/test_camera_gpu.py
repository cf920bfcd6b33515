"""The camera request stage on the GPU against the oracle, through the C ABI: the same bricks
(bit-exact ids, ascending) and the same levels of detail for every camera; the serving form
queues one request per camera whose decoded bricks match the oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_36898_gb300 as vc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vc._lib_handle()


def orbit_cameras(dims, n, seed, W, H, fov=0.8):
    """Cameras on spheres around the volume centre (radius 1.2 to 3 diagonals), looking at points
    near the centre."""
    rng = np.random.default_rng(seed)
    centre = np.array(dims, np.float64) / 2
    diag = float(np.linalg.norm(dims))
    cams = []
    for _ in range(n):
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        pos = centre + axis * diag * rng.uniform(0.6, 1.5)
        target = centre + rng.normal(size=3) * diag * 0.05
        up = np.cross(target - pos, rng.normal(size=3))
        cams.append((pos, target - pos, up, fov, W, H))
    return cams


@pytest.mark.parametrize("log2b,coder,bg", [(4, 0, 0.4), (5, 1, 0.1), (3, 1, 0.3)])
def test_camera_bricks_match_oracle(log2b, coder, bg):
    dims = (160, 128, 96)
    V = synth.fill(synth.small(dims=dims, seed=30 + log2b, grid=16, diameter=16.0, bg=bg))
    enc = vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=coder)
    vol = vc.vc_load_compressed(enc, 0, 0)
    try:
        specs = orbit_cameras(dims, 6, log2b, 96, 64)
        # plus one camera inside the volume and one axis-aligned
        specs.append((np.array([80.0, 60.0, 40.0]), np.array([1.0, 0.3, 0.2]), np.array([0.0, 0.0, 1.0]), 1.2, 64, 48))
        specs.append((np.array([72.0, 56.0, -50.0]), np.array([0.0, 0.0, 1.0]), np.array([0.0, 1.0, 0.0]), 0.5, 33, 17))
        cams = [vc.make_camera(*s) for s in specs]
        got = vc.vc_camera_bricks(vol, cams, max_lod=log2b)
        for (pos, d, up, fov, W, H), (gi, gl) in zip(specs, got):
            wi, wl = oracle.camera_bricks(enc, pos.astype(np.float32), d.astype(np.float32), up.astype(np.float32),
                                          fov, W, H, log2b)
            assert np.array_equal(gi, wi), (len(gi), len(wi))
            assert np.array_equal(gl, wl)
            assert len(wi) > 0
    finally:
        vc.vc_release(vol)


def test_request_bricks_serves_camera_requests():
    dims = (128, 128, 128)
    V = synth.fill(synth.small(dims=dims, seed=41, grid=16, diameter=16.0, bg=0.3))
    enc = vc.vc_encode_volume(V, 5, op_mask=0x7F, coder=1)
    vol = vc.vc_load_compressed(enc, 0, 0)
    srv = vc.vc_server_create(64 << 20, 0)
    try:
        vi = vc.vc_server_add_volume(srv, vol)
        specs = orbit_cameras(dims, 4, 7, 64, 48)
        cams = [vc.make_camera(*s) for s in specs]
        rids = vc.vc_request_bricks(srv, vi, cams, max_lod=3)
        ptr, nbytes = vc.vc_server_cache(srv)

        class _H:
            __cuda_array_interface__ = {"shape": (nbytes // 4,), "typestr": "<i4", "data": (ptr, False), "version": 3}
        cache = torch.as_tensor(_H(), device="cuda")
        for (pos, d, up, fov, W, H), rid in zip(specs, rids):
            wi, wl = oracle.camera_bricks(enc, pos.astype(np.float32), d.astype(np.float32), up.astype(np.float32),
                                          fov, W, H, 3)
            assert vc.vc_wait(srv, rid, 60000) == vc.VC_REQ_DONE
            info = vc.vc_request_info_get(srv, rid)
            assert info.n_bricks == len(wi)
            _, offs = vc.vc_poll(srv, rid, len(wi))
            for k in range(0, len(wi), max(1, len(wi) // 8)):
                e = 32 >> int(wl[k])
                w0 = int(offs[k]) // 4
                got = cache[w0:w0 + e ** 3].cpu().numpy().view(np.uint32).reshape(e, e, e)
                assert np.array_equal(got, oracle.decode_brick(enc, int(wi[k]), int(wl[k])))
            vc.vc_request_release(srv, rid)
    finally:
        vc.vc_release(srv)
        vc.vc_release(vol)
