"""The GPU input generator (synth_gpu.cu) against the CPU generator (synth.c): the same voxels, bit
for bit, on sampled boxes of every workload recipe (plain Voronoi, power diagram with forced-uniform
bricks, hash grids of edge 8 to 64, ragged and negative origins). The large benchmark volumes are
generated on the GPU only because the CPU generator would take hours for them."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _both(spec, origin, shape):
    nx, ny, nz = shape
    want = synth.fill(spec, origin, shape)
    out = torch.full((nz, ny, nx), -1, dtype=torch.int32, device="cuda")
    synth.fill_gpu(spec, origin, shape, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return want, out.cpu().numpy().view(np.uint32)


RECIPES = [synth.c1(), synth.c2(), synth.c3(), synth.c4()] + synth.c5() + [
    synth.small(dims=(40, 24, 20)), synth.small(dims=(100, 90, 80), seed=9, grid=16, diameter=30.0, bg=0.3)]


@pytest.mark.parametrize("i", range(len(RECIPES)))
def test_gpu_generator_matches_cpu_generator(i):
    spec = RECIPES[i]
    rng = np.random.default_rng(100 + i)
    boxes = [((0, 0, 0), (48, 40, 36))]
    for _ in range(3):
        shape = tuple(int(s) for s in rng.integers(17, 70, size=3))
        origin = tuple(int(rng.integers(0, max(1, d - s))) for d, s in zip(spec.dims, shape))
        boxes.append((origin, shape))
    boxes.append(((-7, 3, -20), (33, 29, 41)))  # the definition covers every integer point
    for origin, shape in boxes:
        want, got = _both(spec, origin, shape)
        assert np.array_equal(want, got), (spec.name, origin, shape, int((want != got).sum()))


def test_gpu_generator_whole_small_volume_and_forced_uniform_bricks():
    spec = synth.c3()
    # a 128 x 96 x 64 corner of the power-diagram volume, several forced-uniform 32^3 bricks in it
    want, got = _both(spec, (0, 0, 0), (128, 96, 64))
    assert np.array_equal(want, got)
    bricks = want.reshape(2, 32, 3, 32, 4, 32).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 32 ** 3)
    assert ((bricks == bricks[:, :1]).all(axis=1)).sum() >= 3
