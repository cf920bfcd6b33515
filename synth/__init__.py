"""Seeded synthetic segmentation volumes (noise-perturbed Voronoi / power-diagram cells).

Thin ctypes wrapper over ``synth.c``. This module produces input volumes only; it holds none of
the compression method's arithmetic, so both the CPU oracle and the GPU path may consume it.
The per-workload recipes (cell sizes, background fraction, brick sizes) stand in for the
connectomics segmentations the paper evaluates on (Results, "CSGV results").
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_SRC_GPU = os.path.join(_HERE, "synth_gpu.cu")
_LIB_GPU = os.path.join(_HERE, "libsynth_gpu.so")
_lib = None
_lib_gpu = None


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return "nvcc"


def build(force: bool = False) -> str:
    """Compile libsynth.so next to its source (gcc, plain C11 + pthreads), and the GPU generator
    libsynth_gpu.so (nvcc, sm_103a) when nvcc is present."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    nvcc = _nvcc()
    if (force or not os.path.exists(_LIB_GPU) or os.path.getmtime(_LIB_GPU) < os.path.getmtime(_SRC_GPU)) and \
            (os.path.exists(nvcc) or nvcc == "nvcc"):
        tmp = _LIB_GPU + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-gencode",
                               "arch=compute_103a,code=sm_103a", _SRC_GPU, "-o", tmp])
        os.replace(tmp, _LIB_GPU)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_uint32 * 3),
        ("grid", ctypes.c_uint32),
        ("seed", ctypes.c_uint64),
        ("lambda_q16", ctypes.c_uint32),
        ("bg_q16", ctypes.c_uint32),
        ("amp_q16", ctypes.c_uint32),
        ("rmean_q16", ctypes.c_uint32),
        ("uniform_brick", ctypes.c_uint32),
        ("uniform_q16", ctypes.c_uint32),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.synth_fill.argtypes = [ctypes.POINTER(_Params), ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int]
        lib.synth_fill.restype = ctypes.c_int
        _lib = lib
    return _lib


def _load_gpu():
    """The GPU generator (libsynth_gpu.so), with the power-diagram weight table of synth.c."""
    global _lib_gpu
    if _lib_gpu is None:
        build()
        lib = ctypes.CDLL(_LIB_GPU)
        lib.synth_fill_gpu.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_fill_gpu.restype = ctypes.c_int
        lib.synth_gpu_set_lognorm.argtypes = [ctypes.c_void_p]
        lib.synth_gpu_set_lognorm.restype = ctypes.c_int
        cpu = _load()
        cpu.synth_lognorm_table.restype = ctypes.c_void_p
        if lib.synth_gpu_set_lognorm(cpu.synth_lognorm_table()) != 0:
            raise RuntimeError("synth_gpu_set_lognorm failed")
        _lib_gpu = lib
    return _lib_gpu


def _q16(x: float) -> int:
    return int(round(x * 65536.0))


@dataclass
class VolumeSpec:
    """Recipe of one synthetic volume.

    dims: voxels (x, y, z). grid: hash-grid edge g. lam: mean seeds per hash-grid cell.
    bg: background probability per seed. amp: boundary displacement amplitude (voxels).
    rmean: mean power-diagram radius (0 = plain Voronoi). uniform_brick / uniform_p: bricks
    forced to one label. brick: the brick edge b used to encode it.
    """
    dims: tuple
    grid: int
    seed: int
    lam: float
    bg: float = 0.0
    amp: float = 2.0
    rmean: float = 0.0
    uniform_brick: int = 0
    uniform_p: float = 0.0
    brick: int = 32
    name: str = ""

    def _c(self) -> _Params:
        p = _Params()
        for a in range(3):
            p.dims[a] = int(self.dims[a])
        p.grid = int(self.grid)
        p.seed = int(self.seed) & ((1 << 64) - 1)
        p.lambda_q16 = _q16(self.lam)
        p.bg_q16 = _q16(self.bg)
        p.amp_q16 = _q16(self.amp)
        p.rmean_q16 = _q16(self.rmean)
        p.uniform_brick = int(self.uniform_brick)
        p.uniform_q16 = _q16(self.uniform_p)
        return p

    @property
    def n_voxels(self) -> int:
        return int(self.dims[0]) * int(self.dims[1]) * int(self.dims[2])


def fill(spec: VolumeSpec, origin=(0, 0, 0), shape=None, nthreads: int | None = None,
         out: np.ndarray | None = None) -> np.ndarray:
    """Labels of the box [origin, origin + shape) as a (z, y, x) uint32 array (x fastest)."""
    if shape is None:
        shape = tuple(int(d) - int(o) for d, o in zip(spec.dims, origin))
    nx, ny, nz = (int(s) for s in shape)
    if out is None:
        out = np.empty((nz, ny, nx), dtype=np.uint32)
    assert out.dtype == np.uint32 and out.flags.c_contiguous and out.size == nx * ny * nz
    if nthreads is None:
        nthreads = max(1, min(64, os.cpu_count() or 1))
    p = spec._c()
    rc = _load().synth_fill(ctypes.byref(p), int(origin[0]), int(origin[1]), int(origin[2]), nx, ny, nz,
                            out.ctypes.data, int(nthreads))
    if rc != 0:
        raise ValueError("synth_fill rejected the parameters")
    return out


def fill_gpu(spec: VolumeSpec, origin, shape, out_ptr: int, stream: int = 0) -> None:
    """The same labels as fill(), written by the GPU generator into device memory at out_ptr
    (nx * ny * nz uint32, x fastest), asynchronously on the CUDA stream `stream`."""
    nx, ny, nz = (int(s) for s in shape)
    p = spec._c()
    rc = _load_gpu().synth_fill_gpu(ctypes.byref(p), int(origin[0]), int(origin[1]), int(origin[2]), nx, ny, nz,
                                    ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream))
    if rc == -1:
        raise ValueError("synth_fill_gpu rejected the parameters")
    if rc != 0:
        raise RuntimeError("synth_fill_gpu: CUDA error")


def _lam_for(grid: int, diameter: float) -> float:
    """Seeds per hash-grid cell so that cells have the volume of a sphere of this diameter."""
    return grid ** 3 / (math.pi / 6.0 * diameter ** 3)


# Workload recipes. Sizes, cell counts, background fractions and brick sizes follow the
# benchmark configurations; everything is seeded.
def c1() -> VolumeSpec:
    """64^3, 32^3 bricks (8), ~40 cells, 20% background."""
    return VolumeSpec(dims=(64, 64, 64), grid=16, seed=1, lam=40 / 64, bg=0.2, brick=32, name="c1_64cube_b32")


def c2() -> VolumeSpec:
    """512^3, 32^3 bricks (4096), ~20k cells (mean diameter ~23 voxels), 10% background."""
    return VolumeSpec(dims=(512, 512, 512), grid=16, seed=2, lam=20000 / 32768, bg=0.1, brick=32,
                      name="c2_512cube_b32")


def c3() -> VolumeSpec:
    """2048x2048x1024, 32^3 bricks (131072), ~2M power-diagram cells with log-normal radii
    (sigma 0.8), 30% of bricks forced uniform."""
    spacing = (2048 * 2048 * 1024 / 2.0e6) ** (1.0 / 3.0)
    return VolumeSpec(dims=(2048, 2048, 1024), grid=16, seed=3, lam=2.0e6 / (128 * 128 * 64), bg=0.1,
                      rmean=spacing / 2.0, uniform_brick=32, uniform_p=0.3, brick=32, name="c3_2048x2048x1024_b32")


def c4() -> VolumeSpec:
    """4096^3 hash-grid Voronoi, one seed per 16^3 grid cell on average (~16M cells)."""
    return VolumeSpec(dims=(4096, 4096, 4096), grid=16, seed=4, lam=1.0, bg=0.1, brick=32, name="c4_4096cube_b32")


def c4_scaled(n: int = 1024) -> VolumeSpec:
    """The 4096^3 recipe (one seed per 16^3 grid cell on average, 10% background) on an n^3 box."""
    return VolumeSpec(dims=(n, n, n), grid=16, seed=4, lam=1.0, bg=0.1, brick=32, name=f"c4_{n}cube_b32")


def c5() -> list:
    """The 8 resident volumes of the mixed serving workload: (dims, brick, cell diameter, background)."""
    rows = [(256, 16, 8, 0.0), (256, 32, 16, 0.1), (512, 32, 24, 0.2), (512, 64, 32, 0.4),
            (1024, 16, 12, 0.05), (1024, 32, 48, 0.3), (2048, 64, 64, 0.15), (2048, 32, 20, 0.1)]
    out = []
    for i, (n, b, d, bg) in enumerate(rows):
        g = 8 if d <= 12 else (16 if d <= 24 else (32 if d <= 48 else 64))
        out.append(VolumeSpec(dims=(n, n, n), grid=g, seed=50 + i, lam=_lam_for(g, d), bg=bg, brick=b,
                              name=f"c5_{i}_{n}cube_b{b}_d{d}"))
    return out


def small(dims=(40, 24, 20), seed=7, grid=8, diameter=10.0, bg=0.2, brick=8, **kw) -> VolumeSpec:
    """A small volume for oracle tests (ragged sizes allowed)."""
    return VolumeSpec(dims=tuple(dims), grid=grid, seed=seed, lam=min(8.0, _lam_for(grid, diameter)), bg=bg,
                      brick=brick, **kw)
