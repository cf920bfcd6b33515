"""CSGV oracle: plain single-threaded CPU encoder / decoder (ctypes over ``csgv_oracle.c``) and the
camera request stage (``camera_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg are
the only callers. The GPU library never imports this package and shares no code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "csgv_oracle.c"), os.path.join(_HERE, "camera_oracle.c"),
         os.path.join(_HERE, "render_oracle.c"), os.path.join(_HERE, "post_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

OP_PARENT, OP_NX, OP_NY, OP_NZ, OP_ADV, OP_LAST, OP_DELTA = range(7)
OP_ALL = 0x7F
CODER_PLAIN, CODER_RANS = 0, 1
FLAG_NO_STOP = 1
FLAG_SHORT_DELTA = 2  # limited delta: one 4-bit entry per delta operation holding delta - 1, 2 <= delta <= 16
FLAG_RUNS_SHIFT = 2   # bits 2..3: log2 of the rANS runs per record (1, 2, 4 or 8 independently coded runs)


def runs_flag(k: int) -> int:
    """The header flag bits of k rANS runs per record (k = 1, 2, 4, 8)."""
    return {1: 0, 2: 1, 4: 2, 8: 3}[k] << FLAG_RUNS_SHIFT
ERR_ARG, ERR_FORMAT, ERR_OOM, ERR_CORRUPT = -1, -2, -3, -5

NODE_DTYPE = np.dtype([("level", "<i4"), ("morton", "<u4"), ("op", "<i4"), ("stop", "<i4"),
                       ("delta", "<u4"), ("label", "<u4"), ("k", "<u4")])


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        super().__init__(f"oracle error {code} {what}".strip())
        self.code = code


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its sources (gcc, plain C11, no floating-point contraction)."""
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(s) for s in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fPIC", "-shared"] + _SRCS
                              + ["-lm", "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, U32, SZ = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_size_t
        lib.oracle_encode_volume.argtypes = [P, P, U32, U32, U32, U32, ctypes.POINTER(P), ctypes.POINTER(SZ)]
        lib.oracle_decode_brick.argtypes = [P, SZ, U32, U32, P]
        lib.oracle_decode_volume.argtypes = [P, SZ, P]
        lib.oracle_brick_nodes.argtypes = [P, SZ, U32, P, U32, P]
        lib.oracle_brick_symbols.argtypes = [P, SZ, U32, P, U32, P]
        lib.oracle_delta_nibbles.argtypes = [U32, P]
        lib.oracle_rans_quantize.argtypes = [P, P]
        lib.oracle_pack_single_brick.argtypes = [U32, U32, U32, U32, P, U32, P, U32, U32, ctypes.POINTER(P),
                                                 ctypes.POINTER(SZ)]
        lib.oracle_pack_bricks.argtypes = [U32, U32, U32, U32, U32, P, P, P, P, P, ctypes.POINTER(P),
                                           ctypes.POINTER(SZ)]
        lib.oracle_pack_bricks.restype = ctypes.c_int
        lib.oracle_free.argtypes = [P]
        lib.oracle_camera_bricks.argtypes = [P, SZ, P, P, P, ctypes.c_float, U32, U32, U32, P, P, U32, P]
        lib.oracle_camera_bricks.restype = ctypes.c_int
        lib.oracle_brick_lods.argtypes = [P, SZ, P, P, P, ctypes.c_float, U32, U32, U32, P]
        lib.oracle_brick_lods.restype = ctypes.c_int
        lib.oracle_head_words.argtypes = [U32, U32, U32]
        lib.oracle_head_words.restype = U32
        lib.oracle_render.argtypes = [P, SZ, P, P, P, P, P, P, ctypes.c_float, U32, U32, P, P, P, P, P]
        lib.oracle_render.restype = ctypes.c_int
        lib.oracle_post.argtypes = [P] * 14
        lib.oracle_post.restype = ctypes.c_int
        for f in ("oracle_encode_volume", "oracle_decode_brick", "oracle_decode_volume", "oracle_brick_nodes",
                  "oracle_brick_symbols", "oracle_delta_nibbles", "oracle_rans_quantize", "oracle_pack_single_brick"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _take(ptr: ctypes.c_void_p, size: int) -> np.ndarray:
    out = np.frombuffer(ctypes.string_at(ptr, size), dtype=np.uint8).copy()
    _load().oracle_free(ptr)
    return out


def encode_volume(V: np.ndarray, log2b: int, op_mask: int = OP_ALL, coder: int = CODER_PLAIN,
                  flags: int = 0) -> np.ndarray:
    """Encode a (z, y, x) uint32 volume; returns the encoded bytes as a uint8 array."""
    V = np.ascontiguousarray(V, dtype=np.uint32)
    assert V.ndim == 3
    dims = (ctypes.c_uint32 * 3)(V.shape[2], V.shape[1], V.shape[0])
    ptr, size = ctypes.c_void_p(), ctypes.c_size_t()
    rc = _load().oracle_encode_volume(V.ctypes.data, dims, log2b, op_mask, coder, flags, ctypes.byref(ptr),
                                      ctypes.byref(size))
    if rc:
        raise OracleError(rc, "encode")
    return _take(ptr, size.value)


def header(vol: np.ndarray) -> dict:
    h = np.frombuffer(vol[:128].tobytes(), dtype="<u4")
    L = int(h[5])
    b = 1 << L
    dims = (int(h[2]), int(h[3]), int(h[4]))
    nb = tuple((d + b - 1) // b for d in dims)
    return {"magic": int(h[0]), "version": int(h[1]), "dims": dims, "log2b": L, "b": b, "op_mask": int(h[6]),
            "coder": int(h[7]), "flags": int(h[8]), "n_bricks": int(h[9]), "max_pal": int(h[10]),
            "max_sym": int(h[11]), "freq": [int(x) for x in h[12:28]], "records_words": int(h[28]),
            "bricks_per_axis": nb}


def decode_brick(vol: np.ndarray, brick_id: int, lod: int = 0) -> np.ndarray:
    """Labels of one brick at level of detail lod, shape (n, n, n) with n = b >> lod (z, y, x)."""
    vol = np.ascontiguousarray(vol, dtype=np.uint8)
    n = header(vol)["b"] >> lod
    out = np.empty((max(n, 1),) * 3, dtype=np.uint32)
    rc = _load().oracle_decode_brick(vol.ctypes.data, vol.size, brick_id, lod, out.ctypes.data)
    if rc:
        raise OracleError(rc, f"decode brick {brick_id}")
    return out


def decode_brick_status(vol: np.ndarray, brick_id: int, lod: int = 0) -> int:
    """Status code (0 or negative) of decoding one brick."""
    vol = np.ascontiguousarray(vol, dtype=np.uint8)
    n = header(vol)["b"] >> lod
    out = np.empty((max(n, 1),) * 3, dtype=np.uint32)
    return int(_load().oracle_decode_brick(vol.ctypes.data, vol.size, brick_id, lod, out.ctypes.data))


def decode_volume(vol: np.ndarray) -> np.ndarray:
    vol = np.ascontiguousarray(vol, dtype=np.uint8)
    dx, dy, dz = header(vol)["dims"]
    out = np.empty((dz, dy, dx), dtype=np.uint32)
    rc = _load().oracle_decode_volume(vol.ctypes.data, vol.size, out.ctypes.data)
    if rc:
        raise OracleError(rc, "decode volume")
    return out


def brick_nodes(vol: np.ndarray, brick_id: int) -> np.ndarray:
    vol = np.ascontiguousarray(vol, dtype=np.uint8)
    b = header(vol)["b"]
    cap = sum(8 ** l for l in range(b.bit_length()))
    out = np.zeros(cap, dtype=NODE_DTYPE)
    n = ctypes.c_uint32()
    rc = _load().oracle_brick_nodes(vol.ctypes.data, vol.size, brick_id, out.ctypes.data, cap, ctypes.byref(n))
    if rc:
        raise OracleError(rc, f"nodes of brick {brick_id}")
    return out[: n.value]


def brick_symbols(vol: np.ndarray, brick_id: int) -> np.ndarray:
    vol = np.ascontiguousarray(vol, dtype=np.uint8)
    S = ctypes.c_uint32()
    rc = _load().oracle_brick_symbols(vol.ctypes.data, vol.size, brick_id, None, 0, ctypes.byref(S))
    if rc:
        raise OracleError(rc, "symbols")
    out = np.zeros(S.value, dtype=np.uint8)
    _load().oracle_brick_symbols(vol.ctypes.data, vol.size, brick_id, out.ctypes.data, S.value, ctypes.byref(S))
    return out


def brick_record(vol: np.ndarray, brick_id: int) -> dict:
    """Header fields and palette of one brick record."""
    h = header(vol)
    starts_off = 128
    a = int(np.frombuffer(vol[starts_off + 4 * brick_id: starts_off + 4 * brick_id + 8].tobytes(), "<u4")[0])
    e = int(np.frombuffer(vol[starts_off + 4 * brick_id: starts_off + 4 * brick_id + 8].tobytes(), "<u4")[1])
    rec_off = (128 + 4 * (h["n_bricks"] + 1) + 15) & ~15
    r = vol[rec_off + 4 * a: rec_off + 4 * e]
    w = np.frombuffer(r.tobytes(), dtype="<u4")
    n_pal, S, cb, nd = (int(x) for x in w[:4])
    ns = int(_load().oracle_head_words(h["coder"], h["flags"], S))
    pal = w[4 + ns: 4 + ns + n_pal].copy()
    return {"n_pal": n_pal, "n_sym": S, "coded_bytes": cb, "n_delta": nd, "palette": pal, "words": e - a,
            "offset_words": a}


def delta_nibbles(delta: int) -> list:
    out = (ctypes.c_uint8 * 16)()
    n = _load().oracle_delta_nibbles(delta, out)
    return [int(out[i]) for i in range(n)]


def rans_quantize(counts) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(counts, dtype=np.uint64))
    f = np.zeros(16, dtype=np.uint32)
    rc = _load().oracle_rans_quantize(c.ctypes.data, f.ctypes.data)
    if rc:
        raise OracleError(rc, "quantize")
    return f


def pack_single_brick(log2b: int, sym, palette, n_delta: int, op_mask: int = OP_ALL, coder: int = CODER_PLAIN,
                      flags: int = 0) -> np.ndarray:
    """A one-brick volume whose record holds exactly the given symbols and palette."""
    s = np.ascontiguousarray(np.asarray(sym, dtype=np.uint8))
    p = np.ascontiguousarray(np.asarray(palette, dtype=np.uint32))
    ptr, size = ctypes.c_void_p(), ctypes.c_size_t()
    rc = _load().oracle_pack_single_brick(log2b, op_mask, coder, flags, s.ctypes.data, s.size,
                                          p.ctypes.data if p.size else None, p.size, n_delta, ctypes.byref(ptr),
                                          ctypes.byref(size))
    if rc:
        raise OracleError(rc, "pack")
    return _take(ptr, size.value)


def pack_bricks(log2b: int, streams, op_mask: int = OP_ALL, coder: int = CODER_PLAIN, flags: int = 0) -> np.ndarray:
    """A volume of len(streams) bricks along x; streams = [(symbols, palette, n_delta), ...]."""
    sym = np.ascontiguousarray(np.concatenate([np.asarray(s, dtype=np.uint8) for s, _, _ in streams]))
    S = np.array([len(s) for s, _, _ in streams], dtype=np.uint32)
    pals = [np.asarray(p, dtype=np.uint32) for _, p, _ in streams]
    pal = np.ascontiguousarray(np.concatenate(pals)) if sum(p.size for p in pals) else np.zeros(1, np.uint32)
    npal = np.array([p.size for p in pals], dtype=np.uint32)
    nd = np.array([d for _, _, d in streams], dtype=np.uint32)
    ptr, size = ctypes.c_void_p(), ctypes.c_size_t()
    rc = _load().oracle_pack_bricks(log2b, op_mask, coder, flags, len(streams), sym.ctypes.data, S.ctypes.data,
                                    pal.ctypes.data, npal.ctypes.data, nd.ctypes.data, ctypes.byref(ptr),
                                    ctypes.byref(size))
    if rc:
        raise OracleError(rc, "pack_bricks")
    return _take(ptr, size.value)


def camera_bricks(vol: np.ndarray, pos, dir, up, fov_y: float, width: int, height: int, max_lod: int = 31):
    """Bricks that a pinhole camera's pixel rays request (ascending ids) and their levels of detail."""
    vol = np.ascontiguousarray(vol, dtype=np.uint8)
    f3 = lambda v: np.ascontiguousarray(np.asarray(v, dtype=np.float32).reshape(3))  # noqa: E731
    p, d, u = f3(pos), f3(dir), f3(up)
    n_out = ctypes.c_uint32()
    lib = _load()
    rc = lib.oracle_camera_bricks(vol.ctypes.data, vol.size, p.ctypes.data, d.ctypes.data, u.ctypes.data,
                                  ctypes.c_float(fov_y), width, height, max_lod, None, None, 0, ctypes.byref(n_out))
    if rc not in (0, -7):
        raise OracleError(rc, "camera bricks")
    n = n_out.value
    ids = np.zeros(max(n, 1), dtype=np.uint32)
    lods = np.zeros(max(n, 1), dtype=np.uint32)
    rc = lib.oracle_camera_bricks(vol.ctypes.data, vol.size, p.ctypes.data, d.ctypes.data, u.ctypes.data,
                                  ctypes.c_float(fov_y), width, height, max_lod, ids.ctypes.data, lods.ctypes.data, n,
                                  ctypes.byref(n_out))
    if rc:
        raise OracleError(rc, "camera bricks")
    return ids[:n], lods[:n]


def brick_lods(vol: np.ndarray, pos, dir, up, fov_y: float, width: int, height: int, max_lod: int = 31) -> np.ndarray:
    """Every brick's level of detail for one camera (the request stage's centre rule), uint8."""
    vol = np.ascontiguousarray(vol, dtype=np.uint8)
    f3 = lambda v: np.ascontiguousarray(np.asarray(v, dtype=np.float32).reshape(3))  # noqa: E731
    p, d, u = f3(pos), f3(dir), f3(up)
    out = np.zeros(max(1, int(header(vol)["n_bricks"])), np.uint8)
    rc = _load().oracle_brick_lods(vol.ctypes.data, vol.size, p.ctypes.data, d.ctypes.data, u.ctypes.data,
                                   ctypes.c_float(fov_y), width, height, max_lod, out.ctypes.data)
    if rc:
        raise OracleError(rc, "brick lods")
    return out[:int(header(vol)["n_bricks"])]


class _RenderParams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("frame", ctypes.c_uint32), ("jitter", ctypes.c_uint32),
                ("max_bounces", ctypes.c_uint32), ("light_dir", ctypes.c_float * 3), ("ambient", ctypes.c_float),
                ("ao_radius", ctypes.c_float), ("sky", ctypes.c_float), ("n_materials", ctypes.c_uint32),
                ("materials", ctypes.c_void_p), ("subsample", ctypes.c_uint32), ("visible", ctypes.c_void_p),
                ("request_depth", ctypes.c_uint32)]


def render(vol: np.ndarray, offsets: np.ndarray, lods: np.ndarray, cache: np.ndarray, pos, dir, up, fov_y: float,
           width: int, height: int, materials: np.ndarray, mode: int = 0, frame: int = 0, jitter: bool = False,
           max_bounces: int = 8, light_dir=(0.3, 0.5, 0.8), ambient: float = 0.25, ao_radius: float = 8.0,
           sky: float = 1.0, subsample: int = 1, out=None, visible=None, request_depth: int = 1):
    """What each pixel ray sees (render_oracle.c): (labels, depth, face, rgb) as (H, W) arrays and
    (H, W, 3). offsets / lods / cache: per brick the word offset of its labels at its level of
    detail in cache (x fastest; 2**64 - 1 = not decoded) and the level. materials: (n, 4) float32
    rows (r, g, b, opacity). visible: a uint8 array of one entry per brick (or None) in which the
    bricks the rays of path depth <= request_depth access are set to 1."""
    vol = np.ascontiguousarray(vol, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    lods = np.ascontiguousarray(lods, dtype=np.uint8)
    cache = np.ascontiguousarray(cache, dtype=np.uint32)
    mats = np.ascontiguousarray(materials, dtype=np.float32)
    p = _RenderParams(mode, frame, int(bool(jitter)), max_bounces, (ctypes.c_float * 3)(*light_dir), ambient,
                      ao_radius, sky, mats.shape[0], mats.ctypes.data, subsample, None, request_depth)
    if visible is not None:
        n_bricks = int.from_bytes(bytes(vol[36:40]), "little")
        if visible.dtype != np.uint8 or not visible.flags.c_contiguous or visible.size < n_bricks:
            raise ValueError("visible must be a contiguous uint8 array of one entry per brick")
        p.visible = visible.ctypes.data
    f3 = lambda v: np.ascontiguousarray(v, dtype=np.float32)  # noqa: E731
    ps, ds, us = f3(pos), f3(dir), f3(up)
    if out is None:  # pixels outside this frame's subset keep what `out` holds
        out = (np.zeros((height, width), np.uint32), np.zeros((height, width), np.float32),
               np.zeros((height, width), np.uint8), np.zeros((height, width, 3), np.float32))
    labels, depth, face, rgb = out
    rc = _load().oracle_render(vol.ctypes.data, vol.size, offsets.ctypes.data, lods.ctypes.data, cache.ctypes.data,
                               ps.ctypes.data, ds.ctypes.data, us.ctypes.data, fov_y, width, height, ctypes.byref(p),
                               labels.ctypes.data, depth.ctypes.data, face.ctypes.data, rgb.ctypes.data)
    if rc:
        raise OracleError(rc, "render")
    return labels, depth, face, rgb


class _PostParams(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("height", ctypes.c_uint32), ("iterations", ctypes.c_uint32),
                ("subsample", ctypes.c_uint32), ("frame", ctypes.c_uint32), ("reset", ctypes.c_uint32),
                ("cam_pos", ctypes.c_float * 3), ("phi_rho", ctypes.c_float), ("phi_d", ctypes.c_float),
                ("exposure", ctypes.c_float), ("gamma", ctypes.c_float), ("n_materials", ctypes.c_uint32),
                ("materials", ctypes.c_void_p)]


def post_state(width: int, height: int) -> dict:
    """Per-pixel state of post() (kept by the caller between frames)."""
    n = width * height
    return {"accum": np.zeros((n, 4), np.float32), "col0": np.zeros((n, 4), np.float32),
            "col1": np.zeros((n, 4), np.float32), "glabel": np.zeros(n, np.uint32),
            "gcode": np.full(n, 7, np.uint32), "off0": np.zeros(n, np.int32), "off1": np.zeros(n, np.int32)}


def post(state: dict, dims, labels, depth, face, rgb, materials, cam_pos, iterations: int = 3, subsample: int = 1,
         frame: int = 0, reset: bool = False, phi_rho: float = 8.0, phi_d: float = 1.0, exposure: float = 1.0,
         gamma: float = 2.2) -> np.ndarray:
    """One frame of post-processing (post_oracle.c): the (H, W) RGBA8 image as uint32."""
    H, W = labels.shape
    mats = np.ascontiguousarray(materials, dtype=np.float32)
    p = _PostParams(W, H, iterations, subsample, frame, int(bool(reset)), (ctypes.c_float * 3)(*cam_pos), phi_rho,
                    phi_d, exposure, gamma, mats.shape[0], mats.ctypes.data)
    dims_a = np.ascontiguousarray(dims, dtype=np.uint32)
    c = lambda a, t: np.ascontiguousarray(a, dtype=t)  # noqa: E731
    labels, depth, face, rgb = c(labels, np.uint32), c(depth, np.float32), c(face, np.uint8), c(rgb, np.float32)
    out = np.zeros((H, W), np.uint32)
    S = state
    rc = _load().oracle_post(ctypes.byref(p), dims_a.ctypes.data, labels.ctypes.data, depth.ctypes.data,
                             face.ctypes.data, rgb.ctypes.data, S["accum"].ctypes.data, S["col0"].ctypes.data,
                             S["col1"].ctypes.data, S["glabel"].ctypes.data, S["gcode"].ctypes.data,
                             S["off0"].ctypes.data, S["off1"].ctypes.data, out.ctypes.data)
    if rc:
        raise OracleError(rc, "post")
    return out
