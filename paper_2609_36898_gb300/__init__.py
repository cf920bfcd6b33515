"""Python binding of libvc.so (the C ABI in include/vc.h): argument marshalling only.

Every step of decoding runs in the library's CUDA kernels; PyTorch is used for device memory and
streams. If libvc.so is missing the import of the native library fails loudly; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvc.so")

VC_OK = 0
VC_ERR_ARG = -1
VC_ERR_FORMAT = -2
VC_ERR_OOM = -3
VC_ERR_CUDA = -4
VC_ERR_CORRUPT = -5
VC_ERR_TIMEOUT = -6
VC_ERR_BUSY = -7
VC_ERR_UNSUPPORTED = -8
VC_STATUS_WORDS = 4
VC_MODE_PLAIN, VC_MODE_GRID, VC_MODE_BATCHED, VC_MODE_PIPELINED = 0, 1, 2, 3
MODES = {"plain": VC_MODE_PLAIN, "grid": VC_MODE_GRID, "batched": VC_MODE_BATCHED, "pipelined": VC_MODE_PIPELINED}


class VCError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        msg = _lib_handle().vc_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})" if where else f"{msg} ({code})")


class vc_volume_info(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_uint32 * 3),
        ("brick_size", ctypes.c_uint32),
        ("log2b", ctypes.c_uint32),
        ("n_bricks", ctypes.c_uint32),
        ("bricks_per_axis", ctypes.c_uint32 * 3),
        ("op_mask", ctypes.c_uint32),
        ("coder", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("max_pal", ctypes.c_uint32),
        ("max_sym", ctypes.c_uint32),
        ("max_delta", ctypes.c_uint32),
        ("encoded_bytes", ctypes.c_uint64),
        ("device_bytes", ctypes.c_uint64),
        ("smem_bytes", ctypes.c_uint32),
        ("device", ctypes.c_uint32),
    ]


class vc_schedule(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_uint32), ("stage_depth", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("chunk", ctypes.c_uint32)]


class vc_kernel_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("timed_calls", ctypes.c_uint32), ("dropped_calls", ctypes.c_uint32),
                ("symbol_ms", ctypes.c_double), ("reconstruct_ms", ctypes.c_double)]


_lib = None


def _lib_handle():
    """Loads libvc.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libvc.so not built ({LIB_PATH}); run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        P, U32, I32, SZ = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32, ctypes.c_size_t
        lib.vc_load_compressed.argtypes = [P, SZ, ctypes.c_int, P, ctypes.POINTER(P)]
        lib.vc_volume_info_get.argtypes = [P, ctypes.POINTER(vc_volume_info)]
        lib.vc_volume_set_schedule.argtypes = [P, ctypes.POINTER(vc_schedule)]
        lib.vc_volume_get_schedule.argtypes = [P, ctypes.POINTER(vc_schedule)]
        lib.vc_decode_bricks.argtypes = [P, P, U32, P, P, U32, U32, P, P]
        lib.vc_decode_bricks_noalloc.argtypes = [P, P, U32, P, P, U32, U32, P, P]
        lib.vc_decode_bricks_host.argtypes = [P, P, U32, U32, U32, P, ctypes.POINTER(I32), P]
        lib.vc_release.argtypes = [P]
        lib.vc_volume_set_profiling.argtypes = [P, ctypes.c_int]
        lib.vc_volume_kernel_stats.argtypes = [P, ctypes.c_int, ctypes.POINTER(vc_kernel_stats)]
        lib.vc_encode_volume.argtypes = [P, P, U32, U32, U32, U32, U32, ctypes.POINTER(P), ctypes.POINTER(SZ)]
        lib.vc_free_bytes.argtypes = [P]
        lib.vc_free_bytes.restype = None
        lib.vc_status_string.argtypes = [I32]
        lib.vc_status_string.restype = ctypes.c_char_p
        for f in ("vc_load_compressed", "vc_volume_info_get", "vc_decode_bricks", "vc_decode_bricks_host",
                  "vc_release", "vc_encode_volume", "vc_volume_set_schedule", "vc_volume_get_schedule",
                  "vc_volume_set_profiling", "vc_volume_kernel_stats", "vc_decode_bricks_noalloc"):
            getattr(lib, f).restype = I32
        _lib = lib
    return _lib


def _check(rc: int, where: str):
    if rc != VC_OK:
        raise VCError(rc, where)


# ------------------------------------------------------------------ C-ABI mirrors (same names)

def vc_load_compressed(host_bytes: np.ndarray, device: int = 0, stream: int = 0) -> ctypes.c_void_p:
    b = np.ascontiguousarray(host_bytes, dtype=np.uint8)
    out = ctypes.c_void_p()
    _check(_lib_handle().vc_load_compressed(b.ctypes.data, b.size, device, ctypes.c_void_p(stream),
                                            ctypes.byref(out)), "vc_load_compressed")
    return out


def vc_volume_info_get(vol) -> vc_volume_info:
    info = vc_volume_info()
    _check(_lib_handle().vc_volume_info_get(vol, ctypes.byref(info)), "vc_volume_info_get")
    return info


def vc_volume_set_schedule(vol, threads: int, stage_depth: int = 1, blocks_per_sm: int = 0, chunk: int = 0) -> None:
    s = vc_schedule(threads, stage_depth, blocks_per_sm, chunk)
    _check(_lib_handle().vc_volume_set_schedule(vol, ctypes.byref(s)), "vc_volume_set_schedule")


def vc_volume_get_schedule(vol) -> tuple:
    s = vc_schedule()
    _check(_lib_handle().vc_volume_get_schedule(vol, ctypes.byref(s)), "vc_volume_get_schedule")
    return (s.threads, s.stage_depth, s.blocks_per_sm, s.chunk)


def vc_decode_bricks(vol, brick_ids_ptr: int, n: int, cache_slots_ptr: int, cache_ptr: int, lod: int, mode: int,
                     status_ptr: int, stream: int = 0) -> None:
    _check(_lib_handle().vc_decode_bricks(vol, ctypes.c_void_p(brick_ids_ptr), n, ctypes.c_void_p(cache_slots_ptr),
                                          ctypes.c_void_p(cache_ptr), lod, mode, ctypes.c_void_p(status_ptr),
                                          ctypes.c_void_p(stream)), "vc_decode_bricks")


def vc_decode_bricks_noalloc(vol, brick_ids_ptr: int, n: int, cache_slots_ptr: int, cache_ptr: int, lod: int,
                             mode: int, status_ptr: int, stream: int = 0) -> None:
    _check(_lib_handle().vc_decode_bricks_noalloc(vol, ctypes.c_void_p(brick_ids_ptr), n,
                                                  ctypes.c_void_p(cache_slots_ptr), ctypes.c_void_p(cache_ptr), lod,
                                                  mode, ctypes.c_void_p(status_ptr), ctypes.c_void_p(stream)),
           "vc_decode_bricks_noalloc")


def vc_decode_bricks_host(vol, brick_ids: np.ndarray, lod: int, mode: int, labels_out: np.ndarray,
                          stream: int = 0) -> int:
    ids = np.ascontiguousarray(brick_ids, dtype=np.uint32)
    assert labels_out.dtype == np.uint32 and labels_out.flags.c_contiguous
    st = ctypes.c_int32()
    _check(_lib_handle().vc_decode_bricks_host(vol, ids.ctypes.data, ids.size, lod, mode, labels_out.ctypes.data,
                                               ctypes.byref(st), ctypes.c_void_p(stream)), "vc_decode_bricks_host")
    return st.value


def vc_volume_set_profiling(vol, enable: bool) -> None:
    _check(_lib_handle().vc_volume_set_profiling(vol, int(bool(enable))), "vc_volume_set_profiling")


def vc_volume_kernel_stats(vol, reset: bool = False) -> vc_kernel_stats:
    st = vc_kernel_stats()
    _check(_lib_handle().vc_volume_kernel_stats(vol, int(bool(reset)), ctypes.byref(st)), "vc_volume_kernel_stats")
    return st


def vc_release(handle) -> None:
    _check(_lib_handle().vc_release(handle), "vc_release")


def vc_encode_volume(V: np.ndarray, log2b: int, op_mask: int = 0x7F, coder: int = 0, flags: int = 0,
                     threads: int = 0) -> np.ndarray:
    """Encode a (z, y, x) uint32 volume with the library's multi-threaded CPU encoder."""
    V = np.ascontiguousarray(V, dtype=np.uint32)
    dims = (ctypes.c_uint32 * 3)(V.shape[2], V.shape[1], V.shape[0])
    ptr, size = ctypes.c_void_p(), ctypes.c_size_t()
    lib = _lib_handle()
    _check(lib.vc_encode_volume(V.ctypes.data, dims, log2b, op_mask, coder, flags, threads, ctypes.byref(ptr),
                                ctypes.byref(size)), "vc_encode_volume")
    out = np.frombuffer(ctypes.string_at(ptr, size.value), dtype=np.uint8).copy()
    lib.vc_free_bytes(ptr)
    return out


# ------------------------------------------------------------------ convenience wrapper (torch)

class Volume:
    """A compressed volume resident on a CUDA device."""

    def __init__(self, encoded: np.ndarray, device: int = 0, stream=None):
        import torch
        self.device = device
        s = stream if stream is not None else torch.cuda.current_stream(device)
        self.handle = vc_load_compressed(encoded, device, s.cuda_stream)
        self.info = vc_volume_info_get(self.handle)
        self.b = int(self.info.brick_size)
        self.L = int(self.info.log2b)
        self.n_bricks = int(self.info.n_bricks)

    def set_schedule(self, threads: int, stage_depth: int = 1, blocks_per_sm: int = 0, chunk: int = 0) -> None:
        vc_volume_set_schedule(self.handle, threads, stage_depth, blocks_per_sm, chunk)
        self.info = vc_volume_info_get(self.handle)

    def edge(self, lod: int = 0) -> int:
        return self.b >> lod

    def decode(self, brick_ids, slots, cache, lod: int = 0, mode: str | int = "batched", status=None, stream=None):
        """Decode into `cache` (uint32/int32 CUDA tensor); ids/slots are CUDA uint32-compatible tensors."""
        import torch
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        n = int(brick_ids.numel())
        if status is None:
            status = torch.zeros(VC_STATUS_WORDS, dtype=torch.int32, device=cache.device)
        s = stream if stream is not None else torch.cuda.current_stream(cache.device)
        vc_decode_bricks(self.handle, brick_ids.data_ptr(), n, slots.data_ptr(), cache.data_ptr(), lod, m,
                         status.data_ptr(), s.cuda_stream)
        return status

    def release(self):
        if self.handle:
            vc_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass
