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
VC_MODE_PALETTED = 0x100
VC_FLAG_NO_STOP, VC_FLAG_SHORT_DELTA = 1, 2


def VC_FLAG_RUNS(k: int) -> int:
    """Encoding flag bits of k (1, 2, 4, 8) independently coded rANS runs per record."""
    return {1: 0, 2: 4, 4: 8, 8: 12}[k]
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
        ("split", ctypes.c_uint32),
        ("host_bytes", ctypes.c_uint64),
    ]


class vc_schedule(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_uint32), ("stage_depth", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("chunk", ctypes.c_uint32)]


class vc_kernel_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("timed_calls", ctypes.c_uint32), ("dropped_calls", ctypes.c_uint32),
                ("symbol_ms", ctypes.c_double), ("reconstruct_ms", ctypes.c_double)]


class vc_server_config(ctypes.Structure):
    _fields_ = [("cache_bytes", ctypes.c_uint64), ("device", ctypes.c_int32), ("max_batch_items", ctypes.c_uint32),
                ("max_inflight", ctypes.c_uint32), ("min_class", ctypes.c_uint32), ("max_class", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 2)]


class vc_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("volume_index", ctypes.c_uint32),
                ("n_bricks", ctypes.c_uint32), ("hits", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("bytes", ctypes.c_uint64), ("t_submit_ns", ctypes.c_uint64), ("t_admit_ns", ctypes.c_uint64),
                ("t_done_ns", ctypes.c_uint64)]


class vc_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "cache_bytes", "cache_free_bytes", "cache_evictable_bytes", "cache_entries", "evictions",
        "requests_submitted", "requests_admitted", "requests_done", "requests_failed", "requests_waiting",
        "bricks_hit", "bricks_missed", "bricks_decoded", "batches", "batches_inflight", "batch_errors",
        "voxels_decoded", "graph_launches", "graph_instantiations")]


class vc_brick_cache_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "capacity_bytes", "free_bytes", "evictable_bytes", "entries", "evictions", "hits", "misses")]


class vc_camera(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_float * 3), ("dir", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("fov_y", ctypes.c_float), ("width", ctypes.c_uint32), ("height", ctypes.c_uint32)]


def make_camera(pos, dir, up, fov_y: float, width: int, height: int) -> vc_camera:
    f3 = ctypes.c_float * 3
    return vc_camera(f3(*[float(x) for x in pos]), f3(*[float(x) for x in dir]), f3(*[float(x) for x in up]),
                     float(fov_y), int(width), int(height))


VC_REQ_WAITING, VC_REQ_ADMITTED, VC_REQ_DONE, VC_REQ_FAILED = 0, 1, 2, 3


class vc_frame_cache_view(ctypes.Structure):
    _fields_ = [("offsets", ctypes.c_void_p), ("lods", ctypes.c_void_p), ("cache", ctypes.c_void_p),
                ("marks", ctypes.c_void_p), ("cache_words", ctypes.c_uint64), ("n_bricks", ctypes.c_uint32),
                ("max_bricks_per_frame", ctypes.c_uint32), ("free_stack_entries", ctypes.c_uint32)]


class vc_frame_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "frames", "bricks_requested", "bricks_decoded", "voxels_decoded", "bricks_freed", "bricks_unassigned",
        "resets", "level_switches", "top_words", "dead_words")] + [(n, ctypes.c_uint32) for n in (
            "last_resident", "last_requested", "last_decoded", "last_unassigned", "last_freed", "reset_pending")] + [
        ("free_entries", ctypes.c_uint32 * 8)]

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
        lib.vc_load_compressed_split.argtypes = [P, SZ, ctypes.c_int, P, ctypes.POINTER(P)]
        lib.vc_split_counts.argtypes = [P, SZ, U32, P]
        lib.vc_volume_info_get.argtypes = [P, ctypes.POINTER(vc_volume_info)]
        lib.vc_volume_set_schedule.argtypes = [P, ctypes.POINTER(vc_schedule)]
        lib.vc_volume_get_schedule.argtypes = [P, ctypes.POINTER(vc_schedule)]
        lib.vc_decode_bricks.argtypes = [P, P, U32, P, P, U32, U32, P, P]
        lib.vc_decode_bricks_noalloc.argtypes = [P, P, U32, P, P, U32, U32, P, P]
        lib.vc_decode_bricks_host.argtypes = [P, P, U32, U32, U32, P, ctypes.POINTER(I32), P]
        lib.vc_coarsest_labels.argtypes = [P, P, U32, P, P, P]
        lib.vc_release.argtypes = [P]
        lib.vc_volume_set_profiling.argtypes = [P, ctypes.c_int]
        lib.vc_volume_kernel_stats.argtypes = [P, ctypes.c_int, ctypes.POINTER(vc_kernel_stats)]
        lib.vc_encode_volume.argtypes = [P, P, U32, U32, U32, U32, U32, ctypes.POINTER(P), ctypes.POINTER(SZ)]
        lib.vc_encode_volume_freq.argtypes = [P, P, U32, U32, U32, U32, U32, P, ctypes.POINTER(P), ctypes.POINTER(SZ)]
        lib.vc_concat_volumes_z.argtypes = [P, P, U32, ctypes.POINTER(P), ctypes.POINTER(SZ)]
        PU64 = ctypes.POINTER(ctypes.c_uint64)
        lib.vc_server_create.argtypes = [ctypes.POINTER(vc_server_config), ctypes.POINTER(P)]
        lib.vc_server_add_volume.argtypes = [P, P, ctypes.POINTER(U32)]
        lib.vc_submit_bricks.argtypes = [P, U32, P, P, U32, PU64]
        lib.vc_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(I32), P]
        lib.vc_wait.argtypes = [P, ctypes.c_uint64, U32, ctypes.POINTER(I32)]
        lib.vc_request_info_get.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(vc_request_info)]
        lib.vc_request_release.argtypes = [P, ctypes.c_uint64]
        lib.vc_server_cache.argtypes = [P, ctypes.POINTER(P), PU64]
        lib.vc_server_stats_get.argtypes = [P, ctypes.POINTER(vc_server_stats)]
        lib.vc_volume_autotune.argtypes = [P, P, U32, P, P, U32, P, P, U32, ctypes.POINTER(vc_schedule),
                                           ctypes.POINTER(U32), ctypes.POINTER(ctypes.c_float)]
        lib.vc_volume_autotune.restype = I32
        lib.vc_volume_slot_words.argtypes = [P, U32, U32, ctypes.POINTER(U32), ctypes.POINTER(U32), ctypes.POINTER(U32)]
        lib.vc_volume_slot_words.restype = I32
        lib.vc_camera_bricks.argtypes = [P, P, U32, U32, U32, P, P, P, P]
        lib.vc_request_bricks.argtypes = [P, U32, P, U32, U32, P]
        lib.vc_camera_bricks.restype = I32
        lib.vc_request_bricks.restype = I32
        lib.vc_brick_cache_create.argtypes = [ctypes.c_uint64, U32, U32, ctypes.POINTER(P)]
        lib.vc_brick_cache_acquire.argtypes = [P, P, P, U32, P, P, P]
        lib.vc_brick_cache_unpin.argtypes = [P, P, U32]
        lib.vc_brick_cache_invalidate.argtypes = [P, U32]
        lib.vc_brick_cache_stats_get.argtypes = [P, ctypes.POINTER(vc_brick_cache_stats)]
        lib.vc_request_coarsest.argtypes = [P, ctypes.c_uint64, P, P, P]
        lib.vc_render.argtypes = [P, P, P, P, ctypes.POINTER(vc_camera), ctypes.POINTER(vc_render_params), P, P, P, P,
                                  P]
        lib.vc_render.restype = I32
        lib.vc_post_state_bytes.argtypes = [U32, U32]
        lib.vc_post_state_bytes.restype = SZ
        lib.vc_postprocess.argtypes = [P, ctypes.POINTER(vc_post_params), P, P, P, P, P, P, P]
        lib.vc_postprocess.restype = I32
        lib.vc_selftest_bounded_wait.argtypes = [U32, P, P]
        lib.vc_selftest_bounded_wait.restype = I32
        lib.vc_frame_cache_create.argtypes = [P, ctypes.c_uint64, U32, U32, ctypes.POINTER(P)]
        lib.vc_frame_cache_view_get.argtypes = [P, ctypes.POINTER(vc_frame_cache_view)]
        lib.vc_frame_mark_cameras.argtypes = [P, P, U32, P]
        lib.vc_frame_update.argtypes = [P, P, U32, U32, P, P]
        lib.vc_frame_stats_get.argtypes = [P, ctypes.POINTER(vc_frame_stats), P]
        for f in ("vc_frame_cache_create", "vc_frame_cache_view_get", "vc_frame_mark_cameras", "vc_frame_update",
                  "vc_frame_stats_get"):
            getattr(lib, f).restype = I32
        for f in ("vc_server_create", "vc_server_add_volume", "vc_submit_bricks", "vc_poll", "vc_wait",
                  "vc_request_coarsest",
                  "vc_request_info_get", "vc_request_release", "vc_server_cache", "vc_server_stats_get",
                  "vc_brick_cache_create", "vc_brick_cache_acquire", "vc_brick_cache_unpin",
                  "vc_brick_cache_invalidate", "vc_brick_cache_stats_get"):
            getattr(lib, f).restype = I32
        lib.vc_free_bytes.argtypes = [P]
        lib.vc_free_bytes.restype = None
        lib.vc_status_string.argtypes = [I32]
        lib.vc_status_string.restype = ctypes.c_char_p
        for f in ("vc_load_compressed", "vc_volume_info_get", "vc_decode_bricks", "vc_decode_bricks_host",
                  "vc_release", "vc_encode_volume", "vc_encode_volume_freq", "vc_concat_volumes_z", "vc_volume_set_schedule", "vc_volume_get_schedule",
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


def vc_load_compressed_split(host_bytes: np.ndarray, device: int = 0, stream: int = 0) -> ctypes.c_void_p:
    b = np.ascontiguousarray(host_bytes, dtype=np.uint8)
    out = ctypes.c_void_p()
    _check(_lib_handle().vc_load_compressed_split(b.ctypes.data, b.size, device, ctypes.c_void_p(stream),
                                                  ctypes.byref(out)), "vc_load_compressed_split")
    return out


def vc_split_counts(host_bytes: np.ndarray, brick_id: int) -> tuple:
    """(S, coarse symbols, coarse palette advances, coarse delta operations) of one brick."""
    b = np.ascontiguousarray(host_bytes, dtype=np.uint8)
    out = np.zeros(4, dtype=np.uint32)
    _check(_lib_handle().vc_split_counts(b.ctypes.data, b.size, brick_id, out.ctypes.data), "vc_split_counts")
    return tuple(int(x) for x in out)


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


def vc_volume_slot_words(vol, lod: int = 0, paletted: bool = False):
    """(words per slot, bits per index, indices per word)."""
    w, b, e = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(_lib_handle().vc_volume_slot_words(vol, lod, int(bool(paletted)), ctypes.byref(w), ctypes.byref(b),
                                              ctypes.byref(e)), "vc_volume_slot_words")
    return w.value, b.value, e.value


def vc_volume_autotune(vol, brick_ids_ptr: int, n: int, cache_slots_ptr: int, cache_ptr: int, lod: int,
                       status_ptr: int, stream: int = 0, reps: int = 3):
    """Returns ((threads, stage_depth, blocks_per_sm, chunk), mode, mean ms) of the fastest schedule."""
    s, m, ms = vc_schedule(), ctypes.c_uint32(), ctypes.c_float()
    _check(_lib_handle().vc_volume_autotune(vol, ctypes.c_void_p(brick_ids_ptr), n, ctypes.c_void_p(cache_slots_ptr),
                                            ctypes.c_void_p(cache_ptr), lod, ctypes.c_void_p(status_ptr),
                                            ctypes.c_void_p(stream), reps, ctypes.byref(s), ctypes.byref(m),
                                            ctypes.byref(ms)), "vc_volume_autotune")
    return (s.threads, s.stage_depth, s.blocks_per_sm, s.chunk), m.value, ms.value


def vc_decode_bricks_noalloc(vol, brick_ids_ptr: int, n: int, cache_slots_ptr: int, cache_ptr: int, lod: int,
                             mode: int, status_ptr: int, stream: int = 0) -> None:
    _check(_lib_handle().vc_decode_bricks_noalloc(vol, ctypes.c_void_p(brick_ids_ptr), n,
                                                  ctypes.c_void_p(cache_slots_ptr), ctypes.c_void_p(cache_ptr), lod,
                                                  mode, ctypes.c_void_p(status_ptr), ctypes.c_void_p(stream)),
           "vc_decode_bricks_noalloc")


def vc_coarsest_labels(vol, brick_ids_ptr: int, n: int, out_ptr: int, status_ptr: int, stream: int = 0) -> None:
    _check(_lib_handle().vc_coarsest_labels(vol, ctypes.c_void_p(brick_ids_ptr), n, ctypes.c_void_p(out_ptr),
                                            ctypes.c_void_p(status_ptr), ctypes.c_void_p(stream)), "vc_coarsest_labels")


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


def _take_bytes(lib, ptr, size) -> np.ndarray:
    out = np.empty(size.value, dtype=np.uint8)
    ctypes.memmove(out.ctypes.data, ptr, size.value)
    lib.vc_free_bytes(ptr)
    return out


def vc_encode_volume(V: np.ndarray, log2b: int, op_mask: int = 0x7F, coder: int = 0, flags: int = 0,
                     threads: int = 0, freq=None) -> np.ndarray:
    """Encode a (z, y, x) uint32 volume with the library's multi-threaded CPU encoder (freq: a fixed
    16-entry rANS frequency table, vc_encode_volume_freq)."""
    V = np.ascontiguousarray(V, dtype=np.uint32)
    dims = (ctypes.c_uint32 * 3)(V.shape[2], V.shape[1], V.shape[0])
    ptr, size = ctypes.c_void_p(), ctypes.c_size_t()
    lib = _lib_handle()
    if freq is None:
        _check(lib.vc_encode_volume(V.ctypes.data, dims, log2b, op_mask, coder, flags, threads, ctypes.byref(ptr),
                                    ctypes.byref(size)), "vc_encode_volume")
    else:
        f = np.ascontiguousarray(freq, dtype=np.uint32)
        _check(lib.vc_encode_volume_freq(V.ctypes.data, dims, log2b, op_mask, coder, flags, threads, f.ctypes.data,
                                         ctypes.byref(ptr), ctypes.byref(size)), "vc_encode_volume_freq")
    return _take_bytes(lib, ptr, size)


def vc_concat_volumes_z(parts) -> np.ndarray:
    """Joins VCZ1 volumes stacked in z (vc_concat_volumes_z)."""
    parts = [np.ascontiguousarray(p, dtype=np.uint8) for p in parts]
    ptrs = (ctypes.c_void_p * len(parts))(*[p.ctypes.data for p in parts])
    sizes = (ctypes.c_size_t * len(parts))(*[p.size for p in parts])
    ptr, size = ctypes.c_void_p(), ctypes.c_size_t()
    lib = _lib_handle()
    _check(lib.vc_concat_volumes_z(ptrs, sizes, len(parts), ctypes.byref(ptr), ctypes.byref(size)),
           "vc_concat_volumes_z")
    return _take_bytes(lib, ptr, size)


# ---- serving

VC_SERVER_GRAPHS = 1


def vc_server_create(cache_bytes: int, device: int = 0, max_batch_items: int = 0, max_inflight: int = 0,
                     min_class: int = 0, max_class: int = 0, flags: int = 0) -> ctypes.c_void_p:
    cfg = vc_server_config(cache_bytes, device, max_batch_items, max_inflight, min_class, max_class, flags)
    out = ctypes.c_void_p()
    _check(_lib_handle().vc_server_create(ctypes.byref(cfg), ctypes.byref(out)), "vc_server_create")
    return out


def vc_server_add_volume(srv, vol) -> int:
    idx = ctypes.c_uint32()
    _check(_lib_handle().vc_server_add_volume(srv, vol, ctypes.byref(idx)), "vc_server_add_volume")
    return idx.value


def vc_submit_bricks(srv, volume_index: int, brick_ids, lods=None) -> int:
    ids = np.ascontiguousarray(brick_ids, dtype=np.uint32)
    lp = None
    if lods is not None:
        lods = np.ascontiguousarray(np.broadcast_to(np.asarray(lods, dtype=np.uint32), ids.shape))
        lp = lods.ctypes.data
    rid = ctypes.c_uint64()
    _check(_lib_handle().vc_submit_bricks(srv, volume_index, ids.ctypes.data if ids.size else None, lp, ids.size,
                                          ctypes.byref(rid)), "vc_submit_bricks")
    return rid.value


def vc_poll(srv, request_id: int, n: int = 0):
    """Returns (state, offsets or None); raises VCError if the request failed."""
    st = ctypes.c_int32()
    offs = np.zeros(n, dtype=np.uint64) if n else None
    _check(_lib_handle().vc_poll(srv, request_id, ctypes.byref(st), offs.ctypes.data if n else None), "vc_poll")
    return st.value, (offs if st.value == VC_REQ_DONE else None)


def vc_wait(srv, request_id: int, timeout_ms: int = 60000) -> int:
    st = ctypes.c_int32()
    _check(_lib_handle().vc_wait(srv, request_id, timeout_ms, ctypes.byref(st)), "vc_wait")
    return st.value


VC_SHADE_LOCAL, VC_SHADE_SHADOW, VC_SHADE_AO, VC_SHADE_PATH = 0, 1, 2, 3


class vc_material(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_float * 3), ("opacity", ctypes.c_float)]


class vc_render_params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("frame", ctypes.c_uint32), ("jitter", ctypes.c_uint32),
                ("max_bounces", ctypes.c_uint32), ("light_dir", ctypes.c_float * 3), ("ambient", ctypes.c_float),
                ("ao_radius", ctypes.c_float), ("sky", ctypes.c_float), ("n_materials", ctypes.c_uint32),
                ("materials", ctypes.c_void_p), ("subsample", ctypes.c_uint32), ("marks", ctypes.c_void_p),
                ("request_depth", ctypes.c_uint32)]


def vc_render(vol, brick_offsets_ptr: int, brick_lods_ptr: int, cache_ptr: int, cam: "vc_camera", materials,
              labels_ptr: int = 0, depth_ptr: int = 0, face_ptr: int = 0, rgb_ptr: int = 0, stream: int = 0,
              mode: int = VC_SHADE_LOCAL, frame: int = 0, jitter: bool = False, max_bounces: int = 8,
              light_dir=(0.3, 0.5, 0.8), ambient: float = 0.25, ao_radius: float = 8.0, sky: float = 1.0,
              subsample: int = 1, marks_ptr: int = 0, request_depth: int = 1) -> None:
    """vc_render: materials is an (n, 4) float array of (r, g, b, opacity) rows (host); marks_ptr:
    device visibility bits (one per brick) or 0."""
    mats = np.ascontiguousarray(materials, dtype=np.float32)
    arr = (vc_material * mats.shape[0])()
    for i, (r, g, b, o) in enumerate(mats):
        arr[i].rgb[:] = [float(r), float(g), float(b)]
        arr[i].opacity = float(o)
    p = vc_render_params(mode, frame, int(bool(jitter)), max_bounces, (ctypes.c_float * 3)(*light_dir), ambient,
                         ao_radius, sky, mats.shape[0], ctypes.cast(arr, ctypes.c_void_p), subsample,
                         ctypes.c_void_p(marks_ptr or None), request_depth)
    _check(_lib_handle().vc_render(vol, ctypes.c_void_p(brick_offsets_ptr), ctypes.c_void_p(brick_lods_ptr),
                                   ctypes.c_void_p(cache_ptr), ctypes.byref(cam), ctypes.byref(p),
                                   ctypes.c_void_p(labels_ptr or None), ctypes.c_void_p(depth_ptr or None),
                                   ctypes.c_void_p(face_ptr or None), ctypes.c_void_p(rgb_ptr or None),
                                   ctypes.c_void_p(stream)), "vc_render")


class vc_post_params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("height", ctypes.c_uint32), ("iterations", ctypes.c_uint32),
                ("subsample", ctypes.c_uint32), ("frame", ctypes.c_uint32), ("reset", ctypes.c_uint32),
                ("cam_pos", ctypes.c_float * 3), ("phi_rho", ctypes.c_float), ("phi_d", ctypes.c_float),
                ("exposure", ctypes.c_float), ("gamma", ctypes.c_float), ("n_materials", ctypes.c_uint32),
                ("materials", ctypes.c_void_p)]


def vc_post_state_bytes(width: int, height: int) -> int:
    return int(_lib_handle().vc_post_state_bytes(width, height))


def vc_postprocess(vol, width: int, height: int, labels_ptr: int, depth_ptr: int, face_ptr: int, rgb_ptr: int,
                   state_ptr: int, rgba_ptr: int, materials, cam_pos, iterations: int = 3, subsample: int = 1,
                   frame: int = 0, reset: bool = False, phi_rho: float = 8.0, phi_d: float = 1.0,
                   exposure: float = 1.0, gamma: float = 2.2, stream: int = 0) -> None:
    mats = np.ascontiguousarray(materials, dtype=np.float32)
    arr = (vc_material * mats.shape[0])()
    for i, (r, g, b, o) in enumerate(mats):
        arr[i].rgb[:] = [float(r), float(g), float(b)]
        arr[i].opacity = float(o)
    p = vc_post_params(width, height, iterations, subsample, frame, int(bool(reset)), (ctypes.c_float * 3)(*cam_pos),
                       phi_rho, phi_d, exposure, gamma, mats.shape[0], ctypes.cast(arr, ctypes.c_void_p))
    _check(_lib_handle().vc_postprocess(vol, ctypes.byref(p), ctypes.c_void_p(labels_ptr), ctypes.c_void_p(depth_ptr),
                                        ctypes.c_void_p(face_ptr), ctypes.c_void_p(rgb_ptr), ctypes.c_void_p(state_ptr),
                                        ctypes.c_void_p(rgba_ptr), ctypes.c_void_p(stream)), "vc_postprocess")


def vc_request_coarsest(srv, request_id: int, labels_ptr: int, status_ptr: int, stream: int = 0) -> None:
    _check(_lib_handle().vc_request_coarsest(srv, ctypes.c_uint64(request_id), ctypes.c_void_p(labels_ptr),
                                             ctypes.c_void_p(status_ptr), ctypes.c_void_p(stream)),
           "vc_request_coarsest")


def vc_request_info_get(srv, request_id: int) -> vc_request_info:
    info = vc_request_info()
    _check(_lib_handle().vc_request_info_get(srv, request_id, ctypes.byref(info)), "vc_request_info_get")
    return info


def vc_request_release(srv, request_id: int) -> None:
    _check(_lib_handle().vc_request_release(srv, request_id), "vc_request_release")


def vc_server_cache(srv):
    p, nb = ctypes.c_void_p(), ctypes.c_uint64()
    _check(_lib_handle().vc_server_cache(srv, ctypes.byref(p), ctypes.byref(nb)), "vc_server_cache")
    return p.value, nb.value


def vc_server_stats_get(srv) -> vc_server_stats:
    st = vc_server_stats()
    _check(_lib_handle().vc_server_stats_get(srv, ctypes.byref(st)), "vc_server_stats_get")
    return st


def vc_camera_bricks(vol, cams, max_lod: int = 31, cap: int | None = None, stream: int = 0):
    """Returns per camera (ids, lods) of the requested bricks (ascending ids)."""
    cams = list(cams)
    arr = (vc_camera * len(cams))(*cams)
    lib = _lib_handle()
    counts = np.zeros(len(cams), dtype=np.uint32)
    if cap is None:
        _check(lib.vc_camera_bricks(vol, ctypes.byref(arr), len(cams), max_lod, 0, counts.ctypes.data, None, None,
                                    ctypes.c_void_p(stream)), "vc_camera_bricks")
        cap = int(counts.max()) if len(cams) else 0
    ids = np.zeros(max(1, len(cams) * cap), dtype=np.uint32)
    lods = np.zeros(max(1, len(cams) * cap), dtype=np.uint32)
    _check(lib.vc_camera_bricks(vol, ctypes.byref(arr), len(cams), max_lod, cap, counts.ctypes.data, ids.ctypes.data,
                                lods.ctypes.data, ctypes.c_void_p(stream)), "vc_camera_bricks")
    return [(ids[i * cap: i * cap + min(int(counts[i]), cap)].copy(), lods[i * cap: i * cap + min(int(counts[i]), cap)].copy())
            for i in range(len(cams))]


def vc_frame_cache_create(vol, cache_bytes: int, max_bricks_per_frame: int = 0,
                          free_stack_entries: int = 0) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    _check(_lib_handle().vc_frame_cache_create(vol, cache_bytes, max_bricks_per_frame, free_stack_entries,
                                               ctypes.byref(out)), "vc_frame_cache_create")
    return out


def vc_frame_cache_view_get(fc) -> vc_frame_cache_view:
    v = vc_frame_cache_view()
    _check(_lib_handle().vc_frame_cache_view_get(fc, ctypes.byref(v)), "vc_frame_cache_view_get")
    return v


def vc_frame_mark_cameras(fc, cams, stream: int = 0) -> None:
    cams = list(cams)
    arr = (vc_camera * max(1, len(cams)))(*cams)
    _check(_lib_handle().vc_frame_mark_cameras(fc, ctypes.byref(arr), len(cams), ctypes.c_void_p(stream)),
           "vc_frame_mark_cameras")


def vc_frame_update(fc, cams, max_lod: int, status_ptr: int, stream: int = 0) -> None:
    cams = list(cams)
    arr = (vc_camera * max(1, len(cams)))(*cams)
    _check(_lib_handle().vc_frame_update(fc, ctypes.byref(arr), len(cams), max_lod, ctypes.c_void_p(status_ptr),
                                         ctypes.c_void_p(stream)), "vc_frame_update")


def vc_frame_stats_get(fc, stream: int = 0) -> vc_frame_stats:
    st = vc_frame_stats()
    _check(_lib_handle().vc_frame_stats_get(fc, ctypes.byref(st), ctypes.c_void_p(stream)), "vc_frame_stats_get")
    return st


def vc_selftest_bounded_wait(budget_us: int, status_ptr: int, stream: int = 0) -> None:
    _check(_lib_handle().vc_selftest_bounded_wait(budget_us, ctypes.c_void_p(status_ptr), ctypes.c_void_p(stream)),
           "vc_selftest_bounded_wait")


def vc_request_bricks(srv, volume_index: int, cams, max_lod: int = 31) -> list:
    cams = list(cams)
    arr = (vc_camera * len(cams))(*cams)
    out = np.zeros(len(cams), dtype=np.uint64)
    _check(_lib_handle().vc_request_bricks(srv, volume_index, ctypes.byref(arr), len(cams), max_lod, out.ctypes.data),
           "vc_request_bricks")
    return [int(x) for x in out]


def vc_brick_cache_create(nbytes: int, min_class: int, max_class: int) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    _check(_lib_handle().vc_brick_cache_create(nbytes, min_class, max_class, ctypes.byref(out)),
           "vc_brick_cache_create")
    return out


def vc_brick_cache_acquire(cache, keys, classes):
    """Returns (entries, offsets, hits) or None if the keys do not fit (VC_ERR_BUSY)."""
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    c = np.ascontiguousarray(np.broadcast_to(np.asarray(classes, dtype=np.uint32), k.shape))
    n = k.size
    ent = np.zeros(n, dtype=np.uint32)
    off = np.zeros(n, dtype=np.uint64)
    hit = np.zeros(n, dtype=np.uint8)
    rc = _lib_handle().vc_brick_cache_acquire(cache, k.ctypes.data, c.ctypes.data, n, ent.ctypes.data,
                                              off.ctypes.data, hit.ctypes.data)
    if rc == VC_ERR_BUSY:
        return None
    _check(rc, "vc_brick_cache_acquire")
    return ent, off, hit.astype(bool)


def vc_brick_cache_unpin(cache, entries) -> None:
    e = np.ascontiguousarray(entries, dtype=np.uint32)
    _check(_lib_handle().vc_brick_cache_unpin(cache, e.ctypes.data, e.size), "vc_brick_cache_unpin")


def vc_brick_cache_invalidate(cache, entry: int) -> None:
    _check(_lib_handle().vc_brick_cache_invalidate(cache, entry), "vc_brick_cache_invalidate")


def vc_brick_cache_stats_get(cache) -> vc_brick_cache_stats:
    st = vc_brick_cache_stats()
    _check(_lib_handle().vc_brick_cache_stats_get(cache, ctypes.byref(st)), "vc_brick_cache_stats_get")
    return st


# ------------------------------------------------------------------ convenience wrapper (torch)

class Volume:
    """A compressed volume resident on a CUDA device."""

    def __init__(self, encoded: np.ndarray, device: int = 0, stream=None, split: bool = False):
        import torch
        self.device = device
        s = stream if stream is not None else torch.cuda.current_stream(device)
        load = vc_load_compressed_split if split else vc_load_compressed
        self.handle = load(encoded, device, s.cuda_stream)
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
