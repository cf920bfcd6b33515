#!/usr/bin/env python3
"""Benchmark: brick-parallel decode of a CSGV-compressed 512^3 segmentation volume (32^3 bricks).

One step = decode every brick of the volume (4096 bricks, 134M voxels) from the device-resident
encoding into a 512 MiB uint32 brick cache, with the batched persistent decoder. Prints one JSON
line (rank 0). `--impl reference` times the CPU oracle on the host cores instead (bounded sample).

Timing: W untimed warm-up steps; K timed steps, each a CUDA-event pair on the launching stream
around the decode; the L2 is flushed (256 MiB write) before every step, outside the event pair;
barrier + synchronize on both sides of the timed region; max over ranks. Clocks are sampled with
nvidia-smi while the timed steps run.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

B_LOG2 = 5
CODER_RANS = 1
METRIC = "decoded Gvoxel/s"
UNIT = "Gvoxel/s"
def kernel_name(mode: str, threads: int, log2b: int = B_LOG2) -> str:
    if log2b >= 6:  # 64^3 bricks: one persistent kernel serves every schedule
        return f"decode_scratch_kernel<L={log2b},u8 grid,rANS,{threads} threads>"
    return f"decode_{mode}_kernel<L={log2b},u8 grid,rANS,{threads} threads>"


def workload_name(log2b: int = B_LOG2, runs: int = 1) -> str:
    b = 1 << log2b
    n = (512 // b) ** 3
    return (f"512^3 uint32 Voronoi volume (~20k cells, 10% background), {b}^3 bricks ({n}), rANS"
            + (f" in {runs} runs per record" if runs > 1 else "") + ", all operations")


WORKLOAD = workload_name()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x: float, device) -> float:
    """The largest x over all ranks (the job is as slow as its slowest rank); x itself at N = 1."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank_step: int, steps: int, slowest_s: float) -> float:
    """Whole-job throughput (weak scaling: every rank decodes its own full workload): units of all
    ranks over the slowest rank's time, in G units per second."""
    return world * units_per_rank_step * steps / slowest_s / 1e9


def make_workload(encoder: str = "library", log2b: int = B_LOG2, runs: int = 1):
    """The 512^3 volume and its encoding (32^3 bricks unless log2b says otherwise; `runs` rANS
    runs per record): by the library's encoder, or (reference arm) by the oracle's, whose bytes are
    identical."""
    import synth
    spec = synth.c2()
    t = time.time()
    V = synth.fill(spec)
    t_gen = time.time() - t
    t = time.time()
    flags = {1: 0, 2: 4, 4: 8, 8: 12}[runs]  # header flag bits 2..3: log2 of the runs
    if encoder == "oracle":
        import oracle
        oracle.build()
        enc = oracle.encode_volume(V, log2b, op_mask=0x7F, coder=CODER_RANS, flags=flags)
    else:
        import paper_2609_36898_gb300 as vc
        enc = vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=CODER_RANS, flags=flags)
    t_enc = time.time() - t
    return spec, V, enc, t_gen, t_enc


def full_table(freq) -> np.ndarray:
    """A rANS table with every symbol at least 1 (taken from the largest entry), summing to 4096, so
    that it codes any slab of a volume."""
    f = np.asarray(freq, dtype=np.int64).copy()
    short = int((f == 0).sum())
    f[f == 0] = 1
    f[int(np.argmax(f))] -= short
    return f.astype(np.uint32)


def generate_encode(spec, log2b: int, coder: int = CODER_RANS, max_slab_voxels: int = 1 << 28, flags: int = 0):
    """VCZ1 bytes of a synthetic volume: generated on the GPU (synth_fill_gpu, the CPU generator's
    voxels) in z slabs of whole bricks, each slab copied to pinned host memory and encoded on the
    host cores by the library's encoder while the next slab is generated; all slabs share the rANS
    table of the first (every symbol kept >= 1) and are joined with vc_concat_volumes_z. Returns
    (bytes, seconds)."""
    import torch
    import synth
    import paper_2609_36898_gb300 as vc
    t0 = time.time()
    nx, ny, nz = (int(d) for d in spec.dims)
    b = 1 << log2b
    slab = max(b, min(-(-nz // b) * b, (max_slab_voxels // (nx * ny)) // b * b))
    z0s = list(range(0, nz, slab))
    dev = torch.empty((slab, ny, nx), dtype=torch.int32, device="cuda")
    host = [torch.empty((slab, ny, nx), dtype=torch.int32, pin_memory=True) for _ in range(min(2, len(z0s)))]
    stream = torch.cuda.current_stream()

    def start(k):
        t = min(slab, nz - z0s[k])
        synth.fill_gpu(spec, (0, 0, z0s[k]), (nx, ny, t), dev.data_ptr(), stream.cuda_stream)
        host[k % len(host)][:t].copy_(dev[:t], non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(stream)
        return ev, t

    parts, table = [], None
    pending = start(0)
    for k in range(len(z0s)):
        ev, t = pending
        ev.synchronize()
        if k + 1 < len(z0s):
            pending = start(k + 1)  # the GPU generates the next slab while this one is encoded
        V = host[k % len(host)][:t].numpy().view(np.uint32)
        if len(z0s) == 1:
            parts.append(vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=coder, flags=flags))
            break
        if table is None and coder == CODER_RANS:
            first = vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=coder, flags=flags)
            h = np.frombuffer(first[:128].tobytes(), dtype="<u4")
            table = full_table(h[12:28])
        parts.append(vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=coder, flags=flags, freq=table))
    torch.cuda.synchronize()
    enc = parts[0] if len(parts) == 1 else vc.vc_concat_volumes_z(parts)
    return enc, time.time() - t0


def verify_all(cache, V: np.ndarray, e: int, what: str) -> None:
    """Every decoded brick (slot i = brick i) equals the input volume's voxels."""
    nz, ny, nx = (s // e for s in V.shape)
    want = V.reshape(nz, e, ny, e, nx, e).transpose(0, 2, 4, 1, 3, 5).reshape(-1)
    got = cache[: want.size].cpu().numpy().view(np.uint32)
    if not np.array_equal(got, want):
        bad = np.flatnonzero((got != want).reshape(-1, e ** 3).any(axis=1))
        raise AssertionError(f"{what}: {bad.size} decoded bricks differ from the input volume, first {bad[:8].tolist()}")


def algorithmic_bytes(enc: np.ndarray, n_bricks: int, edge: int) -> int:
    """Per launch: Brick Starts entry + record bytes + queue item (id + slot) + decoded labels."""
    h = np.frombuffer(enc[:128].tobytes(), dtype="<u4")
    records_words = int(h[28])
    return 4 * n_bricks + 4 * records_words + 8 * n_bricks + 4 * edge ** 3 * n_bricks


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"vc_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):  # noqa: D105
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(kernel_src_hash: str, mode: str, threads: int, log2b: int = B_LOG2, runs: int = 1):
    """DRAM bytes per launch from the committed ncu summary of this schedule's kernel, if taken on
    the current kernel source and the same workload."""
    tag = f"b{1 << log2b}" + (f"_runs{runs}" if runs > 1 else "")
    p = os.path.join(ROOT, "profiles", f"decode_{mode if log2b < 6 else 'scratch'}_512cube_{tag}_rans.json")
    try:
        d = json.load(open(p))
        if d.get("kernel_source_sha256") == kernel_src_hash and d.get("kernel") == kernel_name(mode, threads, log2b):
            return d.get("dram_bytes_per_launch_full_workload")
    except Exception:
        pass
    return None


KERNEL_SOURCES = ("decode_kernels.cuh", "decode_nt.cu")


def kernel_hash():
    """Identifies the reconstruction kernel's source (traffic figures are only valid for it)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2609_36898_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def host_cpu():
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"host_cores": os.cpu_count(), "host_cpu": model}


def oracle_rate(enc: np.ndarray, seconds: float, max_bricks: int, first: int = 0):
    """Single-threaded oracle decode on a bounded sample of the workload's bricks (at least one
    brick, then until `seconds` have passed or `max_bricks` were decoded), cycling over the volume."""
    import oracle
    h = oracle.header(enc)
    n_bricks, log2b = h["n_bricks"], h["log2b"]
    n_b = 0
    t0 = time.perf_counter()
    while n_b < 1 or (n_b < max_bricks and time.perf_counter() - t0 < seconds):
        oracle.decode_brick(enc, (first + n_b) % n_bricks, 0)
        n_b += 1
    dt = time.perf_counter() - t0
    vox = n_b * (1 << (3 * log2b))
    return vox / dt / 1e9, n_b, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    spec, V, enc, _, _ = make_workload(encoder="oracle", log2b=args.log2b, runs=args.runs)
    import oracle
    total_vox, total_t, nb = 0, 0.0, 0
    for _ in range(args.warmup):
        oracle.decode_brick(enc, 0, 0)
    per_step = 20.0 / max(1, args.steps)  # the whole timed run takes about 20 s of one core
    for k in range(args.steps):
        r, n_b, dt = oracle_rate(enc, per_step, 4096, first=nb)
        total_vox += n_b * (1 << (3 * args.log2b))
        total_t += dt
        nb += n_b
    value = total_vox / total_t / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total_t / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": workload_name(args.log2b, args.runs),
                       "bricks_per_step": (512 >> args.log2b) ** 3, "sample": "bounded"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{nb} brick decodes of the 512^3 volume in {total_t:.1f} s, single thread",
                             **host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def orbit_camera(vc, i: int, frame: int, dims, width: int, height: int, fov: float = 0.8):
    """Camera i of the serving workload at a frame: an orbit of radius 1.2-3 volume diagonals
    around the volume centre, on a seeded random axis and phase, 1 degree per frame."""
    import math
    rng = np.random.default_rng(1000 + i)
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    a = np.cross(axis, rng.normal(size=3))
    a /= np.linalg.norm(a)
    b = np.cross(axis, a)
    radius = float(np.linalg.norm(dims)) * rng.uniform(1.2, 3.0)
    phase = rng.uniform(0, 2 * math.pi) + math.radians(frame)
    centre = np.asarray(dims, np.float64) / 2
    pos = centre + radius * (math.cos(phase) * a + math.sin(phase) * b)
    return vc.make_camera(pos, centre - pos, axis, fov, width, height)


def frame_cache_leg(vc, vol, dims, ncam: int, W: int, H: int, max_lod: int, frames: int, stream) -> dict:
    """The same cameras through the device-side cache stages (vc_frame_*: mark, then request,
    provision, assign and decode on the GPU with no host round trip), 2 GiB of labels. (a) all
    cameras' brick rays mark, one update per frame for all of them; (b) one camera at W x H
    rendered with shadow rays, its rays marking the bricks for the next frame's update. CUDA
    events around each stage; the frame statistics are read after the frame."""
    import torch
    pct = lambda a, q: float(np.percentile(np.asarray(a), q)) if len(a) else None  # noqa: E731
    status = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
    out = {"cache_bytes": 2 << 30}
    fc = vc.vc_frame_cache_create(vol, 2 << 30)
    try:
        view = vc.vc_frame_cache_view_get(fc)
        out["max_bricks_per_frame"] = int(view.max_bricks_per_frame)
        mark_ms, upd_ms, dec, vox, rows = [], [], [], [], []
        prev = vc.vc_frame_stats_get(fc, stream.cuda_stream)
        for f in range(frames):
            cams = [orbit_camera(vc, i, f, dims, W, H) for i in range(ncam)]
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            vc.vc_frame_mark_cameras(fc, cams, stream.cuda_stream)
            ev[1].record(stream)
            vc.vc_frame_update(fc, cams, max_lod, status.data_ptr(), stream.cuda_stream)
            ev[2].record(stream)
            st = vc.vc_frame_stats_get(fc, stream.cuda_stream)
            mark_ms.append(ev[0].elapsed_time(ev[1]))
            upd_ms.append(ev[1].elapsed_time(ev[2]))
            dec.append(int(st.last_decoded))
            vox.append(int(st.voxels_decoded - prev.voxels_decoded))
            rows.append({"mark_ms": mark_ms[-1], "update_ms": upd_ms[-1], "resident": int(st.last_resident),
                         "requested": int(st.last_requested), "decoded": int(st.last_decoded),
                         "freed": int(st.last_freed), "reset": bool(st.resets > prev.resets)})
            prev = st
        if int(status[0]) != 0:
            raise RuntimeError(f"frame cache decode status {status.tolist()}")
        out["brick_rays"] = {
            "cameras": ncam, "frames": frames, "update_ms_p50": pct(upd_ms, 50), "update_ms_p99": pct(upd_ms, 99),
            "mark_ms_p50": pct(mark_ms, 50),
            "decoded_gvoxel_s": sum(vox) / (sum(upd_ms) / 1000.0) / 1e9 if sum(upd_ms) > 0 else None,
            "resets": int(prev.resets), "dead_words": int(prev.dead_words), "top_words": int(prev.top_words),
            "per_frame": rows,
            "note": "update = request + provision + assign + decode of all cameras' bricks (device counts, no host "
                    "sync); latency of a frame's bricks = its update time"}
    finally:
        vc.vc_release(fc)
    # (b) the renderer's rays mark: one camera, the paper's per-frame pipeline
    fc = vc.vc_frame_cache_create(vol, 2 << 30)
    try:
        view = vc.vc_frame_cache_view_get(fc)
        lab = torch.empty(W * H, dtype=torch.int32, device="cuda")
        rows = []
        prev = vc.vc_frame_stats_get(fc, stream.cuda_stream)
        for f in range(frames):
            cam = orbit_camera(vc, 0, f, dims, W, H)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            vc.vc_frame_update(fc, [cam], max_lod, status.data_ptr(), stream.cuda_stream)
            ev[1].record(stream)
            vc.vc_render(vol, view.offsets, view.lods, view.cache, cam, RENDER_MATERIALS, lab.data_ptr(),
                         stream=stream.cuda_stream, mode=vc.VC_SHADE_SHADOW, frame=f, marks_ptr=view.marks,
                         request_depth=1)
            ev[2].record(stream)
            st = vc.vc_frame_stats_get(fc, stream.cuda_stream)
            rows.append({"update_ms": ev[0].elapsed_time(ev[1]), "render_ms": ev[1].elapsed_time(ev[2]),
                         "resident": int(st.last_resident), "decoded": int(st.last_decoded),
                         "voxels": int(st.voxels_decoded - prev.voxels_decoded)})
            prev = st
        if int(status[0]) != 0:
            raise RuntimeError(f"frame cache decode status {status.tolist()}")
        upd = [r["update_ms"] for r in rows[1:]]
        out["render_rays"] = {
            "image": f"{W}x{H}", "mode": "shadow rays (request depth 1)", "frames": frames,
            "update_ms_p50": pct(upd, 50), "update_ms_p99": pct(upd, 99),
            "render_ms_p50": pct([r["render_ms"] for r in rows[1:]], 50), "per_frame": rows,
            "note": "frame f: update from the marks of frame f-1's render, then render (undecoded bricks show their "
                    "coarsest label); frame 0 renders an empty cache"}
    finally:
        vc.vc_release(fc)
    return out


def serving_leg(args, local: int):
    """Camera-driven serving on the 4096^3 hash-grid Voronoi volume (one seed per 16^3 grid cell,
    ~16M cells; --serve-size n runs the same recipe on n^3 with the image scaled by n/4096): 64
    orbiting cameras at 1920x1080 request their visible bricks every frame (request stage on the
    GPU), the server admits, batches and decodes them into a 2 GiB cache, and each request is
    released as soon as it is complete (the client has used its bricks); versus plain per-request
    decoding (one launch per brick, no cache)."""
    import torch
    import synth
    import paper_2609_36898_gb300 as vc
    n = args.serve_size
    spec = synth.c4() if n == 4096 else synth.c4_scaled(n)
    enc, prep = generate_encode(spec, B_LOG2)
    stream = torch.cuda.current_stream(local)
    vol = vc.vc_load_compressed(enc, local, stream.cuda_stream)
    enc_bytes = int(enc.size)
    del enc
    srv = vc.vc_server_create(2 << 30, local)
    vi = vc.vc_server_add_volume(srv, vol)
    dims = (n, n, n)
    # 1920 x 1080 on the 4096^3 volume; scaled with the volume edge on smaller stand-ins so that a
    # voxel covers the same share of the image (the level-of-detail rule sees the same ratios)
    ncam, max_lod = args.serve_cameras, 3
    W, H = max(16, 1920 * n // 4096), max(9, 1080 * n // 4096)
    lat, rstage, frame_ms, per_cam = [], [], [], []
    delivered = 0
    t_all = time.perf_counter()
    for f in range(args.serve_frames):
        cams = [orbit_camera(vc, i, f, dims, W, H) for i in range(ncam)]
        t0 = time.perf_counter()
        rids = vc.vc_request_bricks(srv, vi, cams, max_lod)
        t1 = time.perf_counter()
        for r in rids:
            if vc.vc_wait(srv, r, 300000) != vc.VC_REQ_DONE:
                raise RuntimeError("serving request failed")
            info = vc.vc_request_info_get(srv, r)
            lat.append((info.t_done_ns - info.t_submit_ns) / 1e6)
            delivered += info.bytes // 4
            per_cam.append(int(info.n_bricks))
            vc.vc_request_release(srv, r)
        t2 = time.perf_counter()
        rstage.append(1000 * (t1 - t0))
        frame_ms.append(1000 * (t2 - t0))
    wall = time.perf_counter() - t_all
    st = vc.vc_server_stats_get(srv)
    vox = st.voxels_decoded
    vc.vc_release(srv)
    cams0 = [orbit_camera(vc, i, 0, dims, W, H) for i in range(ncam)]
    vc.vc_camera_bricks(vol, cams0[:1], max_lod)  # warm-up
    t0 = time.perf_counter()
    lists = vc.vc_camera_bricks(vol, cams0, max_lod, cap=int(vc.vc_volume_info_get(vol).n_bricks))
    camera_stage_ms = 1000 * (time.perf_counter() - t0)
    edge = 1 << B_LOG2

    # plain: the first cameras' requests of frame 0, one launch per brick, one request after the
    # other (bounded: a full frame would take minutes)
    lists = lists[:args.serve_plain_cameras]
    e = [torch.cuda.Event(enable_timing=True) for _ in range(len(lists) + 1)]
    status = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
    maxn = max(len(i) for i, _ in lists)
    cache = torch.empty(maxn * edge ** 3, dtype=torch.int32, device="cuda")
    slots = torch.arange(maxn, dtype=torch.int32, device="cuda")
    plain_vox = 0
    torch.cuda.synchronize()
    e[0].record(stream)
    for c, (ids, lods) in enumerate(lists):
        for lod in np.unique(lods):
            sel = ids[lods == lod]
            ids_t = torch.from_numpy(sel.view(np.int32)).cuda()
            vc.vc_decode_bricks(vol, ids_t.data_ptr(), sel.size, slots.data_ptr(), cache.data_ptr(), int(lod),
                                vc.VC_MODE_PLAIN, status.data_ptr(), stream.cuda_stream)
            plain_vox += sel.size * (edge >> int(lod)) ** 3
        e[c + 1].record(stream)
    torch.cuda.synchronize()
    plain_lat = [e[0].elapsed_time(e[c + 1]) for c in range(len(lists))]
    plain_s = plain_lat[-1] / 1000.0
    gpu_frames = frame_cache_leg(vc, vol, dims, ncam, W, H, max_lod, args.serve_frames + 4, stream)
    vc.vc_release(vol)
    del cache
    pct = lambda a, q: float(np.percentile(np.asarray(a), q)) if len(a) else None  # noqa: E731
    return {
        "gpu_frames": gpu_frames,
        "workload": f"{n}^3 Voronoi (hash grid, one seed per 16^3 cell, 10% background), 32^3 bricks, rANS "
                    f"({8.0 * enc_bytes / n ** 3:.2f} bit/voxel, resident on the device); {ncam} orbiting cameras at "
                    f"{W}x{H}, {args.serve_frames} frames, 2 GiB cache, lod <= {max_lod}; each request released when "
                    "complete",
        "served": {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "requests": len(lat),
                   "gvoxel_s": delivered / wall / 1e9, "decoded_gvoxel_s": vox / wall / 1e9,
                   "request_stage_ms_median": pct(rstage, 50),
                   "camera_stage_alone_ms": camera_stage_ms,
                   "bricks_requested_per_camera": float(np.mean(per_cam)) if per_cam else None,
                   "frame_ms_median": pct(frame_ms, 50), "bricks_decoded": int(st.bricks_decoded),
                   "bricks_hit": int(st.bricks_hit), "batches": int(st.batches), "evictions": int(st.evictions)},
        "plain": {"p50_ms": pct(plain_lat, 50), "p99_ms": pct(plain_lat, 99), "requests": len(lists),
                  "gvoxel_s": plain_vox / plain_s / 1e9 if plain_s > 0 else None,
                  "note": f"frame 0's requests of the first {len(lists)} cameras, decoded one after the other with one "
                          "launch per brick, no cache"},
        "metrics": "gvoxel_s = voxels delivered to requests (hits and decodes) per second of the frame loop; "
                   "decoded_gvoxel_s = voxels the server decoded per second; latency = submit to resident",
        "status": int(status[0]),
        "prep_s": prep,
    }


def mixed_serving_leg(args, local: int):
    """The mixed serving workload: 8 resident volumes of the 8-volume recipe at their stated sizes
    (256^3 .. 2048^3, cell diameters 8..64 voxels, 0..40 % background, bricks of 16^3 / 32^3 / 64^3),
    Poisson-arriving requests of log-uniform size (1..4096 bricks, at most half the cache) of a
    random volume, a 4 GiB cache (the volumes decode to ~78 GB, so most bricks are decoded),
    admission by free cache memory; arrival rates of 50, 80 and 95 % of the server's measured
    capacity (the same requests back to back); latency submit -> resident. Versus plain
    per-request decoding of the 80 % arrivals: one launch per brick, one request after another,
    no cache."""
    import queue
    import threading
    import torch
    import synth
    import paper_2609_36898_gb300 as vc
    rng = np.random.default_rng(77)
    cache_bytes = 4 << 30
    vols, edges, names = [], [], []
    prep = 0.0
    stream = torch.cuda.current_stream(local)
    enc_bytes = 0
    for sp in synth.c5():
        b = sp.brick
        # 64^3 bricks: 4 rANS runs per record, so that 4 warps share each brick's symbol chain
        enc, t = generate_encode(sp, b.bit_length() - 1, flags=vc.VC_FLAG_RUNS(4) if b == 64 else 0)
        prep += t
        enc_bytes += int(enc.size)
        vols.append(vc.vc_load_compressed(enc, local, stream.cuda_stream))
        edges.append(b)
        names.append(f"{sp.dims[0]}^3/b{b}")
        del enc
    nreq = args.mixed_requests
    reqs = []
    for _ in range(nreq):
        vi = int(rng.integers(len(vols)))
        nb = int(vc.vc_volume_info_get(vols[vi]).n_bricks)
        cap = (cache_bytes // 2) // (4 * edges[vi] ** 3)
        size = int(min(nb, cap, max(1, round(float(np.exp(rng.uniform(0, np.log(4096))))))))
        reqs.append((vi, rng.choice(nb, size=size, replace=False).astype(np.uint32)))
    vox_of = [len(ids) * edges[vi] ** 3 for vi, ids in reqs]

    def new_server():
        srv = vc.vc_server_create(cache_bytes, local, max_batch_items=16384, flags=vc.VC_SERVER_GRAPHS)
        for h in vols:
            vc.vc_server_add_volume(srv, h)
        return srv

    # capacity: the same requests back to back with no pacing (after a warm-up pass of the graphs)
    srv = new_server()
    for vi, ids in reqs[:20]:
        r = vc.vc_submit_bricks(srv, vi, ids)
        vc.vc_wait(srv, r, 300000)
        vc.vc_request_release(srv, r)
    vc.vc_release(srv)
    srv = new_server()
    t0 = time.perf_counter()
    rids = [vc.vc_submit_bricks(srv, vi, ids) for vi, ids in reqs]
    for r in rids:
        vc.vc_wait(srv, r, 300000)
        vc.vc_request_release(srv, r)
    cap_s = time.perf_counter() - t0
    cap_rate = nreq / cap_s
    vc.vc_release(srv)

    def run_at(frac):
        srv = new_server()
        rate = frac * cap_rate
        arrivals = np.cumsum(np.random.default_rng(78).exponential(1.0 / rate, size=nreq))
        lat = []
        q = queue.Queue()

        def waiter():  # completes (and releases) requests in arrival order while more arrive
            for _ in range(nreq):
                r = q.get()
                vc.vc_wait(srv, r, 300000)
                info = vc.vc_request_info_get(srv, r)
                lat.append((info.t_done_ns - info.t_submit_ns) / 1e6)
                vc.vc_request_release(srv, r)

        th = threading.Thread(target=waiter)
        th.start()
        t0 = time.perf_counter()
        for (vi, ids), at in zip(reqs, arrivals):
            while time.perf_counter() - t0 < at:
                pass
            q.put(vc.vc_submit_bricks(srv, vi, ids))
        th.join()
        wall = time.perf_counter() - t0
        st = vc.vc_server_stats_get(srv)
        vc.vc_release(srv)
        pct = lambda a, p: float(np.percentile(np.asarray(a), p))  # noqa: E731
        return {"load": frac, "requests_per_s": rate, "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                "decoded_gvoxel_s": st.voxels_decoded / wall / 1e9, "delivered_gvoxel_s": sum(vox_of) / wall / 1e9,
                "bricks_hit": int(st.bricks_hit), "bricks_decoded": int(st.bricks_decoded),
                "evictions": int(st.evictions), "graph_launches": int(st.graph_launches)}, arrivals

    served = []
    arrivals80 = None
    for frac in (0.5, 0.8, 0.95):
        res, arr = run_at(frac)
        served.append(res)
        if frac == 0.8:
            arrivals80 = arr

    # plain: the first requests of the 80 % arrivals, each decoded on arrival (or when the previous
    # one ends) with one launch per brick
    status = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
    n_plain = min(nreq, args.mixed_plain_requests)
    maxn = max(len(ids) for _, ids in reqs[:n_plain])
    cache = torch.empty(max(len(ids) * edges[vi] ** 3 for vi, ids in reqs[:n_plain]), dtype=torch.int32, device="cuda")
    slots = torch.arange(maxn, dtype=torch.int32, device="cuda")
    plain_lat = []
    t0 = time.perf_counter()
    for (vi, ids), at in zip(reqs[:n_plain], arrivals80[:n_plain]):
        while time.perf_counter() - t0 < at:
            pass
        ids_t = torch.from_numpy(ids.view(np.int32)).cuda()
        vc.vc_decode_bricks(vols[vi], ids_t.data_ptr(), ids.size, slots.data_ptr(), cache.data_ptr(), 0,
                            vc.VC_MODE_PLAIN, status.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        plain_lat.append(1000 * (time.perf_counter() - t0 - at))
    del cache
    for h in vols:
        vc.vc_release(h)
    pct = lambda a, q: float(np.percentile(np.asarray(a), q)) if len(a) else None  # noqa: E731
    return {
        "workload": "8 volumes of the mixed recipe at their stated sizes (" + ", ".join(names) + f"; {enc_bytes / 2**30:.2f} "
                    f"GiB encoded, resident), rANS (64^3 bricks in 4 runs per record); {nreq} Poisson requests of "
                    "1..4096 bricks (at most half the cache) "
                    "at 50 / 80 / 95 % of the measured capacity; 4 GiB cache; CUDA-graph batches",
        "capacity": {"requests_per_s": cap_rate, "gvoxel_s": sum(vox_of) / cap_s / 1e9},
        "served": served,
        "plain": {"p50_ms": pct(plain_lat, 50), "p99_ms": pct(plain_lat, 99), "requests": len(plain_lat),
                  "note": "the first requests of the 80 % arrival sequence, decoded one after the other with one "
                          "launch per brick, no cache; latency from arrival to completion"},
        "status": int(status[0]),
        "prep_s": prep,
    }


def subsets_leg(args, local: int):
    """The uneven power-diagram workload (2048 x 2048 x 1024, ~2M cells, log-normal radii, 30 %
    forced-uniform bricks, 131,072 bricks of 32^3): random subsets of 100,000 distinct bricks
    (seeds 30 ..), each decoded in one call with the autotuned schedule into a 13.1 GB slot array;
    inputs resident, CUDA events around each call (--subsets K of them)."""
    import torch
    import synth
    import paper_2609_36898_gb300 as vc
    spec = synth.c3()
    enc, prep = generate_encode(spec, B_LOG2)
    vol = vc.Volume(enc, device=local)
    n_all, e = vol.n_bricks, vol.b
    stream = torch.cuda.current_stream(local)
    n = 100_000
    slots = torch.arange(n, dtype=torch.int32, device="cuda")
    cache = torch.empty(n * e ** 3, dtype=torch.int32, device="cuda")
    status = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
    first = torch.from_numpy(np.random.default_rng(30).choice(n_all, size=n, replace=False).astype(np.int32)).cuda()
    sched, mode, _ = vc.vc_volume_autotune(vol.handle, first.data_ptr(), 10_000, slots.data_ptr(), cache.data_ptr(), 0,
                                           status.data_ptr(), stream.cuda_stream, reps=1)
    status.zero_()
    rates, recs = [], []
    rb = np.frombuffer(enc[128:128 + 4 * (n_all + 1)].tobytes(), dtype="<u4").astype(np.int64)
    for k in range(args.subsets):
        sub = np.random.default_rng(30 + k).choice(n_all, size=n, replace=False)
        ids = torch.from_numpy(sub.astype(np.int32)).cuda()
        vc.vc_decode_bricks(vol.handle, ids.data_ptr(), n, slots.data_ptr(), cache.data_ptr(), 0, mode,
                            status.data_ptr(), stream.cuda_stream)  # warm-up of this subset's shapes
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        vc.vc_decode_bricks(vol.handle, ids.data_ptr(), n, slots.data_ptr(), cache.data_ptr(), 0, mode,
                            status.data_ptr(), stream.cuda_stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        rates.append(n * e ** 3 / (ms / 1000.0) / 1e9)
        recs.append(int((rb[sub + 1] - rb[sub]).sum()) * 4)
    if int(status[0]) != 0:
        raise RuntimeError(f"subset decode status {status.tolist()}")
    vol.release()
    algo = [4 * n + r + 8 * n + 4 * e ** 3 * n for r in recs]
    return {"workload": "2048x2048x1024 power diagram (~2M cells, log-normal radii sigma 0.8, 30 % forced-uniform "
                        "bricks), 32^3 bricks, rANS; subsets of 100,000 random distinct bricks (seeds 30 ..)",
            "schedule": {"mode": next(m for m in ("grid", "batched") if vc.MODES[m] == mode),
                         "threads_per_brick": sched[0], "stage_depth": sched[1], "blocks_per_sm": sched[2]},
            "subsets": len(rates), "gvoxel_s": rates, "gvoxel_s_mean": float(np.mean(rates)),
            "algorithmic_gbs_mean": float(np.mean([a * r / (n * e ** 3) for a, r in zip(algo, rates)])),
            "bits_per_voxel": 8.0 * enc.size / (2048 * 2048 * 1024), "prep_s": prep}


ABLATION_PREFIXES = [("P", 0x10, 0), ("P+parent", 0x11, 0), ("P+parent+x", 0x13, 0), ("P+parent+x+y", 0x17, 0),
                     ("P+parent+x+y+z", 0x1F, 0), ("P+parent+x+y+z+last", 0x3F, 0),
                     ("P+parent+x+y+z+last+delta(limited, 1<d<=16)", 0x7F, 2), ("P+parent+x+y+z+last+delta", 0x7F, 0)]


def ablation_leg(V: np.ndarray) -> list:
    """Compression of the 512^3 volume with the palette operation plus each prefix of the ordered
    operation set {parent, x, y, z, last, delta} (the delta in its limited and unlimited form),
    stored plain (4 bits per symbol) and rANS coded: the synthetic counterpart of the paper's
    operation ablation (Supplementary Fig. "CSGV ablation"). Library encoder on the host cores."""
    import paper_2609_36898_gb300 as vc
    rows = []
    for name, mask, flags in ABLATION_PREFIXES:
        for coder in (0, 1):
            enc = vc.vc_encode_volume(V, B_LOG2, op_mask=mask, coder=coder, flags=flags)
            h = np.frombuffer(enc[:128].tobytes(), dtype="<u4")
            n = int(h[9])
            starts = np.frombuffer(enc[128:128 + 4 * (n + 1)].tobytes(), dtype="<u4").astype(np.int64)
            rec0 = (128 + 4 * (n + 1) + 15) & ~15
            words = np.frombuffer(enc[rec0:].tobytes(), dtype="<u4")
            n_pal = words[starts[:-1]]
            rows.append({"operations": name, "coder": "rANS" if coder else "plain",
                         "bits_per_voxel": 8.0 * enc.size / V.size, "percent_of_raw": 100.0 * enc.size / (4.0 * V.size),
                         "palette_mean": float(n_pal.mean()), "palette_max": int(n_pal.max())})
    return rows


RENDER_MATERIALS = np.array([[0.85, 0.35, 0.25, 1.0], [0.25, 0.7, 0.4, 1.0], [0.3, 0.45, 0.9, 1.0],
                             [0.8, 0.75, 0.2, 1.0], [0.6, 0.3, 0.75, 0.5], [0.2, 0.8, 0.85, 1.0]], np.float32)


def render_leg(vol, cache, n: int, e: int, stream, local: int) -> dict:
    """1920 x 1080 frames of the 512^3 volume from its decoded bricks (every brick at the finest
    level, brick i in slot i of the benchmark's cache): local shading and path tracing (up to 8
    bounces), one sample per pixel, CUDA events around each frame."""
    import torch
    import paper_2609_36898_gb300 as vc
    offsets = torch.arange(n, dtype=torch.int64, device="cuda") * (e ** 3)
    lods = torch.zeros(n, dtype=torch.uint8, device="cuda")
    W, H = 1920, 1080
    cam = vc.make_camera((-350.0, 700.0, -520.0), (606.0, -444.0, 776.0), (0.0, 1.0, 0.0), 0.75, W, H)
    lab = torch.empty(W * H, dtype=torch.int32, device="cuda")
    rgb = torch.empty(3 * W * H, dtype=torch.float32, device="cuda")
    out = {"image": f"{W}x{H}", "volume": "512^3, every brick decoded at the finest level", "modes": {}}
    for name, mode in (("local", vc.VC_SHADE_LOCAL), ("path_tracing", vc.VC_SHADE_PATH)):
        def frame(f):
            vc.vc_render(vol, offsets.data_ptr(), lods.data_ptr(), cache.data_ptr(), cam, RENDER_MATERIALS,
                         lab.data_ptr(), 0, 0, rgb.data_ptr(), stream.cuda_stream, mode=mode, frame=f, jitter=True,
                         max_bounces=8)
        frame(0)
        torch.cuda.synchronize()
        ms = []
        for f in range(1, 6):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            frame(f)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        med = float(np.median(ms))
        out["modes"][name] = {"frame_ms": med, "mrays_s": W * H / med / 1e3,
                              "hit_fraction": float((lab != 0).float().mean())}
    # post-processing of path-traced frames: accumulation, G-buffer, 3 À-trous passes with
    # upsampling, tone map; every pixel rendered, and one pixel of each 4 x 4 block per frame
    dep = torch.empty(W * H, dtype=torch.float32, device="cuda")
    face = torch.empty(W * H, dtype=torch.uint8, device="cuda")
    state = torch.zeros(vc.vc_post_state_bytes(W, H), dtype=torch.uint8, device="cuda")
    rgba = torch.empty(W * H, dtype=torch.int32, device="cuda")
    for sub in (1, 4):
        ms_r, ms_p = [], []
        for f in range(6):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            vc.vc_render(vol, offsets.data_ptr(), lods.data_ptr(), cache.data_ptr(), cam, RENDER_MATERIALS,
                         lab.data_ptr(), dep.data_ptr(), face.data_ptr(), rgb.data_ptr(), stream.cuda_stream,
                         mode=vc.VC_SHADE_PATH, frame=f, jitter=False, max_bounces=8, subsample=sub)
            e1.record(stream)
            vc.vc_postprocess(vol, W, H, lab.data_ptr(), dep.data_ptr(), face.data_ptr(), rgb.data_ptr(),
                              state.data_ptr(), rgba.data_ptr(), RENDER_MATERIALS, (-350.0, 700.0, -520.0),
                              iterations=3, subsample=sub, frame=f, reset=f == 0, stream=stream.cuda_stream)
            e2.record(stream)
            torch.cuda.synchronize()
            if f:
                ms_r.append(e0.elapsed_time(e1))
                ms_p.append(e1.elapsed_time(e2))
        out["modes"][f"path_tracing_subsample{sub}_with_post"] = {
            "render_ms": float(np.median(ms_r)), "post_ms": float(np.median(ms_p)),
            "frame_ms": float(np.median(ms_r) + np.median(ms_p))}
    return out


def run_ours(args):
    import torch
    import paper_2609_36898_gb300 as vc
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec, V, enc, t_gen, t_enc = make_workload(log2b=args.log2b, runs=args.runs)
    vol = vc.Volume(enc, device=local)
    n = vol.n_bricks
    e = vol.b
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    cache = torch.empty(n * e ** 3, dtype=torch.int32, device=dev)
    status = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    if args.mode == "auto":
        # the library's autotuner picks the schedule (grid or batched, threads per brick, staging
        # depth, blocks per SM) on this very request, before the warm-up
        sched, mode, _ = vc.vc_volume_autotune(vol.handle, ids.data_ptr(), n, ids.data_ptr(), cache.data_ptr(), 0,
                                               status.data_ptr(), stream.cuda_stream, reps=3)
        torch.cuda.synchronize()
        status.zero_()
        mode_name = next(k for k in ("grid", "batched") if vc.MODES[k] == mode)
    else:
        mode_name = args.mode
        mode = vc.MODES[mode_name]
    sched = vc.vc_volume_get_schedule(vol.handle)

    def step():
        vc.vc_decode_bricks(vol.handle, ids.data_ptr(), n, ids.data_ptr(), cache.data_ptr(), 0, mode,
                            status.data_ptr(), stream.cuda_stream)

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    if int(status[0]) != 0:
        raise RuntimeError(f"decode status {status.tolist()}")
    # correctness of the whole warm-up output against the generator (lossless), every brick,
    # outside the timed region
    verify_all(cache, V, e, "warm-up")

    vc.vc_volume_kernel_stats(vol.handle, reset=True)
    vc.vc_volume_set_profiling(vol.handle, True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        time.sleep(0.5)  # let the sampler start before the timed region
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k)
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    kst = vc.vc_volume_kernel_stats(vol.handle, reset=True)
    vc.vc_volume_set_profiling(vol.handle, False)
    step_ms = [s.elapsed_time(t) for s, t in zip(starts, ends)]
    dev_s = max_over_ranks(sum(step_ms) / 1000.0, dev)
    if int(status[0]) != 0:
        raise RuntimeError(f"decode status {status.tolist()}")
    verify_all(cache, V, e, "timed steps")  # outside the timed region
    vox_per_step = n * e ** 3
    value = job_rate(world, vox_per_step, args.steps, dev_s)
    algo = algorithmic_bytes(enc, n, e)
    # the dominant kernel is the reconstruction kernel: its average launch duration comes from the
    # library's timing events on the launching stream (one launch per step)
    if kst.timed_calls != args.steps or kst.reconstruct_ms <= 0:
        raise RuntimeError(f"kernel timing incomplete: {kst.timed_calls} of {args.steps} steps")
    recon_s = kst.reconstruct_ms / 1000.0 / kst.timed_calls
    symbol_s = kst.symbol_ms / 1000.0 / kst.timed_calls
    peak, peak_kind = measured_peak()
    achieved = algo / recon_s / 1e9
    step_achieved = algo / (dev_s / args.steps) / 1e9
    traffic = ncu_traffic(kernel_hash(), mode_name, sched[0], args.log2b, args.runs)

    # other schedules on the same data (context): plain = one launch per brick, grid = one launch
    # (the one-launch-per-brick schedule runs on the first 512 bricks only, to bound launch counts)
    modes = {}
    for mname in ("plain", "grid", "batched"):
        m = vc.MODES[mname]
        nsub = 512 if mname == "plain" else n
        reps = 3
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(reps):
            flush.fill_(3)
            ev0.record(stream)
            vc.vc_decode_bricks(vol.handle, ids.data_ptr(), nsub, ids.data_ptr(), cache.data_ptr(), 0, m,
                                status.data_ptr(), stream.cuda_stream)
            ev1.record(stream)
            torch.cuda.synchronize()
            tot += ev0.elapsed_time(ev1)
        modes[mname] = nsub * e ** 3 * reps / (tot / 1000.0) / 1e9

    # cache paletting (packed palette indices instead of u32 labels), same bricks, batched schedule
    pw, pbits, pper = vc.vc_volume_slot_words(vol.handle, 0, True)
    pcache = torch.empty(n * pw, dtype=torch.int32, device=dev)
    pm = mode | vc.VC_MODE_PALETTED
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    vc.vc_decode_bricks(vol.handle, ids.data_ptr(), n, ids.data_ptr(), pcache.data_ptr(), 0, pm, status.data_ptr(),
                        stream.cuda_stream)
    ptot = 0.0
    for _ in range(5):
        flush.fill_(5)
        ev0.record(stream)
        vc.vc_decode_bricks(vol.handle, ids.data_ptr(), n, ids.data_ptr(), pcache.data_ptr(), 0, pm,
                            status.data_ptr(), stream.cuda_stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ptot += ev0.elapsed_time(ev1)
    p_s = ptot / 5 / 1000.0
    p_algo = algo - 4 * n * e ** 3 + 4 * n * pw
    paletted = {"gvoxel_s": vox_per_step / p_s / 1e9, "bits_per_index": pbits, "indices_per_word": pper,
                "bytes_per_voxel_written": 4.0 * pw / e ** 3, "step_ms": 1000 * p_s,
                "algorithmic_bytes_per_step": p_algo, "step_frac_of_peak": p_algo / p_s / 1e9 / peak}
    del pcache
    if int(status[0]) != 0:
        raise RuntimeError(f"paletted decode status {status.tolist()}")

    # end to end through the host entry point: ids host->device, decode, labels device->host (pinned)
    ids_h = torch.arange(n, dtype=torch.int32).numpy().view(np.uint32)
    labels_h = torch.empty(n * e ** 3, dtype=torch.int32, pin_memory=True)
    labels_np = labels_h.numpy().view(np.uint32)
    e2e_steps = max(2, min(args.steps, 5))
    vc.vc_decode_bricks_host(vol.handle, ids_h, 0, mode, labels_np, stream.cuda_stream)  # warm-up / allocation
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        st = vc.vc_decode_bricks_host(vol.handle, ids_h, 0, mode, labels_np, stream.cuda_stream)
        if st != 0:
            raise RuntimeError(f"host decode status {st}")
    e2e_s = time.perf_counter() - t0
    e2e_val = world * vox_per_step * e2e_steps / e2e_s / 1e9
    nz, ny, nx = (s // e for s in V.shape)
    if not np.array_equal(labels_np, V.reshape(nz, e, ny, e, nx, e).transpose(0, 2, 4, 1, 3, 5).reshape(-1)):
        raise AssertionError("end-to-end decode differs from the input volume")

    # detail split: the same volume with its finest level left in (mapped, pinned) host memory
    split = None
    if not args.no_split:
        sv = vc.Volume(enc, device=local, split=True)
        sinfo, finfo = vc.vc_volume_info_get(sv.handle), vc.vc_volume_info_get(vol.handle)
        smode = vc.MODES["grid"]
        split = {"device_bytes": int(sinfo.device_bytes), "device_bytes_unsplit": int(finfo.device_bytes),
                 "host_bytes": int(sinfo.host_bytes),
                 "device_saving": 1.0 - sinfo.device_bytes / finfo.device_bytes}
        for lod in (0, 1):
            e_l = e >> lod
            words_l = n * e_l ** 3
            vc.vc_decode_bricks(sv.handle, ids.data_ptr(), n, ids.data_ptr(), cache.data_ptr(), lod, smode,
                                status.data_ptr(), stream.cuda_stream)
            tot, reps = 0.0, 5
            for _ in range(reps):
                flush.fill_(7)
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                vc.vc_decode_bricks(sv.handle, ids.data_ptr(), n, ids.data_ptr(), cache.data_ptr(), lod, smode,
                                    status.data_ptr(), stream.cuda_stream)
                ev1.record(stream)
                torch.cuda.synchronize()
                tot += ev0.elapsed_time(ev1)
            split[f"lod{lod}_gvoxel_s"] = words_l * reps / (tot / 1000.0) / 1e9
            split[f"lod{lod}_reads"] = "whole records from mapped host memory" if lod == 0 else \
                "coarse-level records in device memory"
        if int(status[0]) != 0:
            raise RuntimeError(f"split decode status {status.tolist()}")
        sv.release()

    ablation = ablation_leg(V) if not args.no_ablation else None
    render = render_leg(vol.handle, cache, n, e, stream, local)
    serving = None
    if args.serve_frames > 0:
        serving = serving_leg(args, local)
    mixed = None
    if args.mixed_requests > 0:
        mixed = mixed_serving_leg(args, local)
    subsets = None
    if args.subsets > 0:
        del cache
        subsets = subsets_leg(args, local)

    out = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            r, nb, dt = oracle_rate(enc, 15.0, 10 ** 9)
            cpu = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{nb} brick decodes (bricks 0, 1, ... cycling over all {n}) of the same 512^3 volume, "
                             f"single-threaded, {dt:.1f} s", **host_cpu()}
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * dev_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": workload_name(args.log2b, args.runs), "bricks_per_step": n,
                       "voxels_per_step": vox_per_step,
                       "schedule": mode_name, "autotuned": args.mode == "auto",
                       "threads_per_brick": sched[0], "stage_depth": sched[1], "blocks_per_sm": sched[2],
                       "encoded_bytes": int(enc.size),
                       "bits_per_voxel": 8.0 * enc.size / V.size, "l2": "flushed before every step (256 MiB write)",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": algo,
                         "kernel": kernel_name(mode_name, sched[0], args.log2b),
                         "kernel_ms": 1000.0 * recon_s, "symbol_kernel_ms": 1000.0 * symbol_s,
                         "step_achieved": step_achieved, "step_frac": step_achieved / peak},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 4 * n,
                    "d2h_bytes_per_step": 4 * n * e ** 3 + 4},
            "gpu_launches": int(kst.launches),
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "schedules_gvoxel_s": modes,
            "paletted": paletted,
            "detail_split": split,
            "serving": serving,
            "mixed_serving": mixed,
            "power_diagram_subsets": subsets,
            "operation_ablation": ablation,
            "render": render,
            "wall_s_timed_region": wall,
            "prep_s": {"generate": t_gen, "encode": t_enc},
        }
        print(json.dumps(out))
    vol.release()
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="auto", choices=["auto", "grid", "batched"])
    ap.add_argument("--log2b", type=int, default=B_LOG2, choices=[4, 5, 6],
                    help="brick size of the main decode leg (5: 32^3 bricks, the benchmark)")
    ap.add_argument("--runs", type=int, default=1, choices=[1, 2, 4, 8], help="rANS runs per record")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-split", action="store_true", help="skip the detail-split leg")
    ap.add_argument("--no-ablation", action="store_true", help="skip the operation-prefix compression sweep")
    ap.add_argument("--subsets", type=int, default=3,
                    help="random 100,000-brick subsets of the 2048x2048x1024 power-diagram volume to time (0 = skip)")
    ap.add_argument("--serve-frames", type=int, default=4, help="frames of the serving leg (0 = skip it)")
    ap.add_argument("--serve-size", type=int, default=4096, help="edge of the serving volume")
    ap.add_argument("--serve-cameras", type=int, default=64)
    ap.add_argument("--serve-plain-cameras", type=int, default=1)
    ap.add_argument("--mixed-requests", type=int, default=300, help="requests of the mixed serving leg (0 = skip)")
    ap.add_argument("--mixed-plain-requests", type=int, default=40)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
