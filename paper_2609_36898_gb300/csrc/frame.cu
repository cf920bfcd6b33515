// Frame cache: the per-frame cache stages of the rendering pipeline on the device, with no host
// round trip inside a frame (Methods, "GPU rendering pipeline"; Results, "GPU-based rendering
// pipeline"; Methods, "Memory management" and "Cache defragmentation"). The contract is written in
// include/vc.h at vc_frame_update; this file holds the stages:
//   begin      one thread: a pending defragmentation empties the cache (top = 0, free stacks
//              empty); the request counters restart.
//   request    one thread per brick: the marks of the last frame say which bricks are visible; a
//              visible brick's level of detail comes from the cameras (brick centre rule); a
//              cached brick that is no longer visible, or visible at another level, gives its
//              region back to its level's free stack (a full stack leaves the region dead); a
//              visible brick not cached at its level goes onto its level's request stack. The marks
//              are cleared for the next frame.
//   provision  one thread: per level, finest first, requests are served from the level's free
//              stack, then from the top of the cache buffer (aligned to the level's region size),
//              within the per-frame brick limit; if the top runs out and the free space held
//              elsewhere (other levels' stacks, dead regions, the rest of the buffer) would fit what
//              is missing, the next frame starts with a defragmentation.
//   assign     one thread per assigned request: the brick's region, offset and level.
//   decode     per level: the persistent decoder over the assigned bricks, the count read on the
//              device.
// Regions of level k are (b / 2^k)^3 labels; a region keeps its level while it is free (free
// stacks are per level), as in the paper.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstring>

#include "vc_internal.h"

namespace vc {

constexpr uint32_t kHandleFrame = 0x464D4331u;  // "FMC1"
constexpr uint32_t kMaxLevels = 8;              // levels of detail 0..L, L <= 6
constexpr uint32_t kMaxLodCams = 256;           // cameras of one vc_frame_update
constexpr uint32_t kNone8 = 0xFFu;
constexpr uint64_t kNotCached = ~0ull;

// Device-side control block.
struct FrameCtrl {
  unsigned long long top;         // labels in use from the bottom of the buffer (bump pointer)
  unsigned long long dead;        // labels in regions lost to full free stacks or alignment
  unsigned long long top_base[kMaxLevels];
  uint32_t req_n[kMaxLevels];     // requests pushed this frame (may exceed the stack's capacity)
  uint32_t free_n[kMaxLevels];    // entries on the free stacks (may exceed capacity after pushes)
  uint32_t take[kMaxLevels];      // requests served from the free stack this frame
  uint32_t free_base[kMaxLevels]; // the first free-stack entry they take
  uint32_t assign_n[kMaxLevels];  // requests assigned this frame (free stack + top)
  uint32_t assign_pre[kMaxLevels + 1];
  uint32_t reset_pending, in_reset;
  // statistics: cumulative, then of the last frame
  unsigned long long frames, requested, assigned, voxels, freed, unassigned, resets, switches;
  uint32_t f_resident, f_requested, f_assigned, f_freed, f_unassigned, f_switches;
};

struct FrameDev {
  uint64_t* offsets;
  uint8_t* lods;
  uint32_t* marks;
  uint32_t* free_stack;  // level l at l * free_cap
  uint32_t* req;         // level l at l * max_req: brick ids (the decode lists)
  uint32_t* slots;       // level l at l * max_req: region index in units of the level's size
  uint32_t n_bricks, L, nb[3];
  uint32_t free_cap, max_req, max_lod;
  unsigned long long cap;  // buffer size in labels
  uint32_t per_frame;      // bricks assigned per frame at most
};

struct LodCams {
  float o[kMaxLodCams][3];
  float s2[kMaxLodCams];  // (2 tan(fov / 2) / H)^2
  uint32_t n;
  float b;
};

struct FrameCache {
  uint32_t kind;  // kHandleFrame
  Volume* v;
  FrameDev d;
  uint32_t* cache;
  FrameCtrl* ctrl;
  uint8_t* ws;
  size_t ws_bytes;
};

namespace {

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Labels in a region of level l.
__host__ __device__ __forceinline__ unsigned long long region(uint32_t L, uint32_t l) {
  return 1ull << (3u * (L - l));
}

// Pushes onto per-level stacks, one atomic per level and warp: key = level or kNone8. Returns the
// position of this lane's entry (undefined for kNone8). Every lane of the warp calls it.
__device__ __forceinline__ uint32_t push_warp(uint32_t key, uint32_t* counters) {
  const uint32_t active = __ballot_sync(0xFFFFFFFFu, key != kNone8);
  uint32_t pos = 0;
  if (key != kNone8) {
    const uint32_t peers = __match_any_sync(active, key);
    const uint32_t leader = __ffs(peers) - 1u;
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&counters[key], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    pos = base + (uint32_t)__popc(peers & lanemask_lt());
  }
  return pos;
}

__device__ __forceinline__ void count_warp(bool pred, uint32_t* ctr) {
  const uint32_t m = __ballot_sync(0xFFFFFFFFu, pred);
  if ((threadIdx.x & 31u) == 0 && m) atomicAdd(ctr, (uint32_t)__popc(m));
}

__global__ void frame_begin_kernel(FrameCtrl* c, uint32_t nlev) {
  if (threadIdx.x != 0) return;
  c->in_reset = c->reset_pending;
  if (c->reset_pending) {  // defragmentation: every region is given up at once
    c->top = 0;
    c->dead = 0;
    for (uint32_t l = 0; l < nlev; ++l) c->free_n[l] = 0;
    c->resets += 1;
    c->reset_pending = 0;
  }
  for (uint32_t l = 0; l < nlev; ++l) c->req_n[l] = 0;
  c->f_resident = c->f_requested = c->f_assigned = c->f_freed = c->f_unassigned = c->f_switches = 0;
}

// Level of detail of brick (bx, by, bz): the largest k <= max_lod with 4^k <= |c - o|^2 s^2 for
// the nearest camera (the request stage's rule, per camera; the finest over the cameras).
__device__ uint32_t brick_lod(const LodCams& C, uint32_t max_lod, uint32_t bx, uint32_t by, uint32_t bz) {
  const float cx0 = fmul(fadd((float)bx, 0.5f), C.b), cy0 = fmul(fadd((float)by, 0.5f), C.b),
              cz0 = fmul(fadd((float)bz, 0.5f), C.b);
  uint32_t best = max_lod;
  for (uint32_t i = 0; i < C.n && best > 0; ++i) {
    const float cx = fsub(cx0, C.o[i][0]), cy = fsub(cy0, C.o[i][1]), cz = fsub(cz0, C.o[i][2]);
    const float q = fmul(fadd(fadd(fmul(cx, cx), fmul(cy, cy)), fmul(cz, cz)), C.s2[i]);
    uint32_t lod = 0;
    while (lod < max_lod && q >= (float)(1u << (2u * (lod + 1u)))) ++lod;
    best = min(best, lod);
  }
  return best;
}

// One thread per brick, a warp per 32 consecutive bricks (one word of marks).
__global__ void __launch_bounds__(256) frame_request_kernel(FrameCtrl* c, const FrameDev D,
                                                            const __grid_constant__ LodCams C) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * blockDim.x;
  const bool reset = c->in_reset != 0;
  for (uint32_t b0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b0 < D.n_bricks; b0 += stride) {
    uint32_t word = 0;
    if (lane == 0) {
      word = D.marks[b0 >> 5];
      if (word) D.marks[b0 >> 5] = 0u;  // cleared for the next frame's marks
    }
    word = __shfl_sync(0xFFFFFFFFu, word, 0);
    const uint32_t b = b0 + lane;
    const bool in = b < D.n_bricks;
    const bool vis = in && ((word >> lane) & 1u);
    uint32_t cur = in ? D.lods[b] : kNone8;
    if (reset && cur != kNone8) {  // defragmentation: the brick is no longer cached
      D.offsets[b] = kNotCached;
      D.lods[b] = (uint8_t)kNone8;
      cur = kNone8;
    }
    uint32_t want = kNone8;
    if (vis) {
      const uint32_t bx = b % D.nb[0], by = (b / D.nb[0]) % D.nb[1], bz = b / (D.nb[0] * D.nb[1]);
      want = brick_lod(C, D.max_lod, bx, by, bz);
    }
    const uint32_t free_l = (cur != kNone8 && cur != want) ? cur : kNone8;
    const uint32_t req_l = (vis && cur != want) ? want : kNone8;
    uint32_t slot = 0;
    if (free_l != kNone8) {
      slot = (uint32_t)(D.offsets[b] / region(D.L, cur));
      D.offsets[b] = kNotCached;
      D.lods[b] = (uint8_t)kNone8;
    }
    const uint32_t fpos = push_warp(free_l, c->free_n);
    if (free_l != kNone8) {
      if (fpos < D.free_cap) D.free_stack[(size_t)free_l * D.free_cap + fpos] = slot;
      else atomicAdd(&c->dead, region(D.L, free_l));  // stack full: the region stays dead until a reset
    }
    const uint32_t rpos = push_warp(req_l, c->req_n);
    if (req_l != kNone8 && rpos < D.max_req) D.req[(size_t)req_l * D.max_req + rpos] = b;
    count_warp(vis && cur == want, &c->f_resident);
    count_warp(free_l != kNone8, &c->f_freed);
    count_warp(free_l != kNone8 && vis, &c->f_switches);
  }
}

__global__ void frame_provision_kernel(FrameCtrl* c, const FrameDev D) {
  if (threadIdx.x != 0) return;
  const uint32_t nlev = D.max_lod + 1u;
  uint32_t left = D.per_frame, requested = 0, assigned = 0;
  unsigned long long top = c->top, dead = c->dead, voxels = 0, missing = 0;
  bool overflow = false;
  c->assign_pre[0] = 0;
  for (uint32_t l = 0; l < kMaxLevels; ++l) {
    if (l >= nlev) {
      c->assign_n[l] = 0;
      c->assign_pre[l + 1] = c->assign_pre[l];
      continue;
    }
    const unsigned long long sz = region(D.L, l);
    const uint32_t avail = min(c->free_n[l], D.free_cap);
    const uint32_t want = min(min(c->req_n[l], D.max_req), left);
    const uint32_t take = min(want, avail);
    const uint32_t need = want - take;
    const unsigned long long at = (top + sz - 1ull) / sz * sz;  // the level's regions start aligned
    const unsigned long long room = at < D.cap ? (D.cap - at) / sz : 0ull;
    const uint32_t from_top = (uint32_t)min((unsigned long long)need, room);
    if (from_top < need) {
      overflow = true;
      missing += (unsigned long long)(need - from_top) * sz;
    }
    if (from_top) {
      dead += at - top;
      c->top_base[l] = at;
      top = at + (unsigned long long)from_top * sz;
    }
    c->take[l] = take;
    c->free_base[l] = avail - take;
    c->free_n[l] = avail - take;
    c->assign_n[l] = take + from_top;
    c->assign_pre[l + 1] = c->assign_pre[l] + take + from_top;
    left -= take + from_top;
    requested += c->req_n[l];
    assigned += take + from_top;
    voxels += (unsigned long long)(take + from_top) * sz;
  }
  c->top = top;
  c->dead = dead;
  // defragmentation (once, at the start of the next frame) when it would make room for what is
  // missing: free regions held by other levels, dead regions and the buffer's rest add up to it
  if (overflow && !c->in_reset) {
    unsigned long long spare = dead + (D.cap - top);
    for (uint32_t l = 0; l < nlev; ++l) spare += (unsigned long long)c->free_n[l] * region(D.L, l);
    if (spare >= missing) c->reset_pending = 1;
  }
  c->f_requested = requested;
  c->f_assigned = assigned;
  c->f_unassigned = requested - assigned;
  c->frames += 1;
  c->requested += requested;
  c->assigned += assigned;
  c->voxels += voxels;
  c->unassigned += requested - assigned;
  c->freed += c->f_freed;
  c->switches += c->f_switches;
}

__global__ void __launch_bounds__(256) frame_assign_kernel(const FrameCtrl* __restrict__ c, const FrameDev D) {
  const uint32_t nlev = D.max_lod + 1u;
  const uint32_t total = c->assign_pre[nlev];
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    uint32_t l = 0;
    while (t >= c->assign_pre[l + 1]) ++l;
    const uint32_t i = t - c->assign_pre[l];
    const unsigned long long sz = region(D.L, l);
    const uint32_t b = D.req[(size_t)l * D.max_req + i];
    const uint32_t slot = i < c->take[l] ? D.free_stack[(size_t)l * D.free_cap + c->free_base[l] + i]
                                         : (uint32_t)(c->top_base[l] / sz) + (i - c->take[l]);
    D.slots[(size_t)l * D.max_req + i] = slot;
    D.offsets[b] = (uint64_t)slot * sz;
    D.lods[b] = (uint8_t)l;
  }
}

}  // namespace

static void free_frame(FrameCache* f) {
  cudaFree(f->cache);
  cudaFree(f->d.offsets);
  cudaFree(f->d.lods);
  cudaFree(f->d.marks);
  cudaFree(f->d.free_stack);
  cudaFree(f->d.req);
  cudaFree(f->d.slots);
  cudaFree(f->ctrl);
  cudaFree(f->ws);
  f->kind = 0;
  delete f;
}

bool release_frame(void* handle) {
  FrameCache* f = static_cast<FrameCache*>(handle);
  if (!f || f->kind != kHandleFrame) return false;
  int prev = -1;
  cudaGetDevice(&prev);
  const int device = f->v->device;  // f is gone after free_frame
  if (prev != device) cudaSetDevice(device);
  cudaDeviceSynchronize();
  free_frame(f);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return true;
}

}  // namespace vc

using namespace vc;

namespace {

FrameCache* as_frame(vc_frame_cache* h) {
  FrameCache* f = reinterpret_cast<FrameCache*>(h);
  return f && f->kind == kHandleFrame ? f : nullptr;
}

bool cams_ok(const vc_camera* cams, uint32_t n) {
  for (uint32_t i = 0; i < n; ++i)
    if (cams[i].width == 0 || cams[i].height == 0 || (uint64_t)cams[i].width * cams[i].height > 0xFFFFFFFFull)
      return false;
  return true;
}

struct DeviceScope {
  int prev = -1, dev;
  explicit DeviceScope(int d) : dev(d) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceScope() {
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

vc_status vc_frame_cache_create(vc_volume* vol, uint64_t cache_bytes, uint32_t max_bricks_per_frame,
                                uint32_t free_stack_entries, vc_frame_cache** out) {
  Volume* v = reinterpret_cast<Volume*>(vol);
  if (!out) return VC_ERR_ARG;
  *out = nullptr;
  if (!v || v->kind != kHandleVolume || cache_bytes < 4 || v->L + 1u > kMaxLevels) return VC_ERR_ARG;
  DeviceScope scope(v->device);
  FrameCache* f = new FrameCache();
  std::memset(f, 0, sizeof(*f));
  f->v = v;
  const uint32_t n = v->n_bricks;
  FrameDev& d = f->d;
  d.n_bricks = n;
  d.L = v->L;
  for (int a = 0; a < 3; ++a) d.nb[a] = v->nb[a];
  d.free_cap = free_stack_entries ? free_stack_entries : (1u << 20);
  d.per_frame = max_bricks_per_frame ? std::min(max_bricks_per_frame, n) : std::min(n, 262144u);
  d.max_req = d.per_frame;
  d.cap = cache_bytes / 4;
  const uint32_t nlev = v->L + 1u;
  const size_t words = ((size_t)n + 31) / 32;
  f->ws_bytes = decode_ws_bytes(*v, d.per_frame);
  bool ok = cudaMalloc(reinterpret_cast<void**>(&f->cache), d.cap * 4) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&d.offsets), (size_t)n * 8) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&d.lods), n) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&d.marks), words * 4) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&d.free_stack), (size_t)nlev * d.free_cap * 4) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&d.req), (size_t)nlev * d.max_req * 4) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&d.slots), (size_t)nlev * d.max_req * 4) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&f->ctrl), sizeof(FrameCtrl)) == cudaSuccess &&
            (f->ws_bytes == 0 || cudaMalloc(reinterpret_cast<void**>(&f->ws), f->ws_bytes) == cudaSuccess);
  ok = ok && cudaMemset(d.offsets, 0xFF, (size_t)n * 8) == cudaSuccess &&
       cudaMemset(d.lods, 0xFF, n) == cudaSuccess && cudaMemset(d.marks, 0, words * 4) == cudaSuccess &&
       cudaMemset(f->ctrl, 0, sizeof(FrameCtrl)) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_frame(f);
    return VC_ERR_OOM;
  }
  f->kind = kHandleFrame;
  *out = reinterpret_cast<vc_frame_cache*>(f);
  return VC_OK;
}

vc_status vc_frame_cache_view_get(vc_frame_cache* fc, vc_frame_cache_view* out) {
  FrameCache* f = as_frame(fc);
  if (!f || !out) return VC_ERR_ARG;
  out->offsets = f->d.offsets;
  out->lods = f->d.lods;
  out->cache = f->cache;
  out->marks = f->d.marks;
  out->cache_words = f->d.cap;
  out->n_bricks = f->d.n_bricks;
  out->max_bricks_per_frame = f->d.per_frame;
  out->free_stack_entries = f->d.free_cap;
  return VC_OK;
}

vc_status vc_frame_mark_cameras(vc_frame_cache* fc, const vc_camera* cams, uint32_t ncams, void* cuda_stream) {
  FrameCache* f = as_frame(fc);
  if (!f || (ncams && !cams) || !cams_ok(cams, ncams)) return VC_ERR_ARG;
  if (ncams == 0) return VC_OK;
  DeviceScope scope(f->v->device);
  const vc_status rc = launch_shared_marks(*f->v, cams, ncams, f->d.marks, static_cast<cudaStream_t>(cuda_stream));
  if (rc == VC_OK) f->v->launches += (ncams + 63u) / 64u;
  return rc;
}

vc_status vc_frame_update(vc_frame_cache* fc, const vc_camera* cams, uint32_t ncams, uint32_t max_lod,
                          int32_t* status_dev, void* cuda_stream) {
  FrameCache* f = as_frame(fc);
  if (!f || !cams || ncams == 0 || ncams > kMaxLodCams || !status_dev || !cams_ok(cams, ncams)) return VC_ERR_ARG;
  Volume& v = *f->v;
  DeviceScope scope(v.device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  FrameDev D = f->d;
  D.max_lod = std::min(max_lod, v.L);
  static_assert(sizeof(LodCams) < 32000, "kernel parameter space");
  LodCams C;
  std::memset(&C, 0, sizeof(C));
  for (uint32_t i = 0; i < ncams; ++i) {
    CamDev cd;
    camera_frame(cams[i], &cd);
    for (int a = 0; a < 3; ++a) C.o[i][a] = cd.o[a];
    C.s2[i] = cd.lod_s2;
  }
  C.n = ncams;
  C.b = (float)(1u << v.L);
  const uint32_t nlev = D.max_lod + 1u;
  const uint32_t sms = std::max(1u, v.sms);
  const uint32_t rblocks = std::min<uint32_t>((D.n_bricks + 255u) / 256u, sms * 8u);
  const uint32_t ablocks = std::min<uint32_t>((D.per_frame + 255u) / 256u, sms * 8u);
  frame_begin_kernel<<<1, 32, 0, st>>>(f->ctrl, v.L + 1u);
  frame_request_kernel<<<rblocks, 256, 0, st>>>(f->ctrl, D, C);
  frame_provision_kernel<<<1, 32, 0, st>>>(f->ctrl, D);
  frame_assign_kernel<<<ablocks, 256, 0, st>>>(f->ctrl, D);
  if (cudaGetLastError() != cudaSuccess) return VC_ERR_CUDA;
  v.launches += 4;
  for (uint32_t l = 0; l < nlev; ++l) {
    const uint32_t* n_dev = reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(f->ctrl) +
                                                              offsetof(FrameCtrl, assign_n) + 4u * l);
    const vc_status rc =
        launch_decode_devcount(v, D.req + (size_t)l * D.max_req, D.max_req, n_dev, D.slots + (size_t)l * D.max_req,
                               f->cache, l, status_dev, st, f->ws, f->ws_bytes);
    if (rc != VC_OK) return rc;
  }
  return VC_OK;
}

vc_status vc_frame_stats_get(vc_frame_cache* fc, vc_frame_stats* out, void* cuda_stream) {
  FrameCache* f = as_frame(fc);
  if (!f || !out) return VC_ERR_ARG;
  DeviceScope scope(f->v->device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  FrameCtrl c;
  if (cudaMemcpyAsync(&c, f->ctrl, sizeof(c), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return VC_ERR_CUDA;
  std::memset(out, 0, sizeof(*out));
  out->frames = c.frames;
  out->bricks_requested = c.requested;
  out->bricks_decoded = c.assigned;
  out->voxels_decoded = c.voxels;
  out->bricks_freed = c.freed;
  out->bricks_unassigned = c.unassigned;
  out->resets = c.resets;
  out->level_switches = c.switches;
  out->top_words = c.top;
  out->dead_words = c.dead;
  out->last_resident = c.f_resident;
  out->last_requested = c.f_requested;
  out->last_decoded = c.f_assigned;
  out->last_unassigned = c.f_unassigned;
  out->last_freed = c.f_freed;
  out->reset_pending = c.reset_pending;
  for (uint32_t l = 0; l < kMaxLevels && l <= f->v->L; ++l)
    out->free_entries[l] = std::min(c.free_n[l], f->d.free_cap);
  return VC_OK;
}

}  // extern "C"
