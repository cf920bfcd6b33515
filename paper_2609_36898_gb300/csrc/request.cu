// Camera request stage: which bricks the pixel rays of pinhole cameras need, and at which level of
// detail. Paper, Methods "GPU rendering pipeline": rays traced through the volume mark the bricks
// they pass as visible, bricks holding no visible label are skipped, and a brick's level of
// detail depends only on its centre position; Results "Ray marching": one voxel of the chosen
// level covers about one pixel, and the DDA keeps an integer cell index plus a sub-cell position
// in [0, 1] for numerical stability. Here the cells are bricks:
//   - a brick is visible iff its palette holds a label other than 0 (0 = background), and a ray
//     ends after the first brick whose palette has no 0 (it certainly hits a surface there);
//   - the ray of pixel (px, py) is o + t (f + sx r + sy u) with sx = ((px + 1/2) 2/W - 1) tan(fov/2)
//     W/H and sy = (1 - (py + 1/2) 2/H) tan(fov/2), (f, r, u) the camera frame;
//   - level of detail k = the largest k <= max_lod with 4^k <= |c - o|^2 (2 tan(fov/2) / H)^2.
// The camera frame and scales are computed once per camera in double precision and rounded to
// float; every per-ray and per-brick step below is one correctly rounded float operation in a
// fixed order (explicit _rn intrinsics, no contraction), so the integer decisions (cells, stops,
// levels) are a pure function of the inputs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "vc_internal.h"

namespace vc {

static_assert(sizeof(CamDev) == kCamDevBytes, "camera staging size");

void camera_frame(const vc_camera& c, CamDev* d) {
  double f[3] = {c.dir[0], c.dir[1], c.dir[2]};
  const double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  for (int a = 0; a < 3; ++a) f[a] /= fl;
  const double up[3] = {c.up[0], c.up[1], c.up[2]};
  double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
  const double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  for (int a = 0; a < 3; ++a) r[a] /= rl;
  const double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
  const double t = std::tan(0.5 * (double)c.fov_y);
  for (int a = 0; a < 3; ++a) {
    d->o[a] = c.pos[a];
    d->f[a] = (float)f[a];
    d->r[a] = (float)r[a];
    d->u[a] = (float)u[a];
  }
  d->sxs = (float)(t * (double)c.width / (double)c.height);
  d->sys = (float)t;
  d->inv_w2 = (float)(2.0 / (double)c.width);
  d->inv_h2 = (float)(2.0 / (double)c.height);
  const double s = 2.0 * t / (double)c.height;
  d->lod_s2 = (float)(s * s);
  d->W = c.width;
  d->H = c.height;
}

namespace {

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

struct Grid {
  uint32_t nb[3];
  float b;
};

// The brick ray of pixel i of camera c: marks the visible bricks it passes in mk (one bit per
// brick) until the first brick with no background.
__device__ void march_pixel(const CamDev& c, const uint8_t* __restrict__ flags, const Grid& g, uint32_t* mk,
                            uint32_t i) {
  const uint32_t px = i % c.W, py = i / c.W;
  const float sx = fmul(fsub(fmul(fadd((float)px, 0.5f), c.inv_w2), 1.0f), c.sxs);
  const float sy = fmul(fsub(1.0f, fmul(fadd((float)py, 0.5f), c.inv_h2)), c.sys);
  float d[3], o[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float da = fadd(fadd(c.f[a], fmul(sx, c.r[a])), fmul(sy, c.u[a]));
    d[a] = fdiv(da, g.b);
    o[a] = fdiv(c.o[a], g.b);
  }
  float t0 = 0.0f, t1 = INFINITY;
  bool miss = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float n = (float)g.nb[a];
    if (d[a] == 0.0f) {
      if (o[a] < 0.0f || o[a] >= n) miss = true;
      continue;
    }
    float ta = fdiv(fsub(0.0f, o[a]), d[a]), tb = fdiv(fsub(n, o[a]), d[a]);
    if (ta > tb) { const float x = ta; ta = tb; tb = x; }
    if (ta > t0) t0 = ta;
    if (tb < t1) t1 = tb;
  }
  if (miss || !(t0 < t1)) return;
  int32_t cell[3];
  float s[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float p = fadd(o[a], fmul(t0, d[a]));
    float fc = floorf(p);
    if (fc < 0.0f) fc = 0.0f;
    if (fc > (float)(g.nb[a] - 1)) fc = (float)(g.nb[a] - 1);
    cell[a] = (int32_t)fc;
    float q = fsub(p, fc);
    if (q < 0.0f) q = 0.0f;
    if (q > 1.0f) q = 1.0f;
    s[a] = q;
  }
  const uint32_t max_steps = g.nb[0] + g.nb[1] + g.nb[2] + 1;
  for (uint32_t step = 0; step < max_steps; ++step) {
    const uint32_t id = (uint32_t)cell[0] + g.nb[0] * ((uint32_t)cell[1] + g.nb[1] * (uint32_t)cell[2]);
    const uint32_t fl = flags[id];
    if (fl & 2u) {
      const uint32_t bit = 1u << (id & 31u);
      if (!(mk[id >> 5] & bit)) atomicOr(&mk[id >> 5], bit);
    }
    if (!(fl & 1u)) break;  // no background in this brick: the ray ends here
    float dist[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (d[a] > 0.0f) dist[a] = fdiv(fsub(1.0f, s[a]), d[a]);
      else if (d[a] < 0.0f) dist[a] = fdiv(fsub(0.0f, s[a]), d[a]);
      else dist[a] = INFINITY;
    }
    int ax = 0;
    if (dist[1] < dist[ax]) ax = 1;
    if (dist[2] < dist[ax]) ax = 2;
    const float t = dist[ax];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == ax) continue;
      float q = fadd(s[a], fmul(t, d[a]));
      if (q < 0.0f) q = 0.0f;
      if (q > 1.0f) q = 1.0f;
      s[a] = q;
    }
    if (d[ax] > 0.0f) {
      cell[ax] += 1;
      s[ax] = 0.0f;
      if (cell[ax] >= (int32_t)g.nb[ax]) break;
    } else {
      cell[ax] -= 1;
      s[ax] = 1.0f;
      if (cell[ax] < 0) break;
    }
  }
}

// One thread per pixel ray (blockIdx.y = camera); marks visible bricks in the camera's bitmask.
__global__ void camera_march_kernel(const CamDev* __restrict__ cams, const uint8_t* __restrict__ flags, Grid g,
                                    uint32_t* __restrict__ marks, uint32_t words) {
  const CamDev& c = cams[blockIdx.y];
  uint32_t* mk = marks + (size_t)blockIdx.y * words;
  const uint32_t npix = c.W * c.H;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x)
    march_pixel(c, flags, g, mk, i);
}

// Up to kMarkCams cameras per launch, passed by value (kernel parameter space: nothing to stage).
constexpr uint32_t kMarkCams = 64;
struct CamBlock {
  CamDev c[kMarkCams];
};

// The same rays of several cameras (blockIdx.y) into one shared bitmask.
__global__ void shared_march_kernel(const __grid_constant__ CamBlock cams, const uint8_t* __restrict__ flags, Grid g,
                                    uint32_t* __restrict__ marks) {
  const CamDev& c = cams.c[blockIdx.y];
  const uint32_t npix = c.W * c.H;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x)
    march_pixel(c, flags, g, marks, i);
}

constexpr uint32_t kCompactThreads = 1024;

// One block per camera: the marked bricks in ascending id order, with their levels of detail.
__global__ void __launch_bounds__(kCompactThreads)
    camera_compact_kernel(const CamDev* __restrict__ cams, const uint32_t* __restrict__ marks, uint32_t words,
                          Grid g, uint32_t max_lod, uint32_t cap, uint32_t* __restrict__ counts,
                          uint32_t* __restrict__ ids, uint32_t* __restrict__ lods) {
  __shared__ uint32_t warp_sum[kCompactThreads / 32];
  __shared__ uint32_t base_s;
  const CamDev& c = cams[blockIdx.x];
  const uint32_t* mk = marks + (size_t)blockIdx.x * words;
  uint32_t* out_ids = ids + (size_t)blockIdx.x * cap;
  uint32_t* out_lods = lods + (size_t)blockIdx.x * cap;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  if (tid == 0) base_s = 0;
  __syncthreads();
  // tiles of kCompactThreads words, in order; each thread one word per tile
  for (uint32_t w0 = 0; w0 < words; w0 += kCompactThreads) {
    const uint32_t w = w0 + tid;
    const uint32_t m = w < words ? mk[w] : 0u;
    const uint32_t cnt = __popc(m);
    uint32_t x = cnt;  // inclusive warp scan
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t v = lane < kCompactThreads / 32 ? warp_sum[lane] : 0u;
#pragma unroll
      for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += y;
      }
      if (lane < kCompactThreads / 32) warp_sum[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    uint32_t pos = base_s + (warp ? warp_sum[warp - 1] : 0u) + x - cnt;
    const uint32_t tile_total = warp_sum[kCompactThreads / 32 - 1];
    uint32_t bits = m;
    while (bits) {
      const uint32_t k = __ffs(bits) - 1u;
      bits &= bits - 1u;
      const uint32_t id = 32u * w + k;
      if (pos < cap) {
        const uint32_t bx = id % g.nb[0], by = (id / g.nb[0]) % g.nb[1], bz = id / (g.nb[0] * g.nb[1]);
        const float cx = fsub(fmul(fadd((float)bx, 0.5f), g.b), c.o[0]);
        const float cy = fsub(fmul(fadd((float)by, 0.5f), g.b), c.o[1]);
        const float cz = fsub(fmul(fadd((float)bz, 0.5f), g.b), c.o[2]);
        const float q = fmul(fadd(fadd(fmul(cx, cx), fmul(cy, cy)), fmul(cz, cz)), c.lod_s2);
        uint32_t lod = 0;
        while (lod < max_lod && q >= (float)(1u << (2u * (lod + 1u)))) ++lod;
        out_ids[pos] = id;
        out_lods[pos] = lod;
      }
      ++pos;
    }
    __syncthreads();
    if (tid == 0) base_s += tile_total;
    __syncthreads();
  }
  if (tid == 0) counts[blockIdx.x] = base_s;
}

}  // namespace

// Enqueues the request stage for ncams cameras on `stream` into device buffers: counts[ncams],
// ids / lods[ncams * cap] (camera i at i * cap). d_scratch must hold camera_scratch_bytes(...).
size_t camera_scratch_bytes(const Volume& v, uint32_t ncams) {
  const size_t words = ((size_t)v.n_bricks + 31) / 32;
  return ((sizeof(CamDev) * ncams + 255) & ~size_t(255)) + 4 * words * ncams;
}

vc_status launch_camera_requests(const Volume& v, const vc_camera* cams, uint32_t ncams, uint32_t max_lod,
                                 uint32_t cap, uint8_t* d_scratch, void* h_cams_pinned, uint32_t* d_counts,
                                 uint32_t* d_ids, uint32_t* d_lods, cudaStream_t stream) {
  const size_t words = ((size_t)v.n_bricks + 31) / 32;
  CamDev* hc = static_cast<CamDev*>(h_cams_pinned);
  uint32_t max_pix = 0;
  for (uint32_t i = 0; i < ncams; ++i) {
    camera_frame(cams[i], &hc[i]);
    max_pix = std::max(max_pix, cams[i].width * cams[i].height);
  }
  CamDev* dc = reinterpret_cast<CamDev*>(d_scratch);
  uint32_t* marks = reinterpret_cast<uint32_t*>(d_scratch + ((sizeof(CamDev) * ncams + 255) & ~size_t(255)));
  Grid g;
  for (int a = 0; a < 3; ++a) g.nb[a] = v.nb[a];
  g.b = (float)(1u << v.L);
  if (max_lod > v.L) max_lod = v.L;
  if (cudaMemcpyAsync(dc, hc, sizeof(CamDev) * ncams, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaMemsetAsync(marks, 0, 4 * words * ncams, stream) != cudaSuccess)
    return VC_ERR_CUDA;
  const uint32_t threads = 256;
  const uint32_t bx = std::min<uint32_t>((max_pix + threads - 1) / threads, 4096u);
  camera_march_kernel<<<dim3(bx, ncams), threads, 0, stream>>>(dc, v.d_flags, g, marks, (uint32_t)words);
  camera_compact_kernel<<<ncams, kCompactThreads, 0, stream>>>(dc, marks, (uint32_t)words, g, max_lod, cap, d_counts,
                                                               d_ids, d_lods);
  return cudaGetLastError() == cudaSuccess ? VC_OK : VC_ERR_CUDA;
}

vc_status launch_shared_marks(const Volume& v, const vc_camera* cams, uint32_t ncams, uint32_t* marks,
                              cudaStream_t stream) {
  Grid g;
  for (int a = 0; a < 3; ++a) g.nb[a] = v.nb[a];
  g.b = (float)(1u << v.L);
  for (uint32_t c0 = 0; c0 < ncams; c0 += kMarkCams) {
    const uint32_t nc = std::min(kMarkCams, ncams - c0);
    CamBlock B;
    std::memset(&B, 0, sizeof(B));
    uint32_t max_pix = 0;
    for (uint32_t i = 0; i < nc; ++i) {
      camera_frame(cams[c0 + i], &B.c[i]);
      max_pix = std::max(max_pix, cams[c0 + i].width * cams[c0 + i].height);
    }
    const uint32_t threads = 256;
    const uint32_t bx = std::min<uint32_t>((max_pix + threads - 1) / threads, std::max(1u, 4096u / nc));
    shared_march_kernel<<<dim3(bx, nc), threads, 0, stream>>>(B, v.d_flags, g, marks);
    if (cudaGetLastError() != cudaSuccess) return VC_ERR_CUDA;
  }
  return VC_OK;
}

}  // namespace vc

using namespace vc;

extern "C" vc_status vc_camera_bricks(vc_volume* vol, const vc_camera* cams, uint32_t ncams, uint32_t max_lod,
                                      uint32_t cap, uint32_t* counts, uint32_t* brick_ids, uint32_t* lods,
                                      void* cuda_stream) {
  Volume* v = reinterpret_cast<Volume*>(vol);
  if (!v || v->kind != kHandleVolume || !cams || !counts || (cap && (!brick_ids || !lods))) return VC_ERR_ARG;
  if (ncams == 0) return VC_OK;
  for (uint32_t i = 0; i < ncams; ++i)
    if (cams[i].width == 0 || cams[i].height == 0 || (uint64_t)cams[i].width * cams[i].height > 0xFFFFFFFFull)
      return VC_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != v->device) cudaSetDevice(v->device);
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  const size_t sb = camera_scratch_bytes(*v, ncams);
  const size_t ob = 4ull * ncams * (1 + 2ull * cap);
  uint8_t *scratch = nullptr, *out = nullptr;
  void* hc = nullptr;
  vc_status rc = VC_OK;
  if (cudaMallocAsync(reinterpret_cast<void**>(&scratch), sb, stream) != cudaSuccess ||
      cudaMallocAsync(reinterpret_cast<void**>(&out), ob, stream) != cudaSuccess ||
      cudaMallocHost(&hc, sizeof(CamDev) * ncams) != cudaSuccess) {
    cudaGetLastError();
    rc = VC_ERR_OOM;
  }
  uint32_t* d_counts = reinterpret_cast<uint32_t*>(out);
  uint32_t* d_ids = d_counts + ncams;
  uint32_t* d_lods = d_ids + (size_t)ncams * cap;
  if (rc == VC_OK)
    rc = launch_camera_requests(*v, cams, ncams, max_lod, cap, scratch, hc, d_counts, d_ids, d_lods, stream);
  if (rc == VC_OK) {
    std::vector<uint32_t> h(ob / 4);
    if (cudaMemcpyAsync(h.data(), out, ob, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
      rc = VC_ERR_CUDA;
    } else {
      std::memcpy(counts, h.data(), 4ull * ncams);
      if (cap) {
        std::memcpy(brick_ids, h.data() + ncams, 4ull * ncams * cap);
        std::memcpy(lods, h.data() + ncams + (size_t)ncams * cap, 4ull * ncams * cap);
      }
    }
  }
  if (scratch) cudaFreeAsync(scratch, stream);
  if (out) cudaFreeAsync(out, stream);
  if (hc) {
    cudaStreamSynchronize(stream);
    cudaFreeHost(hc);
  }
  if (prev >= 0 && prev != v->device) cudaSetDevice(prev);
  return rc;
}
