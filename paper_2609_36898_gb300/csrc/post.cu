// Post-processing of rendered frames (Methods, "Post-processing"): per-pixel accumulation of the
// rendered samples and a G-buffer of the most recent frame, an edge-avoiding À-trous filter run as
// a few passes over 3 x 3 pixels at distances 1, 2, 4, ..., and, in the same passes, the nearest
// rendered pixel of every pixel not rendered yet (jump-flood rule), whose filtered colour it takes.
// The contract is written in include/vc.h at vc_postprocess.
//
// State per pixel: the accumulated colour (3 floats) and sample count, the G-buffer (label, and a
// 16-bit code: normal in bits 0..2, quantised depth in bits 3..15), and two ping-pong slots of
// (filtered colour, offset to the nearest rendered pixel).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "vc_internal.h"

namespace vc {
namespace {

constexpr uint32_t kMaxMat = 256;
constexpr uint32_t kNoHit = 3u, kInvalid = 7u;
constexpr int32_t kNoOffset = 0x7FFF7FFF;  // (dx, dy) = (0x7FFF, 0x7FFF): no rendered pixel found yet

struct PostDev {
  uint32_t W, H, iterations, subsample, frame, reset;
  float d_near, d_scale;  // depth code = (t - d_near) * d_scale * 8191, clamped
  float vox_per_code;     // voxels per depth-code step
  float phi_rho, phi_d, exposure, inv_gamma;
  float hsv[kMaxMat][3];
  uint32_t n_mat;
};

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

__device__ __forceinline__ uint32_t material_of(uint32_t l, uint32_t n) {
  uint32_t h = l * 0x9E3779B1u;
  h ^= h >> 15;
  h *= 0x85EBCA77u;
  h ^= h >> 13;
  return h % n;
}

struct State {
  float4* accum;      // rgb sums, sample count
  uint32_t* glabel;
  uint32_t* gcode;
  float4* col[2];     // filtered rgb (w unused)
  int32_t* off[2];    // dx | dy << 16 (16-bit two's complement each), kNoOffset = none
};

__host__ __device__ inline State state_at(void* base, size_t n) {
  uint8_t* p = static_cast<uint8_t*>(base);
  State s;
  s.accum = reinterpret_cast<float4*>(p);
  p += 16 * n;
  s.col[0] = reinterpret_cast<float4*>(p);
  p += 16 * n;
  s.col[1] = reinterpret_cast<float4*>(p);
  p += 16 * n;
  s.glabel = reinterpret_cast<uint32_t*>(p);
  p += 4 * n;
  s.gcode = reinterpret_cast<uint32_t*>(p);
  p += 4 * n;
  s.off[0] = reinterpret_cast<int32_t*>(p);
  p += 4 * n;
  s.off[1] = reinterpret_cast<int32_t*>(p);
  return s;
}

// 1. this frame's samples into the accumulation and the G-buffer; the first colours and offsets
__global__ void post_accum_kernel(const __grid_constant__ PostDev P, State S, const uint32_t* __restrict__ labels,
                                  const float* __restrict__ depth, const uint8_t* __restrict__ face,
                                  const float* __restrict__ rgb) {
  const uint32_t n = P.W * P.H;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t px = i % P.W, py = i / P.W;
    float4 a = P.reset ? make_float4(0.0f, 0.0f, 0.0f, 0.0f) : S.accum[i];
    uint32_t code = P.reset ? kInvalid : S.gcode[i];
    uint32_t lab = P.reset ? 0u : S.glabel[i];
    if (subset_pixel(px, py, P.subsample, P.frame)) {
      a.x = fadd(a.x, rgb[3u * i]);
      a.y = fadd(a.y, rgb[3u * i + 1u]);
      a.z = fadd(a.z, rgb[3u * i + 2u]);
      a.w = fadd(a.w, 1.0f);
      lab = labels[i];
      const uint32_t f = face[i];
      if (lab == 0u || f == 0u) {
        code = kNoHit | (8191u << 3);
      } else {
        const uint32_t normal = ((f - 1u) >> 1) | ((f & 1u) << 2);
        float dn = fmul(fsub(depth[i], P.d_near), P.d_scale);
        dn = dn < 0.0f ? 0.0f : (dn > 1.0f ? 1.0f : dn);
        code = normal | ((uint32_t)fadd(fmul(dn, 8191.0f), 0.5f) << 3);
      }
    }
    S.accum[i] = a;
    S.gcode[i] = code;
    S.glabel[i] = lab;
    if ((code & 7u) != kInvalid) {
      const float inv = fdiv(1.0f, a.w);
      S.col[0][i] = make_float4(fmul(a.x, inv), fmul(a.y, inv), fmul(a.z, inv), 0.0f);
      S.off[0][i] = 0;
    } else {
      S.col[0][i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      S.off[0][i] = kNoOffset;
    }
  }
}

__device__ __forceinline__ int32_t off_dx(int32_t o) { return (int32_t)(int16_t)(o & 0xFFFF); }
__device__ __forceinline__ int32_t off_dy(int32_t o) { return o >> 16; }
__device__ __forceinline__ int32_t make_off(int32_t dx, int32_t dy) { return (dx & 0xFFFF) | (dy << 16); }

// 2. one pass at distance 2^it: rendered pixels filter, the others search the nearest rendered one
__global__ void __launch_bounds__(256) post_pass_kernel(const __grid_constant__ PostDev P, State S, uint32_t it) {
  __shared__ float hsv[kMaxMat][3];  // the materials' albedo in HSV
  for (uint32_t m = threadIdx.x; m < P.n_mat; m += blockDim.x) {
    hsv[m][0] = P.hsv[m][0];
    hsv[m][1] = P.hsv[m][1];
    hsv[m][2] = P.hsv[m][2];
  }
  __syncthreads();
  const uint32_t n = P.W * P.H;
  const uint32_t src = it & 1u, dst = src ^ 1u;
  const int32_t step = 1 << it;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t px = (int32_t)(i % P.W), py = (int32_t)(i / P.W);
    const uint32_t code = S.gcode[i];
    if ((code & 7u) != kInvalid) {
      const uint32_t lab = S.glabel[i];
      const float* hp = hsv[lab ? material_of(lab, P.n_mat) : 0u];
      const bool hit_p = (code & 7u) != kNoHit;
      const float dp = (float)(code >> 3);
      float sw = 0.0f, acc[3] = {0.0f, 0.0f, 0.0f};
      for (int32_t dy = -1; dy <= 1; ++dy)
        for (int32_t dx = -1; dx <= 1; ++dx) {
          const int32_t qx = px + dx * step, qy = py + dy * step;
          if (qx < 0 || qy < 0 || qx >= (int32_t)P.W || qy >= (int32_t)P.H) continue;
          const uint32_t j = (uint32_t)qy * P.W + (uint32_t)qx;
          const uint32_t cq = S.gcode[j];
          if ((cq & 7u) == kInvalid || (cq & 7u) != (code & 7u)) continue;  // not rendered / other normal
          const float h = (float)((dx == 0 ? 2 : 1) * (dy == 0 ? 2 : 1));
          float w = 1.0f;
          if (hit_p) {
            const uint32_t lq = S.glabel[j];
            const float* hq = hsv[lq ? material_of(lq, P.n_mat) : 0u];
            const float r0 = fmul(fsub(hp[0], hq[0]), P.phi_rho), r1 = fmul(fsub(hp[1], hq[1]), P.phi_rho),
                        r2 = fmul(fsub(hp[2], hq[2]), P.phi_rho);
            const float rr = fadd(fadd(fmul(r0, r0), fmul(r1, r1)), fmul(r2, r2));
            const float dd = fmul(fabsf(fsub(dp, (float)(cq >> 3))), P.vox_per_code);
            w = fmul(fdiv(1.0f, fadd(1.0f, rr)), expf(fmul(-P.phi_d, dd)));
          }
          const float hw = fmul(h, w);
          const float4 c = S.col[src][j];
          acc[0] = fadd(acc[0], fmul(hw, c.x));
          acc[1] = fadd(acc[1], fmul(hw, c.y));
          acc[2] = fadd(acc[2], fmul(hw, c.z));
          sw = fadd(sw, hw);
        }
      S.col[dst][i] = make_float4(fdiv(acc[0], sw), fdiv(acc[1], sw), fdiv(acc[2], sw), 0.0f);
      S.off[dst][i] = 0;
    } else {
      int32_t best = S.off[src][i];
      int64_t bl = best == kNoOffset ? INT64_MAX
                                     : (int64_t)off_dx(best) * off_dx(best) + (int64_t)off_dy(best) * off_dy(best);
      for (int32_t dy = -1; dy <= 1; ++dy)
        for (int32_t dx = -1; dx <= 1; ++dx) {
          const int32_t qx = px + dx * step, qy = py + dy * step;
          if ((dx == 0 && dy == 0) || qx < 0 || qy < 0 || qx >= (int32_t)P.W || qy >= (int32_t)P.H) continue;
          const int32_t oq = S.off[src][(uint32_t)qy * P.W + (uint32_t)qx];
          if (oq == kNoOffset) continue;
          const int32_t cx = off_dx(oq) + dx * step, cy = off_dy(oq) + dy * step;
          const int64_t l = (int64_t)cx * cx + (int64_t)cy * cy;
          if (l < bl) {
            bl = l;
            best = make_off(cx, cy);
          }
        }
      S.off[dst][i] = best;
      S.col[dst][i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
  }
}

__device__ __forceinline__ float aces(float x) {
  const float num = fmul(x, fadd(fmul(2.51f, x), 0.03f));
  const float den = fadd(fmul(x, fadd(fmul(2.43f, x), 0.59f)), 0.14f);
  float y = fdiv(num, den);
  return y < 0.0f ? 0.0f : (y > 1.0f ? 1.0f : y);
}

// 3. colours of the not-yet-rendered pixels from their nearest rendered pixel; tone map, gamma
__global__ void post_final_kernel(const __grid_constant__ PostDev P, State S, uint32_t fin,
                                  uint32_t* __restrict__ out) {
  const uint32_t n = P.W * P.H;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t px = (int32_t)(i % P.W), py = (int32_t)(i / P.W);
    float4 c = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if ((S.gcode[i] & 7u) != kInvalid) {
      c = S.col[fin][i];
    } else {
      const int32_t o = S.off[fin][i];
      if (o != kNoOffset) c = S.col[fin][(uint32_t)(py + off_dy(o)) * P.W + (uint32_t)(px + off_dx(o))];
    }
    const float v[3] = {c.x, c.y, c.z};
    uint32_t px8 = 0xFF000000u;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float y = aces(fmul(v[a], P.exposure));
      y = powf(y, P.inv_gamma);
      const uint32_t b = (uint32_t)fadd(fmul(y, 255.0f), 0.5f);
      px8 |= (b > 255u ? 255u : b) << (8 * a);
    }
    out[i] = px8;
  }
}

// HSV of an rgb albedo in [0, 1]^3 (hue in [0, 1)), double precision, rounded once.
void rgb_to_hsv(const float rgb[3], float hsv[3]) {
  const double r = rgb[0], g = rgb[1], b = rgb[2];
  const double mx = std::max(r, std::max(g, b)), mn = std::min(r, std::min(g, b)), c = mx - mn;
  double h = 0.0;
  if (c > 0.0) {
    if (mx == r) h = std::fmod((g - b) / c + 6.0, 6.0);
    else if (mx == g) h = (b - r) / c + 2.0;
    else h = (r - g) / c + 4.0;
    h /= 6.0;
  }
  hsv[0] = (float)h;
  hsv[1] = (float)(mx > 0.0 ? c / mx : 0.0);
  hsv[2] = (float)mx;
}

}  // namespace
}  // namespace vc

using namespace vc;

extern "C" size_t vc_post_state_bytes(uint32_t width, uint32_t height) {
  return (size_t)width * height * (16u * 3u + 4u * 4u);
}

extern "C" vc_status vc_postprocess(vc_volume* vol, const vc_post_params* params, const uint32_t* labels,
                                    const float* depth, const uint8_t* face, const float* rgb, void* state,
                                    uint32_t* rgba_out, void* cuda_stream) {
  Volume* v = reinterpret_cast<Volume*>(vol);
  if (!v || v->kind != kHandleVolume || !params || !labels || !depth || !face || !rgb || !state || !rgba_out)
    return VC_ERR_ARG;
  const vc_post_params& Q = *params;
  if (!Q.width || !Q.height || (uint64_t)Q.width * Q.height > 0x7FFFFFFFull || Q.width > 32767 || Q.height > 32767 ||
      Q.iterations > 10 || !(Q.subsample <= 2u || Q.subsample == 4u || Q.subsample == 8u) || Q.n_materials == 0 ||
      Q.n_materials > kMaxMat || !Q.materials || !(Q.gamma > 0.0f) || (reinterpret_cast<uintptr_t>(state) & 15u))
    return VC_ERR_ARG;
  static_assert(sizeof(PostDev) < 32000, "kernel parameter space");
  PostDev P;
  std::memset(&P, 0, sizeof(P));
  P.W = Q.width;
  P.H = Q.height;
  P.iterations = Q.iterations;
  P.subsample = Q.subsample;
  P.frame = Q.frame;
  P.reset = Q.reset ? 1u : 0u;
  // the dataset's bounding sphere: centre dims / 2, radius |dims| / 2; depth 0 at its near side
  double c[3], R2 = 0.0, D2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    c[a] = 0.5 * v->dims[a];
    R2 += c[a] * c[a];
    D2 += (Q.cam_pos[a] - c[a]) * (Q.cam_pos[a] - c[a]);
  }
  const double R = std::sqrt(R2);
  P.d_near = (float)(std::sqrt(D2) - R);
  P.d_scale = (float)(1.0 / (2.0 * R));
  P.vox_per_code = (float)(2.0 * R / 8191.0);
  P.phi_rho = Q.phi_rho;
  P.phi_d = Q.phi_d;
  P.exposure = Q.exposure;
  P.inv_gamma = (float)(1.0 / (double)Q.gamma);
  P.n_mat = Q.n_materials;
  for (uint32_t m = 0; m < Q.n_materials; ++m) rgb_to_hsv(Q.materials[m].rgb, P.hsv[m]);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the parameter block travels with each launch (kernel parameter space): no staging copy, no wait
  const size_t n = (size_t)P.W * P.H;
  const State S = state_at(state, n);
  const uint32_t blocks = (uint32_t)std::min<size_t>((n + 255) / 256, (size_t)std::max(1u, v->sms) * 16u);
  post_accum_kernel<<<blocks, 256, 0, st>>>(P, S, labels, depth, face, rgb);
  for (uint32_t it = 0; it < P.iterations; ++it) post_pass_kernel<<<blocks, 256, 0, st>>>(P, S, it);
  post_final_kernel<<<blocks, 256, 0, st>>>(P, S, P.iterations & 1u, rgba_out);
  if (cudaGetLastError() != cudaSuccess) return VC_ERR_CUDA;
  v->launches += 2u + P.iterations;
  return VC_OK;
}
