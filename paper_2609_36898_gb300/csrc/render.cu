// Rendering from decoded bricks: one thread per pixel ray marches the voxels front to back (Methods,
// "Volcanite rendering": "Shading Modes", "Transparency", "Ray marching", "Random number
// generation"). The contract (materials, shading modes, outputs) is written in include/vc.h at
// vc_render; this file holds the kernel.
//
// Traversal. A position is an integer voxel index v plus a sub-voxel position p in [0, 1)^3, the
// paper's numerically stable DDA: distances to the next faces are computed from p alone, so they do
// not lose precision far from the origin. Inside a brick decoded at level of detail k (or crossed
// whole when it shows nothing, or seen as its coarsest label when it is not decoded) the ray
// steps through cells of edge S = 2^k: the position is taken to the coarse cell (v >> k, and
// ((v mod S) + p) / S), one step is made there, and the result is taken back to voxel units
// (v = c S + floor(q S), p = q S - floor(q S)); scaling by a power of two is exact in float, so
// the step loses nothing to the change of units. The step itself: per axis the ray distance to
// the cell's face ahead is ((1 if d > 0 else 0) - q) / d; the smallest (ties to x, then y) wins;
// the other axes advance by that distance times d (clamped into [0, 1)), the winning axis enters
// the next cell at its near face. The paper prints this as GLSL (its update line for the other
// axes is garbled in the text: this file takes the geometric update written here).
//
// Every float step is one correctly rounded operation (explicit _rn intrinsics, no contraction) in
// a fixed order, so the result is a pure function of the inputs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "vc_internal.h"

namespace vc {
namespace {

constexpr uint32_t kMaxMaterials = 256;
constexpr float kOneMinus = 0.99999994f;  // the largest float below 1
constexpr uint64_t kNotDecoded = ~0ull;

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float clamp01(float x) { return x < 0.0f ? 0.0f : (x > kOneMinus ? kOneMinus : x); }

struct RenderDev {
  CamDev cam;
  uint32_t subsample;
  float light[3];  // unit length, towards the light
  float ambient, ao_radius, sky;
  uint32_t mode, frame, jitter, max_bounces, n_mat;
  uint32_t dims[3], nb[3], L;
  float mat[kMaxMaterials][4];  // rgb albedo, opacity
};

struct Inputs {
  const uint64_t* offsets;
  const uint8_t* lods;
  const uint32_t* cache;
  const uint8_t* flags;     // per brick: bit 1 = palette holds a label other than 0
  const uint32_t* starts;   // encoding: Brick Starts (words)
  const uint32_t* records;  // encoding: records
  uint32_t coder, vflags;   // the volume's coder and header flags (rANS runs)
  uint32_t* marks;          // visibility bits (one per brick) set by rays of depth <= request_depth, or null
  uint32_t request_depth;
};

// Jarzynski and Olano's PCG2D integer hash (Hash Functions for GPU Rendering, 2020).
__device__ __forceinline__ void pcg2d(uint32_t& x, uint32_t& y) {
  x = x * 1664525u + 1013904223u;
  y = y * 1664525u + 1013904223u;
  x += y * 1664525u;
  y += x * 1664525u;
  x ^= x >> 16;
  y ^= y >> 16;
  x += y * 1664525u;
  y += x * 1664525u;
  x ^= x >> 16;
  y ^= y >> 16;
}
__device__ __forceinline__ float unit_float(uint32_t h) { return (float)(h >> 8) * 5.9604645e-8f; }  // [0, 1), 2^-24 steps

// Random stream of one pixel: state (x, y), advanced by one PCG2D per draw of two numbers.
struct Rng {
  uint32_t x, y;
  __device__ void next2(float& a, float& b) {
    pcg2d(x, y);
    a = unit_float(x);
    b = unit_float(y);
  }
};

// Material of label l != 0: index hash(l) mod n.
__device__ __forceinline__ uint32_t material_of(uint32_t l, uint32_t n) {
  uint32_t h = l * 0x9E3779B1u;
  h ^= h >> 15;
  h *= 0x85EBCA77u;
  h ^= h >> 13;
  return h % n;
}

struct RayState {
  int32_t v[3];
  float p[3], d[3];
  float t;
  uint32_t face;  // entered face of the current voxel (0 = none)
};

// Marks brick id as visible (Methods, "GPU rendering pipeline": rays mark the bricks they
// access), once per brick entered: `last` is the ray's previously marked brick.
__device__ __forceinline__ void mark_brick(uint32_t* marks, uint32_t id, uint32_t& last) {
  if (!marks || id == last) return;
  last = id;
  const uint32_t bit = 1u << (id & 31u);
  if (!(marks[id >> 5] & bit)) atomicOr(&marks[id >> 5], bit);
}

// Label and cell size (log2) of the cell containing voxel v; bricks holding a visible label are
// marked in `marks` (null: no marking).
__device__ __forceinline__ uint32_t cell_at(const RenderDev& R, const Inputs& in, const int32_t v[3], uint32_t* s_log,
                                            uint32_t* marks, uint32_t& last) {
  const uint32_t L = R.L, b = 1u << L;
  const uint32_t id = ((uint32_t)v[0] >> L) + R.nb[0] * (((uint32_t)v[1] >> L) + R.nb[1] * ((uint32_t)v[2] >> L));
  if (!(in.flags[id] & 2u)) {  // nothing but background: cross the brick in one step
    *s_log = L;
    return 0u;
  }
  mark_brick(marks, id, last);
  const uint64_t off = in.offsets[id];
  if (off == kNotDecoded) {  // the coarsest label, straight from the encoding
    *s_log = L;
    const uint32_t* rec = in.records + in.starts[id];
    const uint32_t S = rec[1];
    const uint32_t ns = in.coder == 1 ? head_words(S, runs_k(in.vflags)) : 0u;
    return rec[0] ? rec[4 + ns] : 0u;
  }
  const uint32_t k = in.lods[id];
  *s_log = k;
  const uint32_t e = b >> k;
  const uint32_t cx = ((uint32_t)v[0] & (b - 1u)) >> k, cy = ((uint32_t)v[1] & (b - 1u)) >> k,
                 cz = ((uint32_t)v[2] & (b - 1u)) >> k;
  return in.cache[off + (uint64_t)((cz * e + cy) * e + cx)];
}

// One step of the stable DDA in cells of edge 2^s_log; false when the ray leaves the volume.
__device__ bool dda_step(const RenderDev& R, RayState& r, uint32_t s_log) {
  const int32_t S = 1 << s_log;
  const float fS = (float)S, inv = fdiv(1.0f, fS);  // powers of two: exact
  int32_t c[3];
  float q[3], dist[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    c[a] = r.v[a] >> s_log;
    q[a] = fmul(fadd((float)(r.v[a] & (S - 1)), r.p[a]), inv);
    if (r.d[a] > 0.0f) dist[a] = fdiv(fsub(1.0f, q[a]), r.d[a]);
    else if (r.d[a] < 0.0f) dist[a] = fdiv(fsub(0.0f, q[a]), r.d[a]);
    else dist[a] = INFINITY;
  }
  int ax = 0;
  if (dist[1] < dist[ax]) ax = 1;
  if (dist[2] < dist[ax]) ax = 2;
  const float tt = dist[ax];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a != ax) q[a] = clamp01(fadd(q[a], fmul(tt, r.d[a])));
  if (r.d[ax] > 0.0f) {
    c[ax] += 1;
    q[ax] = 0.0f;
    r.face = 2u * (uint32_t)ax + 1u;  // entered through the cell's -axis side
  } else {
    c[ax] -= 1;
    q[ax] = kOneMinus;
    r.face = 2u * (uint32_t)ax + 2u;
  }
  r.t = fadd(r.t, fmul(tt, fS));
  bool inside = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float w = fmul(q[a], fS);
    const float fl = floorf(w);
    r.v[a] = c[a] * S + (int32_t)fl;
    r.p[a] = fsub(w, fl);
    inside = inside && r.v[a] >= 0 && r.v[a] < (int32_t)R.dims[a];
  }
  return inside;
}

// Materials (rgb albedo, opacity), copied into shared memory by each block.
__device__ __forceinline__ bool opaque(const float4* mat, uint32_t n_mat, uint32_t l) {
  return l != 0u && mat[material_of(l, n_mat)].w >= 1.0f;
}

// Marches from r until an opaque voxel (true, its label in *hit) or the volume's end / max_t;
// marks the bricks it accesses in `marks` (null: none).
__device__ bool march_opaque(const RenderDev& R, const Inputs& in, const float4* mat, RayState& r, float max_t,
                             uint32_t* hit, uint32_t* marks) {
  const uint32_t max_steps = 3u * (R.dims[0] + R.dims[1] + R.dims[2]) + 64u;
  uint32_t last = ~0u;
  for (uint32_t step = 0; step < max_steps; ++step) {
    uint32_t s;
    const uint32_t l = cell_at(R, in, r.v, &s, marks, last);
    if (opaque(mat, R.n_mat, l)) {
      *hit = l;
      return true;
    }
    if (!dda_step(R, r, s) || r.t > max_t) return false;
  }
  return false;
}

// The normal of an entered face (pointing back out of the voxel).
__device__ __forceinline__ void face_normal(uint32_t face, float n[3]) {
  n[0] = n[1] = n[2] = 0.0f;
  if (face) n[(face - 1u) >> 1] = (face & 1u) ? -1.0f : 1.0f;
}

// A secondary ray leaving the entered face of voxel v: it starts in the neighbour across that face.
__device__ __forceinline__ RayState from_face(const RayState& h, const float dir[3]) {
  RayState r;
  const int ax = (int)((h.face - 1u) >> 1);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r.v[a] = h.v[a];
    r.p[a] = h.p[a];
    r.d[a] = dir[a];
  }
  if (h.face & 1u) {  // entered through the -axis side: the neighbour is at -1, at its +side face
    r.v[ax] -= 1;
    r.p[ax] = kOneMinus;
  } else {
    r.v[ax] += 1;
    r.p[ax] = 0.0f;
  }
  r.t = 0.0f;
  r.face = 0u;
  return r;
}

__device__ __forceinline__ float dot3(const float a[3], const float b[3]) {
  return fadd(fadd(fmul(a[0], b[0]), fmul(a[1], b[1])), fmul(a[2], b[2]));
}

// A cosine-weighted random direction around unit n: n plus a uniform point of the unit sphere
// (a uniform point of the unit ball by rejection, at most 16 tries, scaled to the sphere),
// normalised; n itself if that sum vanishes or every try is rejected.
__device__ void cosine_dir(Rng& g, const float n[3], float out[3]) {
  float v[3] = {0.0f, 0.0f, 0.0f}, r2 = 0.0f;
  bool ok = false;
  for (int k = 0; k < 16 && !ok; ++k) {
    float a, b, c, unused;
    g.next2(a, b);
    g.next2(c, unused);
    v[0] = fsub(fmul(2.0f, a), 1.0f);
    v[1] = fsub(fmul(2.0f, b), 1.0f);
    v[2] = fsub(fmul(2.0f, c), 1.0f);
    r2 = dot3(v, v);
    ok = r2 > 0.0f && r2 <= 1.0f;
  }
  if (ok) {
    const float len = __fsqrt_rn(r2);
    float w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) w[a] = fadd(n[a], fdiv(v[a], len));
    const float w2 = dot3(w, w);
    if (w2 > 1e-12f) {
      const float wl = __fsqrt_rn(w2);
#pragma unroll
      for (int a = 0; a < 3; ++a) out[a] = fdiv(w[a], wl);
      return;
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) out[a] = n[a];
}

__global__ void __launch_bounds__(128) render_kernel(const __grid_constant__ RenderDev R, Inputs in,
                                                     uint32_t* labels_out, float* depth_out, uint8_t* face_out,
                                                     float* rgb_out) {
  __shared__ float4 mat[kMaxMaterials];
  for (uint32_t m = threadIdx.x; m < R.n_mat; m += blockDim.x)
    mat[m] = make_float4(R.mat[m][0], R.mat[m][1], R.mat[m][2], R.mat[m][3]);
  __syncthreads();
  const CamDev& c = R.cam;
  // rays of path depth <= request_depth mark the bricks they access: the primary ray is depth 0,
  // shadow, ambient occlusion and the first path-tracing bounce depth 1, bounce k depth k
  auto marks_at = [&](uint32_t depth) -> uint32_t* { return depth <= in.request_depth ? in.marks : nullptr; };
  const uint32_t npix = c.W * c.H;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x) {
    const uint32_t px = i % c.W, py = i / c.W;
    if (!subset_pixel(px, py, R.subsample, R.frame)) continue;
    // primary ray through the pixel centre, or a jittered sub-pixel position (temporal
    // anti-aliasing: offsets from the sum of three uniforms, a bell shape on (-1, 1) standing in
    // for the Blackman-Harris window)
    float jx = 0.0f, jy = 0.0f;
    if (R.jitter) {
      Rng gj{R.frame, 0xA511E9B3u};
      float u0, u1, u2, u3, u4, u5;
      gj.next2(u0, u1);
      gj.next2(u2, u3);
      gj.next2(u4, u5);
      jx = fmul(fsub(fadd(fadd(u0, u1), u2), 1.5f), 0.6666667f);
      jy = fmul(fsub(fadd(fadd(u3, u4), u5), 1.5f), 0.6666667f);
    }
    const float sx = fmul(fsub(fmul(fadd(fadd((float)px, 0.5f), jx), c.inv_w2), 1.0f), c.sxs);
    const float sy = fmul(fsub(1.0f, fmul(fadd(fadd((float)py, 0.5f), jy), c.inv_h2)), c.sys);
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = fadd(fadd(c.f[a], fmul(sx, c.r[a])), fmul(sy, c.u[a]));
    const float dl = __fsqrt_rn(dot3(d, d));
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = fdiv(d[a], dl);
    // entry into the volume's box [0, dims)
    float t0 = 0.0f, t1 = INFINITY;
    int entry_ax = -1;
    bool miss = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float n = (float)R.dims[a];
      if (d[a] == 0.0f) {
        if (c.o[a] < 0.0f || c.o[a] >= n) miss = true;
        continue;
      }
      float ta = fdiv(fsub(0.0f, c.o[a]), d[a]), tb = fdiv(fsub(n, c.o[a]), d[a]);
      if (ta > tb) {
        const float x = ta;
        ta = tb;
        tb = x;
      }
      if (ta > t0) {
        t0 = ta;
        entry_ax = a;
      }
      if (tb < t1) t1 = tb;
    }
    uint32_t out_label = 0u, out_face = 0u;
    float out_depth = INFINITY, rgb[3] = {0.0f, 0.0f, 0.0f};
    Rng g{px ^ (R.frame * 0x9E3779B9u), py + (R.frame << 16)};
    pcg2d(g.x, g.y);
    if (!miss && t0 < t1) {
      RayState r;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        r.d[a] = d[a];
        const float pa = fadd(c.o[a], fmul(t0, d[a]));
        float fc = floorf(pa);
        if (fc < 0.0f) fc = 0.0f;
        if (fc > (float)(R.dims[a] - 1u)) fc = (float)(R.dims[a] - 1u);
        r.v[a] = (int32_t)fc;
        r.p[a] = clamp01(fsub(pa, fc));
      }
      r.t = t0;
      r.face = entry_ax < 0 ? 0u : 2u * (uint32_t)entry_ax + (d[entry_ax] > 0.0f ? 1u : 2u);
      // front to back: semi-transparent materials composite, the first opaque one is the hit
      float T = 1.0f;
      uint32_t prev = 0u;
      bool hit = false;
      const uint32_t max_steps = 3u * (R.dims[0] + R.dims[1] + R.dims[2]) + 64u;
      uint32_t* const mk0 = marks_at(0);
      uint32_t last = ~0u;
      for (uint32_t step = 0; step < max_steps && T >= 0.00390625f; ++step) {
        uint32_t s;
        const uint32_t l = cell_at(R, in, r.v, &s, mk0, last);
        if (l != prev && l != 0u) {
          const float4 mm = mat[material_of(l, R.n_mat)];
          const float m[4] = {mm.x, mm.y, mm.z, mm.w};
          if (m[3] > 0.0f) {
            float n[3];
            face_normal(r.face, n);
            if (!r.face) {  // the camera is inside this voxel: light it from the viewer's side
#pragma unroll
              for (int a = 0; a < 3; ++a) n[a] = fsub(0.0f, d[a]);
            }
            if (m[3] >= 1.0f) {
              hit = true;
              out_label = l;
              out_depth = r.t;
              out_face = r.face;
              break;
            }
            float nl = dot3(n, R.light);
            if (nl < 0.0f) nl = 0.0f;
            const float shade = fadd(R.ambient, fmul(fsub(1.0f, R.ambient), nl));
            const float w = fmul(T, m[3]);
#pragma unroll
            for (int a = 0; a < 3; ++a) rgb[a] = fadd(rgb[a], fmul(w, fmul(m[a], shade)));
            T = fmul(T, fsub(1.0f, m[3]));
          }
        }
        prev = l;
        if (!dda_step(R, r, s)) break;
      }
      if (hit) {
        const float4 mm = mat[material_of(out_label, R.n_mat)];
        const float m[3] = {mm.x, mm.y, mm.z};
        float n[3];
        face_normal(r.face, n);
        if (!r.face) {
#pragma unroll
          for (int a = 0; a < 3; ++a) n[a] = fsub(0.0f, d[a]);
        }
        float c3[3] = {0.0f, 0.0f, 0.0f};
        if (R.mode == VC_SHADE_LOCAL || R.mode == VC_SHADE_SHADOW) {
          float nl = dot3(n, R.light);
          if (nl < 0.0f) nl = 0.0f;
          if (R.mode == VC_SHADE_SHADOW && nl > 0.0f && r.face) {
            RayState sr = from_face(r, R.light);
            uint32_t l2;
            if (sr.v[0] >= 0 && sr.v[0] < (int32_t)R.dims[0] && sr.v[1] >= 0 && sr.v[1] < (int32_t)R.dims[1] &&
                sr.v[2] >= 0 && sr.v[2] < (int32_t)R.dims[2] && march_opaque(R, in, mat, sr, INFINITY, &l2, marks_at(1)))
              nl = 0.0f;
          }
          const float shade = fadd(R.ambient, fmul(fsub(1.0f, R.ambient), nl));
#pragma unroll
          for (int a = 0; a < 3; ++a) c3[a] = fmul(m[a], shade);
        } else if (R.mode == VC_SHADE_AO) {
          float dir[3];
          cosine_dir(g, n, dir);
          bool occluded = false;
          if (r.face) {
            RayState ar = from_face(r, dir);
            uint32_t l2;
            occluded = ar.v[0] >= 0 && ar.v[0] < (int32_t)R.dims[0] && ar.v[1] >= 0 && ar.v[1] < (int32_t)R.dims[1] &&
                       ar.v[2] >= 0 && ar.v[2] < (int32_t)R.dims[2] &&
                       march_opaque(R, in, mat, ar, R.ao_radius, &l2, marks_at(1));
          }
#pragma unroll
          for (int a = 0; a < 3; ++a) c3[a] = occluded ? 0.0f : fmul(m[a], R.sky);
        } else {  // path tracing
          float tp[3] = {m[0], m[1], m[2]};
          RayState h = r;
          for (uint32_t bounce = 1; bounce <= R.max_bounces && h.face; ++bounce) {
            float nn[3], dir[3];
            face_normal(h.face, nn);
            cosine_dir(g, nn, dir);
            RayState br = from_face(h, dir);
            uint32_t l2 = 0u;
            const bool inside = br.v[0] >= 0 && br.v[0] < (int32_t)R.dims[0] && br.v[1] >= 0 &&
                                br.v[1] < (int32_t)R.dims[1] && br.v[2] >= 0 && br.v[2] < (int32_t)R.dims[2];
            if (!inside || !march_opaque(R, in, mat, br, INFINITY, &l2, marks_at(bounce))) {
#pragma unroll
              for (int a = 0; a < 3; ++a) c3[a] = fadd(c3[a], fmul(tp[a], R.sky));
              break;
            }
            const float4 m2 = mat[material_of(l2, R.n_mat)];
            tp[0] = fmul(tp[0], m2.x);
            tp[1] = fmul(tp[1], m2.y);
            tp[2] = fmul(tp[2], m2.z);
            if (bounce >= 4u) {  // Russian roulette
              float q = tp[0] > tp[1] ? tp[0] : tp[1];
              if (tp[2] > q) q = tp[2];
              if (q > 1.0f) q = 1.0f;
              float u, unused;
              g.next2(u, unused);
              if (!(u < q)) break;
#pragma unroll
              for (int a = 0; a < 3; ++a) tp[a] = fdiv(tp[a], q);
            }
            h = br;
          }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) rgb[a] = fadd(rgb[a], fmul(T, c3[a]));
      }
    }
    if (labels_out) labels_out[i] = out_label;
    if (depth_out) depth_out[i] = out_depth;
    if (face_out) face_out[i] = (uint8_t)out_face;
    if (rgb_out) {
      rgb_out[3u * i] = rgb[0];
      rgb_out[3u * i + 1u] = rgb[1];
      rgb_out[3u * i + 2u] = rgb[2];
    }
  }
}

}  // namespace
}  // namespace vc

using namespace vc;

extern "C" vc_status vc_render(vc_volume* vol, const uint64_t* brick_offsets, const uint8_t* brick_lods,
                               const uint32_t* cache, const vc_camera* cam, const vc_render_params* params,
                               uint32_t* labels_out, float* depth_out, uint8_t* face_out, float* rgb_out,
                               void* cuda_stream) {
  Volume* v = reinterpret_cast<Volume*>(vol);
  if (!v || v->kind != kHandleVolume || !brick_offsets || !brick_lods || !cache || !cam || !params) return VC_ERR_ARG;
  const vc_render_params& P = *params;
  if (cam->width == 0 || cam->height == 0 || (uint64_t)cam->width * cam->height > 0x7FFFFFFFull) return VC_ERR_ARG;
  if (P.mode > VC_SHADE_PATH || P.n_materials == 0 || P.n_materials > kMaxMaterials || !P.materials ||
      (P.mode == VC_SHADE_PATH && (P.max_bounces == 0 || P.max_bounces > 32)) ||
      (P.mode == VC_SHADE_AO && !(P.ao_radius > 0.0f)) ||
      !(P.subsample <= 2u || P.subsample == 4u || P.subsample == 8u))
    return VC_ERR_ARG;
  const double l2 = (double)P.light_dir[0] * P.light_dir[0] + (double)P.light_dir[1] * P.light_dir[1] +
                    (double)P.light_dir[2] * P.light_dir[2];
  if (!(l2 > 0.0)) return VC_ERR_ARG;
  static_assert(sizeof(RenderDev) < 32000, "kernel parameter space");
  RenderDev R;
  std::memset(&R, 0, sizeof(R));
  camera_frame(*cam, &R.cam);
  const double ll = std::sqrt(l2);
  for (int a = 0; a < 3; ++a) R.light[a] = (float)(P.light_dir[a] / ll);
  R.ambient = P.ambient;
  R.ao_radius = P.ao_radius;
  R.sky = P.sky;
  R.mode = P.mode;
  R.frame = P.frame;
  R.jitter = P.jitter ? 1u : 0u;
  R.max_bounces = P.max_bounces;
  R.n_mat = P.n_materials;
  R.subsample = P.subsample;
  for (uint32_t m = 0; m < P.n_materials; ++m) {
    for (int a = 0; a < 3; ++a) R.mat[m][a] = P.materials[m].rgb[a];
    R.mat[m][3] = P.materials[m].opacity;
  }
  R.L = v->L;
  for (int a = 0; a < 3; ++a) {
    R.dims[a] = v->dims[a];
    R.nb[a] = v->nb[a];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  Inputs in;
  in.offsets = brick_offsets;
  in.lods = brick_lods;
  in.cache = cache;
  in.flags = v->d_flags;
  in.starts = v->dv.starts;
  in.records = v->dv.records;
  in.coder = v->coder;
  in.vflags = v->flags;
  in.marks = P.marks;
  in.request_depth = P.request_depth;
  // the parameter block travels with the launch (kernel parameter space): no staging copy, no wait
  const uint32_t npix = cam->width * cam->height;
  const uint32_t blocks = std::min<uint32_t>((npix + 127u) / 128u, std::max(1u, v->sms) * 16u);
  render_kernel<<<blocks, 128, 0, st>>>(R, in, labels_out, depth_out, face_out, rgb_out);
  if (cudaGetLastError() != cudaSuccess) return VC_ERR_CUDA;
  ++v->launches;
  return VC_OK;
}
