/*
 * Rendering oracle: what each pixel ray of a pinhole camera sees in a volume whose bricks are given
 * at chosen levels of detail. TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's
 * CPU legs); it shares no code with the GPU library.
 *
 * Paper, Methods "Volcanite rendering": rays march the voxels of the volume front to back
 * ("Ray marching": an integer voxel index plus a sub-voxel position in [0, 1) per axis, so that
 * face distances are computed in [0, 1) and stay precise; in a brick decoded at level of detail k
 * the ray steps through cells of edge 2^k by taking the position to the coarse cell, stepping,
 * and taking it back); "Transparency": entering a semi-transparent material adds its Lambertian
 * local shading times its opacity and lowers the throughput by that opacity; "Shading Modes":
 * local shading, one shadow ray towards the light, one ambient-occlusion ray in a random
 * direction, or path tracing with Russian roulette and at most 32 bounces; "Random number
 * generation": PCG2D seeded per pixel and frame. Readings taken here, one per point the paper
 * leaves open (the same in the library):
 *   - label 0 is background; label l != 0 has material hash(l) mod n_materials, a material is
 *     (albedo rgb, opacity); opacity 0 hides the label, opacity 1 makes it a surface;
 *   - a brick whose palette has no label other than 0 is crossed in one step of edge b; a brick
 *     not decoded is one cell holding its first palette entry (its coarsest level of detail);
 *   - the step: per axis the distance to the cell face ahead is ((1 if d > 0 else 0) - q) / d
 *     (q the position in cell units), the smallest wins (ties to x, then y), the other axes
 *     advance by it (clamped into [0, 1)), the winning axis enters the next cell at its near face
 *     (the paper's update line for the other axes is garbled in its listing);
 *   - shadow, occlusion and path rays leave the hit voxel through the face the primary ray entered
 *     (they start in the neighbour across it), stop only at opaque voxels; ambient occlusion counts
 *     occluders within ao_radius voxels; path tracing takes cosine-weighted Lambertian bounces
 *     (a uniform point of the unit sphere added to the normal, normalised; sphere points by
 *     rejection in the unit ball, at most 16 tries), sky radiance when a path leaves the volume,
 *     roulette from the fourth bounce with the largest throughput component as survival chance;
 *   - temporal anti-aliasing jitter: per frame one sub-pixel offset per axis, (u1 + u2 + u3 -
 *     3/2) 2/3 (a bell shape on (-1, 1) standing in for the Blackman-Harris window).
 * Every float step below is one IEEE single operation in the order written (compile without
 * floating-point contraction): a GPU implementation taking the same steps gives the same bits.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  float o[3], f[3], r[3], u[3];
  float sxs, sys, inv_w2, inv_h2, lod_s2;
} cam_frame;

int oracle_palette_flags(const uint8_t* vol, size_t size, uint32_t nb[3], uint32_t* L_out, uint8_t** flags_out);
uint32_t oracle_head_words(uint32_t coder, uint32_t flags, uint32_t S);
void oracle_camera_frame(const float pos[3], const float dir[3], const float up[3], float fov_y, uint32_t W,
                         uint32_t H, cam_frame* c);

typedef struct {
  uint32_t mode;  /* 0 local, 1 shadow, 2 ambient occlusion, 3 path tracing */
  uint32_t frame, jitter, max_bounces;
  float light_dir[3];
  float ambient, ao_radius, sky;
  uint32_t n_materials;
  const float* materials; /* n_materials x (r, g, b, opacity) */
  uint32_t subsample;     /* 0/1 every pixel; 2, 4, 8: one pixel of each s x s block per frame */
  uint8_t* visible;       /* per brick, or NULL: set to 1 for every brick holding a label other than 0
                             that a ray of path depth <= request_depth enters (Methods, "GPU rendering
                             pipeline": rays mark the bricks they access; "Brick request limitation":
                             a ray depth limit for requests). Depth 0 = the primary ray; shadow, ambient
                             occlusion rays and the first path-tracing bounce 1; bounce k k. */
  uint32_t request_depth;
} oracle_render_params;

/* Stratified subsets (Methods, "Upsampling": one pixel of each s^2 block per frame, every pixel
 * of the block within s^2 frames; block sequences displaced by a fixed integer hash of the block,
 * standing in for the paper's blue-noise displacement). */
int oracle_subset_pixel(uint32_t px, uint32_t py, uint32_t s, uint32_t f) {
  if (s <= 1u) return 1;
  uint32_t h = (px / s) * 0x8DA6B343u ^ (py / s) * 0xD8163841u;
  h ^= h >> 13;
  h *= 0x85EBCA6Bu;
  h ^= h >> 16;
  return (px % s) + s * (py % s) == (f + h) % (s * s);
}

#define R_ONE_MINUS 0.99999994f
#define R_NOT_DECODED (~0ull)

typedef struct {
  uint32_t dims[3], nb[3], L, coder, vflags;
  const uint8_t* vol;
  const uint32_t* starts; /* not 4-byte aligned in general: read through rd32 */
  size_t rec_off;
  const uint8_t* flags;
  const uint64_t* offsets;
  const uint8_t* lods;
  const uint32_t* cache;
  float light[3], ambient, ao_radius, sky;
  uint32_t mode, max_bounces, n_mat;
  const float* mat;
  uint8_t* visible;
  uint32_t request_depth;
} rctx;

static uint32_t rd32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

/* Jarzynski and Olano's PCG2D integer hash, restated. */
static void pcg2d(uint32_t* x, uint32_t* y) {
  *x = *x * 1664525u + 1013904223u;
  *y = *y * 1664525u + 1013904223u;
  *x += *y * 1664525u;
  *y += *x * 1664525u;
  *x ^= *x >> 16;
  *y ^= *y >> 16;
  *x += *y * 1664525u;
  *y += *x * 1664525u;
  *x ^= *x >> 16;
  *y ^= *y >> 16;
}
static float unit_float(uint32_t h) { return (float)(h >> 8) * 5.9604645e-8f; }
static void next2(uint32_t st[2], float* a, float* b) {
  pcg2d(&st[0], &st[1]);
  *a = unit_float(st[0]);
  *b = unit_float(st[1]);
}

static uint32_t material_of(uint32_t l, uint32_t n) {
  uint32_t h = l * 0x9E3779B1u;
  h ^= h >> 15;
  h *= 0x85EBCA77u;
  h ^= h >> 13;
  return h % n;
}
static const float* mat_of(const rctx* C, uint32_t l) { return C->mat + 4 * (size_t)material_of(l, C->n_mat); }
static int opaque(const rctx* C, uint32_t l) { return l != 0u && mat_of(C, l)[3] >= 1.0f; }

static float clamp01(float x) { return x < 0.0f ? 0.0f : (x > R_ONE_MINUS ? R_ONE_MINUS : x); }
static float dot3(const float a[3], const float b[3]) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

typedef struct {
  int32_t v[3];
  float p[3], d[3], t;
  uint32_t face; /* 1..6: entered through the -x, +x, -y, +y, -z, +z side; 0 none */
} ray;

/* Label of the cell holding voxel v, and the cell's edge as a power of two; a ray of path depth
 * `depth` marks the brick as visible. */
static uint32_t cell_at(const rctx* C, const int32_t v[3], uint32_t* s_log, uint32_t depth) {
  const uint32_t L = C->L, b = 1u << L;
  const uint32_t bx = (uint32_t)v[0] >> L, by = (uint32_t)v[1] >> L, bz = (uint32_t)v[2] >> L;
  const uint32_t id = bx + C->nb[0] * (by + C->nb[1] * bz);
  if (!(C->flags[id] & 2u)) {
    *s_log = L;
    return 0u;
  }
  if (C->visible && depth <= C->request_depth) C->visible[id] = 1u;
  if (C->offsets[id] == R_NOT_DECODED) {
    *s_log = L;
    const uint8_t* rec = C->vol + C->rec_off + 4 * (size_t)rd32(C->vol + 128 + 4 * (size_t)id);
    const uint32_t n_pal = rd32(rec), S = rd32(rec + 4);
    const uint32_t ns = oracle_head_words(C->coder, C->vflags, S);
    return n_pal ? rd32(rec + 16 + 4 * (size_t)ns) : 0u;
  }
  const uint32_t k = C->lods[id], e = b >> k;
  const uint32_t cx = ((uint32_t)v[0] - bx * b) >> k, cy = ((uint32_t)v[1] - by * b) >> k,
                 cz = ((uint32_t)v[2] - bz * b) >> k;
  *s_log = k;
  return C->cache[C->offsets[id] + (uint64_t)((cz * e + cy) * e + cx)];
}

/* One step in cells of edge 2^s_log; 0 when the ray leaves the volume. */
static int step(const rctx* C, ray* r, uint32_t s_log) {
  const int32_t S = 1 << s_log;
  const float fS = (float)S, inv = 1.0f / fS;
  int32_t c[3];
  float q[3], dist[3];
  for (int a = 0; a < 3; ++a) {
    c[a] = r->v[a] / S; /* v >= 0 */
    q[a] = ((float)(r->v[a] - c[a] * S) + r->p[a]) * inv;
    if (r->d[a] > 0.0f) dist[a] = (1.0f - q[a]) / r->d[a];
    else if (r->d[a] < 0.0f) dist[a] = (0.0f - q[a]) / r->d[a];
    else dist[a] = INFINITY;
  }
  int ax = 0;
  if (dist[1] < dist[ax]) ax = 1;
  if (dist[2] < dist[ax]) ax = 2;
  const float tt = dist[ax];
  for (int a = 0; a < 3; ++a)
    if (a != ax) q[a] = clamp01(q[a] + tt * r->d[a]);
  if (r->d[ax] > 0.0f) {
    c[ax] += 1;
    q[ax] = 0.0f;
    r->face = 2u * (uint32_t)ax + 1u;
  } else {
    c[ax] -= 1;
    q[ax] = R_ONE_MINUS;
    r->face = 2u * (uint32_t)ax + 2u;
  }
  r->t = r->t + tt * fS;
  int inside = 1;
  for (int a = 0; a < 3; ++a) {
    const float w = q[a] * fS;
    const float fl = floorf(w);
    r->v[a] = c[a] * S + (int32_t)fl;
    r->p[a] = w - fl;
    inside = inside && r->v[a] >= 0 && r->v[a] < (int32_t)C->dims[a];
  }
  return inside;
}

static int march_opaque(const rctx* C, ray* r, float max_t, uint32_t* hit, uint32_t depth) {
  const uint32_t max_steps = 3u * (C->dims[0] + C->dims[1] + C->dims[2]) + 64u;
  for (uint32_t k = 0; k < max_steps; ++k) {
    uint32_t s;
    const uint32_t l = cell_at(C, r->v, &s, depth);
    if (opaque(C, l)) {
      *hit = l;
      return 1;
    }
    if (!step(C, r, s) || r->t > max_t) return 0;
  }
  return 0;
}

static void face_normal(uint32_t face, float n[3]) {
  n[0] = n[1] = n[2] = 0.0f;
  if (face) n[(face - 1u) >> 1] = (face & 1u) ? -1.0f : 1.0f;
}

static ray from_face(const ray* h, const float dir[3]) {
  ray r;
  const int ax = (int)((h->face - 1u) >> 1);
  for (int a = 0; a < 3; ++a) {
    r.v[a] = h->v[a];
    r.p[a] = h->p[a];
    r.d[a] = dir[a];
  }
  if (h->face & 1u) {
    r.v[ax] -= 1;
    r.p[ax] = R_ONE_MINUS;
  } else {
    r.v[ax] += 1;
    r.p[ax] = 0.0f;
  }
  r.t = 0.0f;
  r.face = 0u;
  return r;
}

static int in_volume(const rctx* C, const int32_t v[3]) {
  for (int a = 0; a < 3; ++a)
    if (v[a] < 0 || v[a] >= (int32_t)C->dims[a]) return 0;
  return 1;
}

static void cosine_dir(uint32_t st[2], const float n[3], float out[3]) {
  float v[3] = {0.0f, 0.0f, 0.0f}, r2 = 0.0f;
  int ok = 0;
  for (int k = 0; k < 16 && !ok; ++k) {
    float a, b, c, unused;
    next2(st, &a, &b);
    next2(st, &c, &unused);
    v[0] = 2.0f * a - 1.0f;
    v[1] = 2.0f * b - 1.0f;
    v[2] = 2.0f * c - 1.0f;
    r2 = dot3(v, v);
    ok = r2 > 0.0f && r2 <= 1.0f;
  }
  if (ok) {
    const float len = sqrtf(r2);
    float w[3];
    for (int a = 0; a < 3; ++a) w[a] = n[a] + v[a] / len;
    const float w2 = dot3(w, w);
    if (w2 > 1e-12f) {
      const float wl = sqrtf(w2);
      for (int a = 0; a < 3; ++a) out[a] = w[a] / wl;
      return;
    }
  }
  for (int a = 0; a < 3; ++a) out[a] = n[a];
}

static void render_pixel(const rctx* C, const cam_frame* cam, uint32_t px, uint32_t py, uint32_t frame, int jitter,
                         uint32_t* label_out, float* depth_out, uint8_t* face_out, float rgb[3]) {
  float jx = 0.0f, jy = 0.0f;
  if (jitter) {
    uint32_t gj[2] = {frame, 0xA511E9B3u};
    float u0, u1, u2, u3, u4, u5;
    next2(gj, &u0, &u1);
    next2(gj, &u2, &u3);
    next2(gj, &u4, &u5);
    jx = ((u0 + u1) + u2 - 1.5f) * 0.6666667f;
    jy = ((u3 + u4) + u5 - 1.5f) * 0.6666667f;
  }
  const float sx = ((((float)px + 0.5f) + jx) * cam->inv_w2 - 1.0f) * cam->sxs;
  const float sy = (1.0f - (((float)py + 0.5f) + jy) * cam->inv_h2) * cam->sys;
  float d[3];
  for (int a = 0; a < 3; ++a) d[a] = (cam->f[a] + sx * cam->r[a]) + sy * cam->u[a];
  const float dl = sqrtf(dot3(d, d));
  for (int a = 0; a < 3; ++a) d[a] = d[a] / dl;
  float t0 = 0.0f, t1 = INFINITY;
  int entry_ax = -1, miss = 0;
  for (int a = 0; a < 3; ++a) {
    const float n = (float)C->dims[a];
    if (d[a] == 0.0f) {
      if (cam->o[a] < 0.0f || cam->o[a] >= n) miss = 1;
      continue;
    }
    float ta = (0.0f - cam->o[a]) / d[a], tb = (n - cam->o[a]) / d[a];
    if (ta > tb) { const float x = ta; ta = tb; tb = x; }
    if (ta > t0) { t0 = ta; entry_ax = a; }
    if (tb < t1) t1 = tb;
  }
  uint32_t out_label = 0u, out_face = 0u;
  float out_depth = INFINITY;
  rgb[0] = rgb[1] = rgb[2] = 0.0f;
  uint32_t g[2] = {px ^ (frame * 0x9E3779B9u), py + (frame << 16)};
  pcg2d(&g[0], &g[1]);
  if (!miss && t0 < t1) {
    ray r;
    for (int a = 0; a < 3; ++a) {
      r.d[a] = d[a];
      const float pa = cam->o[a] + t0 * d[a];
      float fc = floorf(pa);
      if (fc < 0.0f) fc = 0.0f;
      if (fc > (float)(C->dims[a] - 1u)) fc = (float)(C->dims[a] - 1u);
      r.v[a] = (int32_t)fc;
      r.p[a] = clamp01(pa - fc);
    }
    r.t = t0;
    r.face = entry_ax < 0 ? 0u : 2u * (uint32_t)entry_ax + (d[entry_ax] > 0.0f ? 1u : 2u);
    float T = 1.0f;
    uint32_t prev = 0u;
    int hit = 0;
    const uint32_t max_steps = 3u * (C->dims[0] + C->dims[1] + C->dims[2]) + 64u;
    for (uint32_t k = 0; k < max_steps && T >= 0.00390625f; ++k) {
      uint32_t s;
      const uint32_t l = cell_at(C, r.v, &s, 0u);
      if (l != prev && l != 0u) {
        const float* m = mat_of(C, l);
        if (m[3] > 0.0f) {
          float n[3];
          face_normal(r.face, n);
          if (!r.face)
            for (int a = 0; a < 3; ++a) n[a] = 0.0f - d[a];
          if (m[3] >= 1.0f) {
            hit = 1;
            out_label = l;
            out_depth = r.t;
            out_face = r.face;
            break;
          }
          float nl = dot3(n, C->light);
          if (nl < 0.0f) nl = 0.0f;
          const float shade = C->ambient + (1.0f - C->ambient) * nl;
          const float w = T * m[3];
          for (int a = 0; a < 3; ++a) rgb[a] = rgb[a] + w * (m[a] * shade);
          T = T * (1.0f - m[3]);
        }
      }
      prev = l;
      if (!step(C, &r, s)) break;
    }
    if (hit) {
      const float* m = mat_of(C, out_label);
      float n[3], c3[3] = {0.0f, 0.0f, 0.0f};
      face_normal(r.face, n);
      if (!r.face)
        for (int a = 0; a < 3; ++a) n[a] = 0.0f - d[a];
      if (C->mode == 0 || C->mode == 1) {
        float nl = dot3(n, C->light);
        if (nl < 0.0f) nl = 0.0f;
        if (C->mode == 1 && nl > 0.0f && r.face) {
          ray sr = from_face(&r, C->light);
          uint32_t l2;
          if (in_volume(C, sr.v) && march_opaque(C, &sr, INFINITY, &l2, 1u)) nl = 0.0f;
        }
        const float shade = C->ambient + (1.0f - C->ambient) * nl;
        for (int a = 0; a < 3; ++a) c3[a] = m[a] * shade;
      } else if (C->mode == 2) {
        float dir[3];
        cosine_dir(g, n, dir);
        int occluded = 0;
        if (r.face) {
          ray ar = from_face(&r, dir);
          uint32_t l2;
          occluded = in_volume(C, ar.v) && march_opaque(C, &ar, C->ao_radius, &l2, 1u);
        }
        for (int a = 0; a < 3; ++a) c3[a] = occluded ? 0.0f : m[a] * C->sky;
      } else {
        float tp[3] = {m[0], m[1], m[2]};
        ray h = r;
        for (uint32_t bounce = 1; bounce <= C->max_bounces && h.face; ++bounce) {
          float nn[3], dir[3];
          face_normal(h.face, nn);
          cosine_dir(g, nn, dir);
          ray br = from_face(&h, dir);
          uint32_t l2 = 0u;
          if (!in_volume(C, br.v) || !march_opaque(C, &br, INFINITY, &l2, bounce)) {
            for (int a = 0; a < 3; ++a) c3[a] = c3[a] + tp[a] * C->sky;
            break;
          }
          const float* m2 = mat_of(C, l2);
          for (int a = 0; a < 3; ++a) tp[a] = tp[a] * m2[a];
          if (bounce >= 4u) {
            float q = tp[0] > tp[1] ? tp[0] : tp[1];
            if (tp[2] > q) q = tp[2];
            if (q > 1.0f) q = 1.0f;
            float u, unused;
            next2(g, &u, &unused);
            if (!(u < q)) break;
            for (int a = 0; a < 3; ++a) tp[a] = tp[a] / q;
          }
          h = br;
        }
      }
      for (int a = 0; a < 3; ++a) rgb[a] = rgb[a] + T * c3[a];
    }
  }
  *label_out = out_label;
  *depth_out = out_depth;
  *face_out = (uint8_t)out_face;
}

/* Renders W x H pixels (row py at py * W). vol: the encoding (palette flags, coarsest labels);
 * offsets / lods / cache: per brick the word offset of its labels at its level of detail (x
 * fastest; ~0 = not decoded), the level, and the labels. Returns 0, -1 (argument) or the
 * palette scan's error. */
int oracle_render(const uint8_t* vol, size_t size, const uint64_t* offsets, const uint8_t* lods, const uint32_t* cache,
                  const float pos[3], const float dir[3], const float up[3], float fov_y, uint32_t W, uint32_t H,
                  const oracle_render_params* P, uint32_t* labels, float* depth, uint8_t* faces, float* rgb) {
  if (!vol || !offsets || !lods || !cache || !P || !labels || !depth || !faces || !rgb || W == 0 || H == 0) return -1;
  if (P->n_materials == 0 || P->n_materials > 256 || !P->materials) return -1;
  rctx C;
  memset(&C, 0, sizeof(C));
  uint8_t* fl = NULL;
  int rc = oracle_palette_flags(vol, size, C.nb, &C.L, &fl);
  if (rc) return rc;
  for (int a = 0; a < 3; ++a) C.dims[a] = rd32(vol + 8 + 4 * a);
  C.coder = rd32(vol + 28);
  C.vflags = rd32(vol + 32);
  const uint32_t n = rd32(vol + 36);
  C.vol = vol;
  C.rec_off = (128 + 4 * ((size_t)n + 1) + 15) & ~(size_t)15;
  C.flags = fl;
  C.offsets = offsets;
  C.lods = lods;
  C.cache = cache;
  const double l2 = (double)P->light_dir[0] * P->light_dir[0] + (double)P->light_dir[1] * P->light_dir[1] +
                    (double)P->light_dir[2] * P->light_dir[2];
  if (!(l2 > 0.0)) { free(fl); return -1; }
  const double ll = sqrt(l2);
  for (int a = 0; a < 3; ++a) C.light[a] = (float)(P->light_dir[a] / ll);
  C.ambient = P->ambient;
  C.ao_radius = P->ao_radius;
  C.sky = P->sky;
  C.mode = P->mode;
  C.max_bounces = P->max_bounces;
  C.n_mat = P->n_materials;
  C.mat = P->materials;
  C.visible = P->visible;
  C.request_depth = P->request_depth;
  cam_frame cam;
  oracle_camera_frame(pos, dir, up, fov_y, W, H, &cam);
  for (uint32_t py = 0; py < H; ++py)
    for (uint32_t px = 0; px < W; ++px) {
      const size_t i = (size_t)py * W + px;
      if (!oracle_subset_pixel(px, py, P->subsample, P->frame)) continue;
      render_pixel(&C, &cam, px, py, P->frame, P->jitter != 0, &labels[i], &depth[i], &faces[i], rgb + 3 * i);
    }
  free(fl);
  return 0;
}
