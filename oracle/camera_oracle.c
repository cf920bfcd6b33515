/*
 * Camera request oracle: which bricks a pinhole camera's pixel rays request, and at which level
 * of detail. TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU-baseline
 * leg); it shares no code with the GPU library.
 *
 * Paper, Methods "GPU rendering pipeline": rays traced through the volume mark the bricks they
 * pass as visible; bricks holding no visible label are skipped; the level of detail of a brick
 * depends only on its centre position. Results "Ray marching": the level of detail is chosen so
 * that one voxel of the brick covers about one pixel, and the traversal is a DDA that keeps an
 * integer cell index and a sub-cell position in [0, 1] for numerical stability. Readings taken
 * here (the paper gives no brick-granularity request rule in code):
 *   - a brick is visible iff its palette holds a label other than 0 (0 = background);
 *   - a ray stops after the first brick whose palette has no 0 (every voxel visible: the ray
 *     certainly hits a surface in it);
 *   - pixel (px, py) shoots the ray o + t d with d = f + sx r + sy u, sx = ((px + 1/2) 2 / W - 1)
 *     tan(fov/2) W / H, sy = (1 - (py + 1/2) 2 / H) tan(fov/2), (f, r, u) the orthonormal camera
 *     frame (f = dir / |dir|, r = f x up / |f x up|, u = r x f);
 *   - level of detail k = the largest k <= max_lod with 4^k <= |c - o|^2 (2 tan(fov/2) / H)^2,
 *     c the brick centre (a brick voxel of edge 2^k then covers at most one pixel's footprint).
 * The camera frame, tan(fov/2), the pixel scales and (2 tan(fov/2) / H)^2 are computed in double
 * precision and rounded to float once; every per-ray and per-brick step is float arithmetic in
 * the order written (compile without floating-point contraction), so that a GPU implementation
 * taking the same float steps makes the same integer decisions.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define C_HEADER_BYTES 128u
#define C_MAGIC 0x315A4356u

static uint32_t crd32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

/* csgv_oracle.c: words between a record's header and its palette (rANS states and run starts). */
uint32_t oracle_head_words(uint32_t coder, uint32_t flags, uint32_t S);

/* Per brick: bit 0 = palette holds label 0, bit 1 = palette holds a label other than 0. */
int oracle_palette_flags(const uint8_t* vol, size_t size, uint32_t nb[3], uint32_t* L_out, uint8_t** flags_out) {
  if (size < C_HEADER_BYTES || crd32(vol) != C_MAGIC) return -2;
  const uint32_t L = crd32(vol + 20), coder = crd32(vol + 28), flags = crd32(vol + 32), n = crd32(vol + 36);
  const uint32_t b = 1u << L;
  for (int a = 0; a < 3; ++a) nb[a] = (crd32(vol + 8 + 4 * a) + b - 1) / b;
  const size_t rec_off = (C_HEADER_BYTES + 4 * ((size_t)n + 1) + 15) & ~(size_t)15;
  uint8_t* fl = (uint8_t*)calloc(n ? n : 1, 1);
  if (!fl) return -3;
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t a = crd32(vol + C_HEADER_BYTES + 4 * (size_t)i);
    const uint8_t* r = vol + rec_off + 4 * (size_t)a;
    const uint32_t n_pal = crd32(r), S = crd32(r + 4);
    const uint32_t ns = oracle_head_words(coder, flags, S);
    const uint8_t* pal = r + 16 + 4 * (size_t)ns;
    for (uint32_t k = 0; k < n_pal; ++k) fl[i] |= crd32(pal + 4 * (size_t)k) == 0 ? 1u : 2u;
  }
  *L_out = L;
  *flags_out = fl;
  return 0;
}

typedef struct {
  float o[3], f[3], r[3], u[3];
  float sxs, sys, inv_w2, inv_h2, lod_s2;
} cam_frame;

void oracle_camera_frame(const float pos[3], const float dir[3], const float up[3], float fov_y, uint32_t W,
                         uint32_t H, cam_frame* c) {
  double f[3] = {dir[0], dir[1], dir[2]};
  double fl = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  for (int a = 0; a < 3; ++a) f[a] /= fl;
  double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
  double rl = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  for (int a = 0; a < 3; ++a) r[a] /= rl;
  double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
  const double t = tan(0.5 * (double)fov_y);
  for (int a = 0; a < 3; ++a) {
    c->o[a] = pos[a];
    c->f[a] = (float)f[a];
    c->r[a] = (float)r[a];
    c->u[a] = (float)u[a];
  }
  c->sxs = (float)(t * (double)W / (double)H);
  c->sys = (float)t;
  c->inv_w2 = (float)(2.0 / (double)W);
  c->inv_h2 = (float)(2.0 / (double)H);
  const double s = 2.0 * t / (double)H;
  c->lod_s2 = (float)(s * s);
}

/* One ray through the brick grid; calls mark(id) for every visible brick it passes. */
static void march(const cam_frame* c, float b, const uint32_t nb[3], const uint8_t* fl, uint32_t px, uint32_t py,
                  uint8_t* marked) {
  const float sx = (((float)px + 0.5f) * c->inv_w2 - 1.0f) * c->sxs;
  const float sy = (1.0f - ((float)py + 0.5f) * c->inv_h2) * c->sys;
  float d[3], o[3];
  for (int a = 0; a < 3; ++a) {
    const float da = (c->f[a] + sx * c->r[a]) + sy * c->u[a];
    d[a] = da / b;       /* brick units (b is a power of two: exact scaling) */
    o[a] = c->o[a] / b;
  }
  /* entry and exit parameters of the grid box [0, nb) */
  float t0 = 0.0f, t1 = INFINITY;
  for (int a = 0; a < 3; ++a) {
    const float n = (float)nb[a];
    if (d[a] == 0.0f) {
      if (o[a] < 0.0f || o[a] >= n) return;
      continue;
    }
    float ta = (0.0f - o[a]) / d[a], tb = (n - o[a]) / d[a];
    if (ta > tb) { const float x = ta; ta = tb; tb = x; }
    if (ta > t0) t0 = ta;
    if (tb < t1) t1 = tb;
  }
  if (!(t0 < t1)) return;
  int32_t cell[3];
  float s[3];  /* sub-cell position in [0, 1] */
  for (int a = 0; a < 3; ++a) {
    const float p = o[a] + t0 * d[a];
    float fc = floorf(p);
    if (fc < 0.0f) fc = 0.0f;
    if (fc > (float)(nb[a] - 1)) fc = (float)(nb[a] - 1);
    cell[a] = (int32_t)fc;
    float q = p - fc;
    if (q < 0.0f) q = 0.0f;
    if (q > 1.0f) q = 1.0f;
    s[a] = q;
  }
  const uint32_t max_steps = nb[0] + nb[1] + nb[2] + 1;
  for (uint32_t step = 0; step < max_steps; ++step) {
    const uint32_t id = (uint32_t)cell[0] + nb[0] * ((uint32_t)cell[1] + nb[1] * (uint32_t)cell[2]);
    if (fl[id] & 2u) marked[id] = 1;
    if (!(fl[id] & 1u)) return;  /* no background in this brick: the ray ends here */
    /* distance to the next cell face along each axis; the smallest wins, ties to x, then y */
    float dist[3];
    for (int a = 0; a < 3; ++a) {
      if (d[a] > 0.0f) dist[a] = (1.0f - s[a]) / d[a];
      else if (d[a] < 0.0f) dist[a] = (0.0f - s[a]) / d[a];
      else dist[a] = INFINITY;
    }
    int ax = 0;
    if (dist[1] < dist[ax]) ax = 1;
    if (dist[2] < dist[ax]) ax = 2;
    const float t = dist[ax];
    for (int a = 0; a < 3; ++a) {
      if (a == ax) continue;
      float q = s[a] + t * d[a];
      if (q < 0.0f) q = 0.0f;
      if (q > 1.0f) q = 1.0f;
      s[a] = q;
    }
    if (d[ax] > 0.0f) {
      cell[ax] += 1;
      s[ax] = 0.0f;
      if (cell[ax] >= (int32_t)nb[ax]) return;
    } else {
      cell[ax] -= 1;
      s[ax] = 1.0f;
      if (cell[ax] < 0) return;
    }
  }
}

/* Level of detail of brick (bx, by, bz) from its centre's squared distance to the camera. */
static uint32_t brick_lod(const cam_frame* c, float b, uint32_t bx, uint32_t by, uint32_t bz, uint32_t max_lod) {
  const float cx = ((float)bx + 0.5f) * b - c->o[0];
  const float cy = ((float)by + 0.5f) * b - c->o[1];
  const float cz = ((float)bz + 0.5f) * b - c->o[2];
  const float q = ((cx * cx + cy * cy) + cz * cz) * c->lod_s2;
  uint32_t k = 0;
  while (k < max_lod && q >= (float)(1u << (2 * (k + 1)))) ++k;
  return k;
}

/* Bricks requested by one camera, ascending ids, with their levels of detail (max_lod is
 * clamped to log2 b). Returns 0, -1 (argument), -2 (format), -3 (memory) or -7 (more than cap
 * bricks; *n_out still receives the count). */
int oracle_camera_bricks(const uint8_t* vol, size_t size, const float pos[3], const float dir[3], const float up[3],
                         float fov_y, uint32_t width, uint32_t height, uint32_t max_lod, uint32_t* ids,
                         uint32_t* lods, uint32_t cap, uint32_t* n_out) {
  if (!vol || !pos || !dir || !up || !n_out || width == 0 || height == 0) return -1;
  uint32_t nb[3], L;
  uint8_t* fl = NULL;
  int rc = oracle_palette_flags(vol, size, nb, &L, &fl);
  if (rc) return rc;
  const uint32_t n = nb[0] * nb[1] * nb[2];
  uint8_t* marked = (uint8_t*)calloc(n ? n : 1, 1);
  if (!marked) { free(fl); return -3; }
  cam_frame c;
  oracle_camera_frame(pos, dir, up, fov_y, width, height, &c);
  const float b = (float)(1u << L);
  for (uint32_t py = 0; py < height; ++py)
    for (uint32_t px = 0; px < width; ++px) march(&c, b, nb, fl, px, py, marked);
  if (max_lod > L) max_lod = L;
  uint32_t cnt = 0;
  for (uint32_t id = 0; id < n; ++id) {
    if (!marked[id]) continue;
    if (cnt < cap && ids && lods) {
      const uint32_t bx = id % nb[0], by = (id / nb[0]) % nb[1], bz = id / (nb[0] * nb[1]);
      ids[cnt] = id;
      lods[cnt] = brick_lod(&c, b, bx, by, bz, max_lod);
    }
    ++cnt;
  }
  *n_out = cnt;
  free(marked);
  free(fl);
  return cnt > cap ? -7 : 0;
}

/* The level of detail of every brick for one camera (the same centre rule; max_lod clamped to
 * log2 b): lods_out[id], one byte per brick. Returns 0, -1 (argument) or the header's error. */
int oracle_brick_lods(const uint8_t* vol, size_t size, const float pos[3], const float dir[3], const float up[3],
                      float fov_y, uint32_t width, uint32_t height, uint32_t max_lod, uint8_t* lods_out) {
  if (!vol || !pos || !dir || !up || !lods_out || width == 0 || height == 0) return -1;
  uint32_t nb[3], L;
  uint8_t* fl = NULL;
  int rc = oracle_palette_flags(vol, size, nb, &L, &fl);
  if (rc) return rc;
  free(fl);
  cam_frame c;
  oracle_camera_frame(pos, dir, up, fov_y, width, height, &c);
  const float b = (float)(1u << L);
  if (max_lod > L) max_lod = L;
  const uint32_t n = nb[0] * nb[1] * nb[2];
  for (uint32_t id = 0; id < n; ++id)
    lods_out[id] = (uint8_t)brick_lod(&c, b, id % nb[0], (id / nb[0]) % nb[1], id / (nb[0] * nb[1]), max_lod);
  return 0;
}
