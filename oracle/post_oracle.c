/*
 * Post-processing oracle: accumulation, G-buffer, edge-avoiding À-trous denoising and upsampling of
 * rendered frames. TEST INFRASTRUCTURE ONLY; it shares no code with the GPU library.
 *
 * Paper, Methods "Post-processing":
 *   - "G-Buffer": per pixel, for the first surface of the most recent frame, the normal (3 bits:
 *     one of six directions; 011 = no surface, 111 = not rendered yet), the depth quantised to 13
 *     bits as the normalised distance from the dataset's bounding sphere, and the 32-bit label;
 *   - "Denoising": at most one sample per pixel and frame is accumulated; pass i combines the 3 x 3
 *     pixels q at distance 2^i around p, c_{i+1}(p) = sum h w c_i(q) / sum h w, h = (1,2,1) x
 *     (1,2,1), w = 0 if the normals differ, else 1 / (1 + <rho_D, rho_D>) exp(-|d_p - d_q| phi_d),
 *     rho_D = (hsv albedo_p - hsv albedo_q) phi_rho; the last pass's result is the output (no
 *     up-passes);
 *   - "Upsampling": a pixel not rendered yet takes part in no filter; the passes carry an offset to
 *     the nearest rendered pixel, o_p <- the shorter of o_p and o_q + (q - p) (jump flooding), and
 *     the pixel then takes that pixel's colour;
 *   - the last step tone maps (Narkowicz's ACES fit) and corrects gamma.
 * Readings (the same in the library): normal code = axis | (1 if the normal points to -axis) << 2;
 * depth code = round(clamp((t - (|cam - centre| - R)) / (2R), 0, 1) 8191), centre = dims / 2,
 * R = |dims| / 2, no-surface pixels 8191; depth differences in voxels (code steps x 2R / 8191);
 * the albedo of a label is its material's (label l -> hash(l) mod n); hue without wrap-around;
 * neighbour order y then x from -1 to 1, the first strictly shorter offset wins; exposure scales
 * before the tone map; bytes round half up. Float steps are single IEEE operations in the order
 * written (compile without contraction); exp and pow come from the C library.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#define P_NOHIT 3u
#define P_INVALID 7u
#define P_NO_OFFSET 0x7FFF7FFF

int oracle_subset_pixel(uint32_t px, uint32_t py, uint32_t s, uint32_t f);

typedef struct {
  uint32_t width, height, iterations, subsample, frame, reset;
  float cam_pos[3];
  float phi_rho, phi_d, exposure, gamma;
  uint32_t n_materials;
  const float* materials; /* n x (r, g, b, opacity) */
} oracle_post_params;

static uint32_t mat_index(uint32_t l, uint32_t n) {
  uint32_t h = l * 0x9E3779B1u;
  h ^= h >> 15;
  h *= 0x85EBCA77u;
  h ^= h >> 13;
  return h % n;
}

static void hsv_of(const float rgb[3], float hsv[3]) {
  const double r = rgb[0], g = rgb[1], b = rgb[2];
  const double mx = fmax(r, fmax(g, b)), mn = fmin(r, fmin(g, b)), c = mx - mn;
  double h = 0.0;
  if (c > 0.0) {
    if (mx == r) h = fmod((g - b) / c + 6.0, 6.0);
    else if (mx == g) h = (b - r) / c + 2.0;
    else h = (r - g) / c + 4.0;
    h /= 6.0;
  }
  hsv[0] = (float)h;
  hsv[1] = (float)(mx > 0.0 ? c / mx : 0.0);
  hsv[2] = (float)mx;
}

static int32_t odx(int32_t o) { return (int32_t)(int16_t)(o & 0xFFFF); }
static int32_t ody(int32_t o) { return o >> 16; }

static float aces(float x) {
  const float num = x * (2.51f * x + 0.03f);
  const float den = x * (2.43f * x + 0.59f) + 0.14f;
  float y = num / den;
  return y < 0.0f ? 0.0f : (y > 1.0f ? 1.0f : y);
}

/* One frame. State (host, n = W H pixels, kept by the caller between frames): accum n x 4 floats,
 * col0 / col1 n x 4 floats, glabel / gcode n u32, off0 / off1 n i32. dims: the volume's extent. */
int oracle_post(const oracle_post_params* P, const uint32_t dims[3], const uint32_t* labels, const float* depth,
                const uint8_t* face, const float* rgb, float* accum, float* col0, float* col1, uint32_t* glabel,
                uint32_t* gcode, int32_t* off0, int32_t* off1, uint32_t* out) {
  if (!P || !dims || !labels || !depth || !face || !rgb || !accum || !col0 || !col1 || !glabel || !gcode || !off0 ||
      !off1 || !out || !P->width || !P->height || P->n_materials == 0 || P->n_materials > 256)
    return -1;
  const uint32_t W = P->width, H = P->height, n = W * H;
  float hsv[256][3];
  for (uint32_t m = 0; m < P->n_materials; ++m) hsv_of(P->materials + 4 * (size_t)m, hsv[m]);
  double c[3], R2 = 0.0, D2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    c[a] = 0.5 * dims[a];
    R2 += c[a] * c[a];
    D2 += (P->cam_pos[a] - c[a]) * (P->cam_pos[a] - c[a]);
  }
  const double R = sqrt(R2);
  const float d_near = (float)(sqrt(D2) - R), d_scale = (float)(1.0 / (2.0 * R));
  const float vox_per_code = (float)(2.0 * R / 8191.0), inv_gamma = (float)(1.0 / (double)P->gamma);
  float* col[2] = {col0, col1};
  int32_t* off[2] = {off0, off1};
  /* accumulation and G-buffer */
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t px = i % W, py = i / W;
    float* a = accum + 4 * (size_t)i;
    if (P->reset) {
      a[0] = a[1] = a[2] = a[3] = 0.0f;
      gcode[i] = P_INVALID;
      glabel[i] = 0u;
    }
    if (oracle_subset_pixel(px, py, P->subsample, P->frame)) {
      for (int k = 0; k < 3; ++k) a[k] = a[k] + rgb[3 * (size_t)i + k];
      a[3] = a[3] + 1.0f;
      glabel[i] = labels[i];
      if (labels[i] == 0u || face[i] == 0u) {
        gcode[i] = P_NOHIT | (8191u << 3);
      } else {
        const uint32_t f = face[i];
        const uint32_t normal = ((f - 1u) >> 1) | ((f & 1u) << 2);
        float dn = (depth[i] - d_near) * d_scale;
        dn = dn < 0.0f ? 0.0f : (dn > 1.0f ? 1.0f : dn);
        gcode[i] = normal | ((uint32_t)(dn * 8191.0f + 0.5f) << 3);
      }
    }
    if ((gcode[i] & 7u) != P_INVALID) {
      const float inv = 1.0f / a[3];
      for (int k = 0; k < 3; ++k) col[0][4 * (size_t)i + k] = a[k] * inv;
      col[0][4 * (size_t)i + 3] = 0.0f;
      off[0][i] = 0;
    } else {
      for (int k = 0; k < 4; ++k) col[0][4 * (size_t)i + k] = 0.0f;
      off[0][i] = P_NO_OFFSET;
    }
  }
  /* passes */
  for (uint32_t it = 0; it < P->iterations; ++it) {
    const uint32_t src = it & 1u, dst = src ^ 1u;
    const int32_t st = 1 << it;
    for (uint32_t i = 0; i < n; ++i) {
      const int32_t px = (int32_t)(i % W), py = (int32_t)(i / W);
      const uint32_t code = gcode[i];
      if ((code & 7u) != P_INVALID) {
        const float* hp = hsv[glabel[i] ? mat_index(glabel[i], P->n_materials) : 0u];
        const int hit_p = (code & 7u) != P_NOHIT;
        const float dp = (float)(code >> 3);
        float sw = 0.0f, acc[3] = {0.0f, 0.0f, 0.0f};
        for (int32_t dy = -1; dy <= 1; ++dy)
          for (int32_t dx = -1; dx <= 1; ++dx) {
            const int32_t qx = px + dx * st, qy = py + dy * st;
            if (qx < 0 || qy < 0 || qx >= (int32_t)W || qy >= (int32_t)H) continue;
            const uint32_t j = (uint32_t)qy * W + (uint32_t)qx;
            const uint32_t cq = gcode[j];
            if ((cq & 7u) == P_INVALID || (cq & 7u) != (code & 7u)) continue;
            const float h = (float)((dx == 0 ? 2 : 1) * (dy == 0 ? 2 : 1));
            float w = 1.0f;
            if (hit_p) {
              const float* hq = hsv[glabel[j] ? mat_index(glabel[j], P->n_materials) : 0u];
              const float r0 = (hp[0] - hq[0]) * P->phi_rho, r1 = (hp[1] - hq[1]) * P->phi_rho,
                          r2 = (hp[2] - hq[2]) * P->phi_rho;
              const float rr = (r0 * r0 + r1 * r1) + r2 * r2;
              const float dd = fabsf(dp - (float)(cq >> 3)) * vox_per_code;
              w = (1.0f / (1.0f + rr)) * expf(-P->phi_d * dd);
            }
            const float hw = h * w;
            for (int k = 0; k < 3; ++k) acc[k] = acc[k] + hw * col[src][4 * (size_t)j + k];
            sw = sw + hw;
          }
        for (int k = 0; k < 3; ++k) col[dst][4 * (size_t)i + k] = acc[k] / sw;
        col[dst][4 * (size_t)i + 3] = 0.0f;
        off[dst][i] = 0;
      } else {
        int32_t best = off[src][i];
        int64_t bl = best == P_NO_OFFSET ? INT64_MAX : (int64_t)odx(best) * odx(best) + (int64_t)ody(best) * ody(best);
        for (int32_t dy = -1; dy <= 1; ++dy)
          for (int32_t dx = -1; dx <= 1; ++dx) {
            const int32_t qx = px + dx * st, qy = py + dy * st;
            if ((dx == 0 && dy == 0) || qx < 0 || qy < 0 || qx >= (int32_t)W || qy >= (int32_t)H) continue;
            const int32_t oq = off[src][(uint32_t)qy * W + (uint32_t)qx];
            if (oq == P_NO_OFFSET) continue;
            const int32_t cx = odx(oq) + dx * st, cy = ody(oq) + dy * st;
            const int64_t l = (int64_t)cx * cx + (int64_t)cy * cy;
            if (l < bl) {
              bl = l;
              best = (cx & 0xFFFF) | (cy << 16);
            }
          }
        off[dst][i] = best;
        for (int k = 0; k < 4; ++k) col[dst][4 * (size_t)i + k] = 0.0f;
      }
    }
  }
  const uint32_t fin = P->iterations & 1u;
  for (uint32_t i = 0; i < n; ++i) {
    const int32_t px = (int32_t)(i % W), py = (int32_t)(i / W);
    const float* cc = NULL;
    static const float zero[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if ((gcode[i] & 7u) != P_INVALID) {
      cc = col[fin] + 4 * (size_t)i;
    } else {
      const int32_t o = off[fin][i];
      cc = o == P_NO_OFFSET ? zero : col[fin] + 4 * ((size_t)(py + ody(o)) * W + (size_t)(px + odx(o)));
    }
    uint32_t px8 = 0xFF000000u;
    for (int k = 0; k < 3; ++k) {
      float y = aces(cc[k] * P->exposure);
      y = powf(y, inv_gamma);
      uint32_t b = (uint32_t)(y * 255.0f + 0.5f);
      px8 |= (b > 255u ? 255u : b) << (8 * k);
    }
    out[i] = px8;
  }
  return 0;
}
