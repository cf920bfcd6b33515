/*
 * Seeded synthetic segmentation volumes: noise-perturbed Voronoi / power-diagram cells.
 *
 * This module generates the INPUT volumes V: N^3 -> N that both the CPU oracle (tests) and the
 * GPU path (tests, benchmark) consume. It holds none of the compression method's arithmetic:
 * it only produces voxel labels. The paper evaluates on connectomics segmentations whose
 * compression depends mainly on brick-local label density (Results, "CSGV results"); these
 * volumes stand in for them with cells of a chosen mean size, boundaries perturbed by
 * 3-octave value noise, a background fraction (label 0) and sparse random 32-bit ids.
 *
 * Everything is integer / fixed point (Q16.16), so the same parameters give the same voxels on
 * every machine and in every evaluation order; any box of voxels can be generated on its own.
 *
 * Definition of label(p) for a voxel p = (x, y, z):
 *   1. Hash grid: cells of edge g voxels. Cell c holds n(c) seeds, n ~ Binomial(8, lambda/8)
 *      drawn from splitmix64 hashes. Seed k of cell c sits at a uniform Q16.16 position inside
 *      the cell, has label id perm32(8*index(c)+k) (a keyed bijection on uint32, so ids are
 *      distinct), and is background (label 0) with probability p_bg.
 *      With rmean > 0 each seed gets a power-diagram weight w = r^2, r = rmean * m, m a
 *      log-normal (sigma 0.8) multiplier clamped to [1/4, 4], drawn from a 256-entry table.
 *   2. Displacement: d_a(p) = sum over octaves o of amp_o * noise_{o,a}(p), periods 16, 8, 4
 *      voxels, amp = A*4/7, A*2/7, A*1/7; noise = trilinear value noise of hashed lattice values
 *      in [-1, 1). The displaced point is q = p + 1/2 + d(p).
 *   3. label(p) = label of the seed that minimises |q - s|^2 - w_s over the 27 hash-grid cells
 *      around the cell containing q; ties go to the smaller global seed index.
 *   4. Forced-uniform bricks: with probability p_uni a brick (edge ub) takes label(centre) for
 *      all its voxels, centre = brick origin + ub/2 on every axis.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef struct synth_params {
  uint32_t dims[3];
  uint32_t grid;          /* hash-grid cell edge in voxels (>= 4) */
  uint64_t seed;
  uint32_t lambda_q16;    /* mean seeds per hash-grid cell, Q16.16, in (0, 8] */
  uint32_t bg_q16;        /* probability that a seed is background (label 0), Q16.16 */
  uint32_t amp_q16;       /* displacement amplitude A in voxels, Q16.16 */
  uint32_t rmean_q16;     /* mean power-diagram radius in voxels, Q16.16; 0 = plain Voronoi */
  uint32_t uniform_brick; /* brick edge for forced-uniform bricks; 0 = off */
  uint32_t uniform_q16;   /* probability that a brick is forced uniform, Q16.16 */
} synth_params;

/* exp(0.8 * Phi^-1((i + 0.5) / 256)) clamped to [1/4, 4], Q16.16 (log-normal quantiles). */
static const uint32_t LOGNORM_Q16[256] = {
     16384,  16384,  16384,  16384,  16384,  16384,  16384,  16384,
     16384,  16384,  16384,  16871,  17419,  17948,  18462,  18962,
     19450,  19928,  20395,  20854,  21305,  21750,  22187,  22619,
     23045,  23467,  23883,  24296,  24705,  25110,  25512,  25912,
     26308,  26702,  27093,  27483,  27870,  28256,  28640,  29022,
     29403,  29783,  30162,  30539,  30916,  31292,  31668,  32042,
     32417,  32790,  33164,  33537,  33910,  34283,  34655,  35028,
     35401,  35774,  36147,  36521,  36895,  37269,  37644,  38019,
     38395,  38771,  39148,  39526,  39904,  40283,  40663,  41044,
     41426,  41809,  42193,  42579,  42965,  43352,  43741,  44131,
     44522,  44915,  45309,  45704,  46101,  46500,  46900,  47302,
     47705,  48110,  48517,  48926,  49337,  49749,  50164,  50580,
     50999,  51420,  51842,  52267,  52695,  53124,  53556,  53990,
     54427,  54866,  55308,  55753,  56200,  56650,  57102,  57557,
     58016,  58477,  58941,  59409,  59879,  60353,  60830,  61310,
     61793,  62281,  62771,  63265,  63763,  64265,  64770,  65280,
     65793,  66311,  66832,  67358,  67888,  68423,  68962,  69505,
     70053,  70607,  71164,  71727,  72295,  72869,  73447,  74031,
     74620,  75216,  75816,  76423,  77036,  77655,  78280,  78912,
     79551,  80196,  80848,  81507,  82173,  82847,  83528,  84217,
     84914,  85619,  86332,  87054,  87785,  88524,  89273,  90031,
     90799,  91577,  92365,  93164,  93973,  94793,  95625,  96468,
     97323,  98191,  99071,  99965, 100872, 101792, 102727, 103677,
    104642, 105623, 106619, 107633, 108663, 109711, 110778, 111864,
    112970, 114095, 115243, 116411, 117603, 118818, 120058, 121323,
    122614, 123933, 125281, 126659, 128067, 129508, 130983, 132493,
    134040, 135626, 137253, 138922, 140637, 142398, 144208, 146071,
    147990, 149966, 152004, 154107, 156279, 158525, 160850, 163258,
    165755, 168348, 171044, 173851, 176776, 179831, 183025, 186372,
    189885, 193579, 197474, 201590, 205952, 210587, 215529, 220819,
    226503, 232640, 239300, 246573, 254570, 262144, 262144, 262144,
    262144, 262144, 262144, 262144, 262144, 262144, 262144, 262144,
};

enum { TAG_COUNT = 1, TAG_POS = 2, TAG_BG = 5, TAG_W = 6, TAG_UNI = 7, TAG_NOISE = 16 };

static inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static inline uint64_t hash5(uint64_t seed, uint64_t tag, int64_t a, int64_t b, int64_t c, uint64_t k) {
  uint64_t h = mix64(seed ^ (tag << 56));
  h = mix64(h ^ (uint64_t)a);
  h = mix64(h ^ (uint64_t)b);
  h = mix64(h ^ (uint64_t)c);
  return mix64(h ^ k);
}
/* keyed bijection on uint32 (xor-shift and odd multiplies are each invertible) */
static inline uint32_t perm32(uint32_t x, uint32_t key) {
  x ^= key;
  x *= 0x7FEB352Du; x ^= x >> 15;
  x *= 0x846CA68Bu; x ^= x >> 16;
  x += key * 0x9E3779B9u; x ^= x >> 13;
  x *= 0xC2B2AE35u; x ^= x >> 16;
  return x;
}
static inline int64_t floordiv(int64_t a, int64_t b) {  /* b > 0 */
  int64_t q = a / b;
  return (a % b != 0 && a < 0) ? q - 1 : q;
}

typedef struct { int64_t pos[3]; int64_t w; uint64_t gidx; uint32_t label; } seed_t;

/* Seeds of one hash-grid cell; returns the count (<= 8). */
static int cell_seeds(const synth_params* P, int64_t cx, int64_t cy, int64_t cz, seed_t* out) {
  const int64_t g = P->grid;
  const uint64_t pq32 = (uint64_t)P->lambda_q16 << 13;  /* lambda/8 as a fraction of 2^32 */
  /* padded-grid linear index: the grid is offset by 1 so that border neighbours stay >= 0 */
  const int64_t ngx = (P->dims[0] + g - 1) / g + 2, ngy = (P->dims[1] + g - 1) / g + 2;
  const uint64_t lin = (uint64_t)(((cz + 1) * ngy + (cy + 1)) * ngx + (cx + 1));
  int n = 0;
  for (int t = 0; t < 8; ++t)
    if ((hash5(P->seed, TAG_COUNT, cx, cy, cz, (uint64_t)t) >> 32) < pq32) ++n;
  const uint32_t key = (uint32_t)mix64(P->seed ^ 0xABCDEF12345ull);
  const int64_t cell_q16 = g << 16;
  for (int k = 0; k < n; ++k) {
    seed_t* s = &out[k];
    int64_t c[3] = {cx, cy, cz};
    for (int a = 0; a < 3; ++a)
      s->pos[a] = c[a] * cell_q16 + (int64_t)(hash5(P->seed, TAG_POS + (a << 2), cx, cy, cz, (uint64_t)k) % (uint64_t)cell_q16);
    s->gidx = lin * 8u + (uint64_t)k;
    uint32_t id = perm32((uint32_t)s->gidx, key);
    if ((hash5(P->seed, TAG_BG, cx, cy, cz, (uint64_t)k) >> 48) < P->bg_q16) id = 0;
    s->label = id;
    s->w = 0;
    if (P->rmean_q16) {
      uint64_t m = LOGNORM_Q16[hash5(P->seed, TAG_W, cx, cy, cz, (uint64_t)k) >> 56];
      int64_t r = (int64_t)(((uint64_t)P->rmean_q16 * m) >> 16); /* Q16.16 */
      s->w = r * r;                                              /* Q32.32 */
    }
  }
  return n;
}

static inline int32_t lattice_value(const synth_params* P, int oct, int comp, int64_t qx, int64_t qy, int64_t qz) {
  uint64_t h = hash5(P->seed, (uint64_t)(TAG_NOISE + oct * 3 + comp), qx, qy, qz, 0);
  return (int32_t)((h >> 47) & 0x1FFFF) - 65536;  /* [-1, 1) in Q16 */
}
static inline int32_t lerp_q16(int32_t a, int32_t b, int32_t t) {
  return a + (int32_t)(((int64_t)(b - a) * t) / 65536);
}

/* Per-block caches: noise lattice values and seeds of nearby hash-grid cells. */
#define BLK 16
typedef struct {
  int64_t org[3];
  /* lattice[oct][comp][...] over the lattice points covering the block */
  int64_t lat_org[3][3];
  int lat_n[3];
  int32_t* lat[3][3];
  int64_t cell_org[3];
  int cell_n[3];
  int* cell_start;  /* per cell: first seed index; cell_start[ncells] = total */
  seed_t* seeds;
} blockcache;

static const int PERIOD[3] = {16, 8, 4};

static void cache_build(const synth_params* P, blockcache* bc, const int64_t org[3]) {
  for (int a = 0; a < 3; ++a) bc->org[a] = org[a];
  for (int o = 0; o < 3; ++o) {
    int per = PERIOD[o];
    int n = BLK / per + 2;
    bc->lat_n[o] = n;
    for (int a = 0; a < 3; ++a) bc->lat_org[o][a] = floordiv(org[a], per);
    for (int comp = 0; comp < 3; ++comp) {
      int32_t* t = bc->lat[o][comp];
      for (int z = 0; z < n; ++z)
        for (int y = 0; y < n; ++y)
          for (int x = 0; x < n; ++x)
            t[(z * n + y) * n + x] = lattice_value(P, o, comp, bc->lat_org[o][0] + x, bc->lat_org[o][1] + y, bc->lat_org[o][2] + z);
    }
  }
  /* displaced points stay within A of the voxel centre; |d| < A + 1 voxel covers rounding */
  const int64_t g = P->grid;
  const int64_t reach = ((int64_t)P->amp_q16 >> 16) + 2;
  int total = 0;
  for (int a = 0; a < 3; ++a) {
    int64_t lo = floordiv(org[a] - reach, g) - 1, hi = floordiv(org[a] + BLK + reach, g) + 1;
    bc->cell_org[a] = lo;
    bc->cell_n[a] = (int)(hi - lo + 1);
  }
  int ncell = bc->cell_n[0] * bc->cell_n[1] * bc->cell_n[2];
  seed_t tmp[8];
  for (int ci = 0; ci < ncell; ++ci) {
    int x = ci % bc->cell_n[0], y = (ci / bc->cell_n[0]) % bc->cell_n[1], z = ci / (bc->cell_n[0] * bc->cell_n[1]);
    bc->cell_start[ci] = total;
    int n = cell_seeds(P, bc->cell_org[0] + x, bc->cell_org[1] + y, bc->cell_org[2] + z, tmp);
    memcpy(&bc->seeds[total], tmp, sizeof(seed_t) * (size_t)n);
    total += n;
  }
  bc->cell_start[ncell] = total;
}

static int32_t noise_at(const blockcache* bc, int o, int comp, const int64_t p[3]) {
  int per = PERIOD[o];
  int n = bc->lat_n[o];
  int32_t t[3];
  int i[3];
  for (int a = 0; a < 3; ++a) {
    int64_t q = floordiv(p[a], per);
    i[a] = (int)(q - bc->lat_org[o][a]);
    t[a] = (int32_t)((p[a] - q * per) * (65536 / per));
  }
  const int32_t* L = bc->lat[o][comp];
#define LV(dx, dy, dz) L[((i[2] + (dz)) * n + (i[1] + (dy))) * n + (i[0] + (dx))]
  int32_t x00 = lerp_q16(LV(0, 0, 0), LV(1, 0, 0), t[0]);
  int32_t x10 = lerp_q16(LV(0, 1, 0), LV(1, 1, 0), t[0]);
  int32_t x01 = lerp_q16(LV(0, 0, 1), LV(1, 0, 1), t[0]);
  int32_t x11 = lerp_q16(LV(0, 1, 1), LV(1, 1, 1), t[0]);
#undef LV
  return lerp_q16(lerp_q16(x00, x10, t[1]), lerp_q16(x01, x11, t[1]), t[2]);
}

/* label of voxel p, p inside the block cached in bc */
static uint32_t label_cached(const synth_params* P, const blockcache* bc, const int64_t p[3]) {
  const int64_t A = P->amp_q16;
  const int64_t amp[3] = {A * 4 / 7, A * 2 / 7, A / 7};
  int64_t q[3];
  for (int a = 0; a < 3; ++a) {
    int64_t d = 0;
    for (int o = 0; o < 3; ++o) d += amp[o] * noise_at(bc, o, a, p) / 65536;
    q[a] = (p[a] << 16) + 32768 + d;
  }
  const int64_t g = P->grid;
  int64_t gc[3];
  for (int a = 0; a < 3; ++a) gc[a] = floordiv(q[a], g << 16);
  int64_t best = INT64_MAX;
  uint64_t best_idx = UINT64_MAX;
  uint32_t best_label = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int x = (int)(gc[0] + dx - bc->cell_org[0]), y = (int)(gc[1] + dy - bc->cell_org[1]), z = (int)(gc[2] + dz - bc->cell_org[2]);
        int ci = (z * bc->cell_n[1] + y) * bc->cell_n[0] + x;
        for (int s = bc->cell_start[ci]; s < bc->cell_start[ci + 1]; ++s) {
          const seed_t* sd = &bc->seeds[s];
          int64_t e0 = q[0] - sd->pos[0], e1 = q[1] - sd->pos[1], e2 = q[2] - sd->pos[2];
          int64_t sc = e0 * e0 + e1 * e1 + e2 * e2 - sd->w;
          if (sc < best || (sc == best && sd->gidx < best_idx)) { best = sc; best_idx = sd->gidx; best_label = sd->label; }
        }
      }
  return best_label;
}

typedef struct {
  const synth_params* P;
  int64_t box_org[3];
  uint32_t box_n[3];
  uint32_t* out;
  int64_t nblk[3];
  int64_t next;  /* atomic work counter */
} fill_job;

static void* cache_alloc(const synth_params* P, blockcache* bc) {
  for (int o = 0; o < 3; ++o) {
    int n = BLK / PERIOD[o] + 2;
    for (int c = 0; c < 3; ++c) bc->lat[o][c] = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n * n * n));
  }
  const int64_t reach = ((int64_t)P->amp_q16 >> 16) + 2;
  const int64_t per_axis = (BLK + 2 * reach) / (int64_t)P->grid + 4;
  const size_t ncell = (size_t)(per_axis * per_axis * per_axis);
  bc->cell_start = (int*)malloc(sizeof(int) * (ncell + 1));
  bc->seeds = (seed_t*)malloc(sizeof(seed_t) * ncell * 8);
  return bc->seeds;
}
static void cache_free(blockcache* bc) {
  for (int o = 0; o < 3; ++o)
    for (int c = 0; c < 3; ++c) free(bc->lat[o][c]);
  free(bc->cell_start);
  free(bc->seeds);
}

/* label at an arbitrary voxel through a throw-away cache (used for forced-uniform centres) */
static uint32_t label_single(const synth_params* P, const int64_t p[3], blockcache* scratch) {
  int64_t org[3];
  for (int a = 0; a < 3; ++a) org[a] = floordiv(p[a], BLK) * BLK;
  cache_build(P, scratch, org);
  return label_cached(P, scratch, p);
}

static void* fill_worker(void* arg) {
  fill_job* J = (fill_job*)arg;
  const synth_params* P = J->P;
  blockcache bc, bc2;
  cache_alloc(P, &bc);
  cache_alloc(P, &bc2);
  int64_t memo_brick[3] = {INT64_MIN, 0, 0};
  uint32_t memo_label = 0;
  const int64_t total = J->nblk[0] * J->nblk[1] * J->nblk[2];
  for (;;) {
    int64_t bi = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
    if (bi >= total) break;
    int64_t bx = bi % J->nblk[0], by = (bi / J->nblk[0]) % J->nblk[1], bz = bi / (J->nblk[0] * J->nblk[1]);
    /* blocks are aligned to the absolute BLK grid so the cache covers them */
    int64_t org[3] = {floordiv(J->box_org[0], BLK) * BLK + bx * BLK, floordiv(J->box_org[1], BLK) * BLK + by * BLK,
                      floordiv(J->box_org[2], BLK) * BLK + bz * BLK};
    cache_build(P, &bc, org);
    for (int z = 0; z < BLK; ++z) {
      int64_t pz = org[2] + z;
      if (pz < J->box_org[2] || pz >= J->box_org[2] + J->box_n[2]) continue;
      for (int y = 0; y < BLK; ++y) {
        int64_t py = org[1] + y;
        if (py < J->box_org[1] || py >= J->box_org[1] + J->box_n[1]) continue;
        for (int x = 0; x < BLK; ++x) {
          int64_t px = org[0] + x;
          if (px < J->box_org[0] || px >= J->box_org[0] + J->box_n[0]) continue;
          int64_t p[3] = {px, py, pz};
          uint32_t lab;
          int forced = 0;
          if (P->uniform_brick) {
            int64_t ub = P->uniform_brick, b3[3];
            for (int a = 0; a < 3; ++a) b3[a] = floordiv(p[a], ub);
            if ((hash5(P->seed, TAG_UNI, b3[0], b3[1], b3[2], 0) >> 48) < P->uniform_q16) {
              if (b3[0] != memo_brick[0] || b3[1] != memo_brick[1] || b3[2] != memo_brick[2]) {
                int64_t c[3];
                for (int a = 0; a < 3; ++a) c[a] = b3[a] * ub + ub / 2;
                memo_label = label_single(P, c, &bc2);
                for (int a = 0; a < 3; ++a) memo_brick[a] = b3[a];
              }
              lab = memo_label;
              forced = 1;
            }
          }
          if (!forced) lab = label_cached(P, &bc, p);
          size_t o = ((size_t)(pz - J->box_org[2]) * J->box_n[1] + (size_t)(py - J->box_org[1])) * J->box_n[0] + (size_t)(px - J->box_org[0]);
          J->out[o] = lab;
        }
      }
    }
  }
  cache_free(&bc);
  cache_free(&bc2);
  return NULL;
}

/* The 256-entry log-normal multiplier table of the power-diagram weights (for the GPU generator,
 * which must use the same values). */
const uint32_t* synth_lognorm_table(void) { return LOGNORM_Q16; }

/* Fill out[nz][ny][nx] (x fastest) with the labels of the box starting at (x0, y0, z0).
 * Voxels outside dims are generated too (the definition extends to all integer points).
 * Returns 0 on success, -1 on bad parameters. */
int synth_fill(const synth_params* P, int64_t x0, int64_t y0, int64_t z0, uint32_t nx, uint32_t ny, uint32_t nz,
               uint32_t* out, int nthreads) {
  if (!P || !out || P->grid < 4 || P->lambda_q16 == 0 || P->lambda_q16 > (8u << 16)) return -1;
  if (P->amp_q16 > (8u << 16)) return -1;
  fill_job J;
  J.P = P;
  J.box_org[0] = x0; J.box_org[1] = y0; J.box_org[2] = z0;
  J.box_n[0] = nx; J.box_n[1] = ny; J.box_n[2] = nz;
  J.out = out;
  int64_t lo[3] = {floordiv(x0, BLK), floordiv(y0, BLK), floordiv(z0, BLK)};
  int64_t hi[3] = {floordiv(x0 + nx - 1, BLK), floordiv(y0 + ny - 1, BLK), floordiv(z0 + nz - 1, BLK)};
  for (int a = 0; a < 3; ++a) J.nblk[a] = hi[a] - lo[a] + 1;
  J.next = 0;
  if (nx == 0 || ny == 0 || nz == 0) return 0;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, fill_worker, &J);
  fill_worker(&J);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  return 0;
}
