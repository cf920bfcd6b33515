/*
 * The seeded synthetic segmentation volumes of synth.c, generated on the GPU.
 *
 * Input generation only (no compression arithmetic): the same definition of label(p) as synth.c
 * (hash-grid seeds, 3-octave value-noise displacement, nearest seed or power-diagram cell,
 * forced-uniform bricks), the same integer / Q16.16 arithmetic in the same order, so every voxel
 * equals the CPU generator's. It exists because the large benchmark volumes (up to 4096^3
 * voxels) take the CPU generator hours; the tests compare the two on sampled boxes.
 *
 * One thread block per 16^3 region of the requested box (aligned to the absolute 16-voxel grid,
 * like the CPU generator's blocks): the block first caches the noise lattice values and the
 * seeds of the hash-grid cells around the region in shared memory, then each thread labels its
 * voxels. Regions whose forced-uniform brick is selected take the label at the brick centre,
 * computed from a cache built around the centre (the brick edge must be a multiple of 16).
 */
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

struct Params {
  uint32_t dims[3];
  uint32_t grid;
  uint64_t seed;
  uint32_t lambda_q16, bg_q16, amp_q16, rmean_q16, uniform_brick, uniform_q16;
};

struct Seed {
  int32_t pos[3];  // Q16.16
  uint32_t gidx;
  int64_t w;       // Q32.32
  uint32_t label;
  uint32_t pad;
};

constexpr int BLK = 16;
constexpr int NT = 256;
constexpr int MAX_CELLS = 343;  // hash-grid cells around a block: ((BLK + 2 reach) / grid + 4)^3 at most
// noise octaves o = 0, 1, 2: lattice period 16 >> o; lattice points per axis around a block
// BLK / period + 2; per component the octaves' points follow one another
__host__ __device__ constexpr int period_of(int o) { return 16 >> o; }
__host__ __device__ constexpr int lat_n(int o) { return BLK / (16 >> o) + 2; }
__host__ __device__ constexpr int lat_off(int o) { return o == 0 ? 0 : (o == 1 ? 27 : 27 + 64); }
constexpr int LAT_POINTS = 27 + 64 + 216;
enum { TAG_COUNT = 1, TAG_POS = 2, TAG_BG = 5, TAG_W = 6, TAG_UNI = 7, TAG_NOISE = 16 };

__constant__ uint32_t c_lognorm[256];

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t hash5(uint64_t seed, uint64_t tag, int64_t a, int64_t b, int64_t c, uint64_t k) {
  uint64_t h = mix64(seed ^ (tag << 56));
  h = mix64(h ^ (uint64_t)a);
  h = mix64(h ^ (uint64_t)b);
  h = mix64(h ^ (uint64_t)c);
  return mix64(h ^ k);
}
__device__ __forceinline__ uint32_t perm32(uint32_t x, uint32_t key) {
  x ^= key;
  x *= 0x7FEB352Du; x ^= x >> 15;
  x *= 0x846CA68Bu; x ^= x >> 16;
  x += key * 0x9E3779B9u; x ^= x >> 13;
  x *= 0xC2B2AE35u; x ^= x >> 16;
  return x;
}
__device__ __forceinline__ int64_t floordiv(int64_t a, int64_t b) {  // b > 0
  const int64_t q = a / b;
  return (a % b != 0 && a < 0) ? q - 1 : q;
}
__device__ __forceinline__ int32_t lerp_q16(int32_t a, int32_t b, int32_t t) {
  return a + (int32_t)(((int64_t)(b - a) * t) / 65536);
}

struct Cache {
  int64_t org[3];
  int64_t lat_org[3][3];
  int64_t cell_org[3];
  int cell_n[3];
  int n_seeds;
};

// Builds the caches of the 16^3 block at org (all threads; ends with a barrier).
__device__ void cache_build(const Params& P, const int64_t org[3], Cache& C, int32_t* lat, int* cell_start,
                            Seed* seeds, int* s_count) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int a = 0; a < 3; ++a) C.org[a] = org[a];
    for (int o = 0; o < 3; ++o)
      for (int a = 0; a < 3; ++a) C.lat_org[o][a] = floordiv(org[a], period_of(o));
    const int64_t g = P.grid, reach = ((int64_t)P.amp_q16 >> 16) + 2;
    for (int a = 0; a < 3; ++a) {
      const int64_t lo = floordiv(org[a] - reach, g) - 1, hi = floordiv(org[a] + BLK + reach, g) + 1;
      C.cell_org[a] = lo;
      C.cell_n[a] = (int)(hi - lo + 1);
    }
  }
  __syncthreads();
  // noise lattice values of the 3 octaves x 3 components
  for (int i = tid; i < 3 * LAT_POINTS; i += NT) {
    const int comp = i / LAT_POINTS, pt = i % LAT_POINTS;
    const int o = pt < 27 ? 0 : (pt < 27 + 64 ? 1 : 2);
    const int n = lat_n(o), li = pt - lat_off(o);
    const int x = li % n, y = (li / n) % n, z = li / (n * n);
    const uint64_t h = hash5(P.seed, (uint64_t)(TAG_NOISE + o * 3 + comp), C.lat_org[o][0] + x, C.lat_org[o][1] + y,
                             C.lat_org[o][2] + z, 0);
    lat[i] = (int32_t)((h >> 47) & 0x1FFFF) - 65536;
  }
  // seeds of the cells around the block: counts first, then an exclusive scan, then the seeds
  const int ncell = C.cell_n[0] * C.cell_n[1] * C.cell_n[2];
  const uint64_t pq32 = (uint64_t)P.lambda_q16 << 13;
  for (int ci = tid; ci < ncell; ci += NT) {
    const int64_t cx = C.cell_org[0] + ci % C.cell_n[0], cy = C.cell_org[1] + (ci / C.cell_n[0]) % C.cell_n[1],
                  cz = C.cell_org[2] + ci / (C.cell_n[0] * C.cell_n[1]);
    int n = 0;
    for (int t = 0; t < 8; ++t)
      if ((hash5(P.seed, TAG_COUNT, cx, cy, cz, (uint64_t)t) >> 32) < pq32) ++n;
    cell_start[ci] = n;
  }
  __syncthreads();
  if (tid == 0) {
    int total = 0;
    for (int ci = 0; ci < ncell; ++ci) {
      const int n = cell_start[ci];
      cell_start[ci] = total;
      total += n;
    }
    cell_start[ncell] = total;
    *s_count = total;
  }
  __syncthreads();
  const int64_t g = P.grid;
  const int64_t ngx = (P.dims[0] + g - 1) / g + 2, ngy = (P.dims[1] + g - 1) / g + 2;
  const uint32_t key = (uint32_t)mix64(P.seed ^ 0xABCDEF12345ull);
  const int64_t cell_q16 = g << 16;
  for (int ci = tid; ci < ncell; ci += NT) {
    const int64_t c[3] = {C.cell_org[0] + ci % C.cell_n[0], C.cell_org[1] + (ci / C.cell_n[0]) % C.cell_n[1],
                          C.cell_org[2] + ci / (C.cell_n[0] * C.cell_n[1])};
    const uint64_t lin = (uint64_t)(((c[2] + 1) * ngy + (c[1] + 1)) * ngx + (c[0] + 1));
    for (int k = 0, s = cell_start[ci]; s < cell_start[ci + 1]; ++k, ++s) {
      Seed& sd = seeds[s];
      for (int a = 0; a < 3; ++a)
        sd.pos[a] = (int32_t)(c[a] * cell_q16 +
                              (int64_t)(hash5(P.seed, TAG_POS + (a << 2), c[0], c[1], c[2], (uint64_t)k) % (uint64_t)cell_q16));
      const uint64_t gidx = lin * 8u + (uint64_t)k;
      sd.gidx = (uint32_t)gidx;
      uint32_t id = perm32((uint32_t)gidx, key);
      if ((hash5(P.seed, TAG_BG, c[0], c[1], c[2], (uint64_t)k) >> 48) < P.bg_q16) id = 0;
      sd.label = id;
      sd.w = 0;
      if (P.rmean_q16) {
        const uint64_t m = c_lognorm[hash5(P.seed, TAG_W, c[0], c[1], c[2], (uint64_t)k) >> 56];
        const int64_t r = (int64_t)(((uint64_t)P.rmean_q16 * m) >> 16);
        sd.w = r * r;
      }
    }
  }
  __syncthreads();
}

__device__ int32_t noise_at(const Cache& C, const int32_t* lat, int o, int comp, const int64_t p[3]) {
  const int per = period_of(o), n = lat_n(o);
  int32_t t[3];
  int i[3];
  for (int a = 0; a < 3; ++a) {
    const int64_t q = floordiv(p[a], per);
    i[a] = (int)(q - C.lat_org[o][a]);
    t[a] = (int32_t)((p[a] - q * per) * (65536 / per));
  }
  const int32_t* L = lat + comp * LAT_POINTS + lat_off(o);
#define LV(dx, dy, dz) L[((i[2] + (dz)) * n + (i[1] + (dy))) * n + (i[0] + (dx))]
  const int32_t x00 = lerp_q16(LV(0, 0, 0), LV(1, 0, 0), t[0]);
  const int32_t x10 = lerp_q16(LV(0, 1, 0), LV(1, 1, 0), t[0]);
  const int32_t x01 = lerp_q16(LV(0, 0, 1), LV(1, 0, 1), t[0]);
  const int32_t x11 = lerp_q16(LV(0, 1, 1), LV(1, 1, 1), t[0]);
#undef LV
  return lerp_q16(lerp_q16(x00, x10, t[1]), lerp_q16(x01, x11, t[1]), t[2]);
}

__device__ uint32_t label_cached(const Params& P, const Cache& C, const int32_t* lat, const int* cell_start,
                                 const Seed* seeds, const int64_t p[3]) {
  const int64_t A = P.amp_q16;
  const int64_t amp[3] = {A * 4 / 7, A * 2 / 7, A / 7};
  int64_t q[3];
  for (int a = 0; a < 3; ++a) {
    int64_t d = 0;
    for (int o = 0; o < 3; ++o) d += amp[o] * noise_at(C, lat, o, a, p) / 65536;
    q[a] = (p[a] << 16) + 32768 + d;
  }
  const int64_t g = P.grid;
  int64_t gc[3];
  for (int a = 0; a < 3; ++a) gc[a] = floordiv(q[a], g << 16);
  int64_t best = INT64_MAX;
  uint32_t best_idx = 0xFFFFFFFFu, best_label = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int x = (int)(gc[0] + dx - C.cell_org[0]), y = (int)(gc[1] + dy - C.cell_org[1]),
                  z = (int)(gc[2] + dz - C.cell_org[2]);
        const int ci = (z * C.cell_n[1] + y) * C.cell_n[0] + x;
        for (int s = cell_start[ci]; s < cell_start[ci + 1]; ++s) {
          const Seed& sd = seeds[s];
          const int64_t e0 = q[0] - sd.pos[0], e1 = q[1] - sd.pos[1], e2 = q[2] - sd.pos[2];
          const int64_t sc = e0 * e0 + e1 * e1 + e2 * e2 - sd.w;
          if (sc < best || (sc == best && sd.gidx < best_idx)) {
            best = sc;
            best_idx = sd.gidx;
            best_label = sd.label;
          }
        }
      }
  return best_label;
}

// out: the box [x0, x0 + nx) x [y0, y0 + ny) x [z0, z0 + nz), x fastest; one block per 16^3 region
// of the absolute grid that meets the box.
__global__ void __launch_bounds__(NT) fill_kernel(const Params P, int64_t x0, int64_t y0, int64_t z0, uint32_t nx,
                                                  uint32_t ny, uint32_t nz, int64_t rx0, int64_t ry0, int64_t rz0,
                                                  uint32_t nrx, uint32_t nry, uint32_t* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Cache C;
  __shared__ int s_count;
  __shared__ uint32_t s_label;
  Seed* seeds = reinterpret_cast<Seed*>(smem);
  int32_t* lat = reinterpret_cast<int32_t*>(smem + sizeof(Seed) * 8 * MAX_CELLS);
  int* cell_start = lat + 3 * LAT_POINTS;
  const uint64_t bi = blockIdx.x;
  const int64_t org[3] = {(rx0 + (int64_t)(bi % nrx)) * BLK, (ry0 + (int64_t)((bi / nrx) % nry)) * BLK,
                          (rz0 + (int64_t)(bi / ((uint64_t)nrx * nry))) * BLK};
  bool forced = false;
  if (P.uniform_brick) {
    const int64_t ub = P.uniform_brick;
    int64_t b3[3];
    for (int a = 0; a < 3; ++a) b3[a] = floordiv(org[a], ub);
    if ((hash5(P.seed, TAG_UNI, b3[0], b3[1], b3[2], 0) >> 48) < P.uniform_q16) {
      forced = true;
      int64_t c[3], corg[3];
      for (int a = 0; a < 3; ++a) {
        c[a] = b3[a] * ub + ub / 2;
        corg[a] = floordiv(c[a], BLK) * BLK;
      }
      cache_build(P, corg, C, lat, cell_start, seeds, &s_count);
      if (threadIdx.x == 0) s_label = label_cached(P, C, lat, cell_start, seeds, c);
      __syncthreads();
    }
  }
  if (!forced) cache_build(P, org, C, lat, cell_start, seeds, &s_count);
  for (int v = threadIdx.x; v < BLK * BLK * BLK; v += NT) {
    const int64_t p[3] = {org[0] + (v & 15), org[1] + ((v >> 4) & 15), org[2] + (v >> 8)};
    if (p[0] < x0 || p[0] >= x0 + nx || p[1] < y0 || p[1] >= y0 + ny || p[2] < z0 || p[2] >= z0 + nz) continue;
    const uint32_t lab = forced ? s_label : label_cached(P, C, lat, cell_start, seeds, p);
    out[((uint64_t)(p[2] - z0) * ny + (uint64_t)(p[1] - y0)) * nx + (uint64_t)(p[0] - x0)] = lab;
  }
}

int64_t host_floordiv(int64_t a, int64_t b) {
  const int64_t q = a / b;
  return (a % b != 0 && a < 0) ? q - 1 : q;
}

}  // namespace

extern "C" {

/* Copies the 256-entry log-normal table of the power-diagram weights (synth.c) to the device. */
int synth_gpu_set_lognorm(const uint32_t* table) {
  return cudaMemcpyToSymbol(c_lognorm, table, sizeof(uint32_t) * 256) == cudaSuccess ? 0 : -2;
}

/* Fills the device array out[nz][ny][nx] with the labels of the box at (x0, y0, z0), as synth_fill
 * does on the CPU; asynchronous on `stream`. The parameter struct has synth.c's layout. Returns 0,
 * -1 on bad parameters (grid < 8, lambda out of (0, 8], forced-uniform brick edge not a multiple
 * of 16) or -2 on a CUDA error. */
int synth_fill_gpu(const void* params, int64_t x0, int64_t y0, int64_t z0, uint32_t nx, uint32_t ny, uint32_t nz,
                   uint32_t* out, void* stream) {
  const Params& P = *static_cast<const Params*>(params);
  if (!out || P.grid < 8 || P.lambda_q16 == 0 || P.lambda_q16 > (8u << 16) || P.amp_q16 > (8u << 16)) return -1;
  if (P.uniform_brick && P.uniform_brick % BLK) return -1;
  const int64_t reach = ((int64_t)P.amp_q16 >> 16) + 2, per_axis = (BLK + 2 * reach) / (int64_t)P.grid + 4;
  if (per_axis * per_axis * per_axis > MAX_CELLS) return -1;
  const uint64_t g = P.grid;  // global seed indices (8 per padded grid cell) must fit 32 bits
  if (((P.dims[0] + g - 1) / g + 2) * ((P.dims[1] + g - 1) / g + 2) * ((P.dims[2] + g - 1) / g + 3) * 8ull >= (1ull << 32))
    return -1;
  if (nx == 0 || ny == 0 || nz == 0) return 0;
  const int64_t rx0 = host_floordiv(x0, BLK), ry0 = host_floordiv(y0, BLK), rz0 = host_floordiv(z0, BLK);
  const uint32_t nrx = (uint32_t)(host_floordiv(x0 + nx - 1, BLK) - rx0 + 1);
  const uint32_t nry = (uint32_t)(host_floordiv(y0 + ny - 1, BLK) - ry0 + 1);
  const uint32_t nrz = (uint32_t)(host_floordiv(z0 + nz - 1, BLK) - rz0 + 1);
  const uint64_t nblocks = (uint64_t)nrx * nry * nrz;
  if (nblocks > 0x7FFFFFFFull) return -1;
  const size_t smem = sizeof(Seed) * 8 * MAX_CELLS + sizeof(int32_t) * 3 * LAT_POINTS + sizeof(int) * (MAX_CELLS + 1);
  if (cudaFuncSetAttribute(fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -2;
  fill_kernel<<<(unsigned)nblocks, NT, smem, static_cast<cudaStream_t>(stream)>>>(P, x0, y0, z0, nx, ny, nz, rx0, ry0, rz0,
                                                                                 nrx, nry, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // extern "C"
