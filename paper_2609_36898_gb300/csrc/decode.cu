// Brick decoder kernels for sm_103a: CSGV operation streams -> uint32 label bricks.
//
// The Decompress stage works on all requested bricks in parallel (Results, "GPU-based rendering
// pipeline"). Here the work of one brick is split into two kernels so that each runs at the
// parallelism it needs:
//
//  A. rans_symbols_kernel (rANS volumes only): one warp per brick, 16 bricks per block. The 32
//     interleaved states decode one symbol each per step; the lanes whose state fell below 2^16
//     take the next 16-bit words in lane order (ballot + popc ranks). The symbols (two per byte,
//     the same layout as the plain coder) go to a stream-ordered workspace. Decoding is a serial
//     chain per brick, so many bricks per SM hide its latency.
//
//  B. reconstruct kernels: one thread block per brick (grid) or persistent blocks pulling bricks
//     from a work counter with a bulk-copy prefetch of the next brick's record (batched):
//       1. parse: the symbol stream alternates between operations and the delta entries that
//          follow a delta operation (Methods, "Compressed segmentation volumes"). Threads
//          summarise byte-sized chunks with a 2-state table for both start states, a warp scan
//          composes the summaries, and a second pass writes the node-indexed operations (8 per
//          u32) and the delta values. Bricks without delta operations skip this: their symbols
//          are the node operations.
//       2. palette cursor: per 32 nodes, SWAR masks of advance / delta operations and exclusive
//          prefix counts, so that any node's cursor k_j is one popc away (Supplementary Fig.
//          "CSGV ablation" caption: advance reads the next entry, last re-reads it, delta re-reads
//          the entry delta back).
//       3. coarse levels 0..L-1: a dense Morton-indexed grid per level of palette indices G and of
//          ranks R among the level's stop-0 nodes (level l+1 emits the 8 children of each, in rank
//          order; Results, "CSGV results"). Neighbour copies are written as marks and resolved by
//          walking at most three hops (each hop turns an even coordinate odd, and a copy needs an
//          even one), so no extra rounds or barriers are needed.
//       4. finest level: one pass over the level-(L-1) cells writes each 2^3 block of the
//          finest grid (a byte or u16 palette index per voxel): constant blocks in four stores,
//          emitted blocks from their 8 operations at once. A second pass reads four voxels,
//          resolves any neighbour marks, maps indices to labels and writes 16 bytes per thread.
// Every rule of the format is checked on the way; the first error of a request goes to the
// caller's status buffer (no traps).
#include "decode_kernels.cuh"

namespace vc {

void* pick_kernel_nt256(uint32_t L, bool gt16, bool rans, bool batched);
void* pick_kernel_nt512(uint32_t L, bool gt16, bool rans, bool batched);
void* pick_kernel_nt1024(uint32_t L, bool gt16, bool rans, bool batched);

namespace {

using namespace dev;

// ------------------------------------------------------------------------------------------
// rANS symbols: one warp per request item. The record's coded words are copied to the warp's
// shared buffer; each step decodes 32 symbols (symbol i on state i mod 32) and writes 16 bytes.
__global__ void __launch_bounds__(32 * kRansWarps) rans_symbols_kernel(const __grid_constant__ Params P,
                                                                      uint8_t* ws) {
  extern __shared__ __align__(128) unsigned char sm[];
  const SmemLayout& SL = P.v.sm;
  uint32_t* tab = reinterpret_cast<uint32_t*>(sm);
  for (uint32_t i = threadIdx.x; i < kRansM; i += 32u * kRansWarps) tab[i] = P.v.rans_tab[i];
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t item = P.item_base + blockIdx.x * kRansWarps + warp;
  if (item >= P.n) return;
  const uint32_t brick = P.ids[item];
  if (brick >= P.v.n_bricks) return;  // reported by the reconstruction kernel
  const uint32_t* rec = P.v.records + P.v.starts[brick];
  const uint32_t np = rec[0], S = rec[1], cb = rec[2];
  const uint32_t ns = S < 32u ? S : 32u;
  const uint32_t nw = cb >> 1;
  // copy the coded bytes (16-byte aligned span) into this warp's buffer
  const uint32_t cofs = 16u + 4u * ns + 4u * np;
  const uint32_t a0 = cofs & ~15u, a1 = (cofs + cb + 15u) & ~15u;
  unsigned char* buf = sm + 4u * kRansM + warp * SL.a_buf;
  const uint16_t* words;
  if (a1 - a0 <= SL.a_buf) {
    const uint4* src = reinterpret_cast<const uint4*>(reinterpret_cast<const unsigned char*>(rec) + a0);
    uint4* dst = reinterpret_cast<uint4*>(buf);
    for (uint32_t i = lane; i < (a1 - a0) / 16u; i += 32u) dst[i] = src[i];
    __syncwarp();
    words = reinterpret_cast<const uint16_t*>(buf + (cofs - a0));
  } else {
    words = reinterpret_cast<const uint16_t*>(reinterpret_cast<const unsigned char*>(rec) + cofs);
  }
  uint8_t* out = ws + (size_t)item * SL.ws_stride;
  uint32_t x = lane < ns ? rec[4 + lane] : (1u << 16);
  bool bad = lane < ns && x < (1u << 16);
  uint32_t ptr = 0;
  for (uint32_t base = 0; base < S; base += 32u) {
    const uint32_t i = base + lane;
    const bool active = i < S;
    uint32_t s = 0;
    if (active) {
      const uint32_t e = tab[x & (kRansM - 1u)];
      s = e & 15u;
      x = ((e >> 4) & 0x1FFFu) * (x >> 12) + (e >> 17);
    }
    const bool need = active && x < (1u << 16);
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, need);
    if (need) {
      const uint32_t at = ptr + __popc(m & lanemask_lt());
      if (at < nw) x = (x << 16) | (uint32_t)words[at];
      else bad = true;
    }
    ptr += __popc(m);
    const uint32_t hi = __shfl_xor_sync(0xFFFFFFFFu, s, 1);
    if (active && !(lane & 1u)) out[i >> 1] = (uint8_t)(s | (i + 1 < S ? hi << 4 : 0u));
  }
  if (ptr != nw) bad = true;
  if (lane < ns && x != (1u << 16)) bad = true;
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) report(P.status, VC_ERR_CORRUPT, item);
}

// ------------------------------------------------------------------------------------------
void* pick_kernel(uint32_t L, uint32_t threads, bool gt16, bool rans, bool batched) {
  switch (threads) {
    case 256: return pick_kernel_nt256(L, gt16, rans, batched);
    case 512: return pick_kernel_nt512(L, gt16, rans, batched);
    case 1024: return pick_kernel_nt1024(L, gt16, rans, batched);
    default: return nullptr;
  }
}

uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

}  // namespace

bool schedule_supported(uint32_t L, uint32_t threads) {
  if (L < 1 || L > 5) return false;
  if (threads == 256) return true;
  return (threads == 512 || threads == 1024) && L >= 4;
}

vc_status compute_layout(const Volume& v, int device, uint32_t threads, uint32_t nstage, SmemLayout* out) {
  const uint32_t L = v.L;
  if (!schedule_supported(L, threads) || nstage < 1 || nstage > 2) return VC_ERR_UNSUPPORTED;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess)
    return VC_ERR_CUDA;
  SmemLayout s{};
  s.gt_bytes = v.max_pal < kMaxIdx8 ? 1u : 2u;
  const uint32_t b = 1u << L;
  const uint32_t ncells = ((1u << (3 * L)) - 1u) / 7u;  // levels 0..L-1
  const uint32_t stream_words = (v.max_sym + 7u) / 8u;
  uint32_t o = 0;
  s.misc_off = o; o += 512;
  s.lut_off = o; o += 1024;
  s.nwords = (v.max_sym + 31u) / 32u + 2u;
  s.mask_off = o; o += align16(4 * 4 * s.nwords);
  s.nodes_words = stream_words + 4u;
  s.nodes_off = o; o += v.max_delta ? align16(4 * s.nodes_words) : 0u;
  s.dlist_cap = v.max_delta;
  s.dlist_off = o; o += align16(4 * (v.max_delta ? v.max_delta : 1u));
  s.g_off = o; o += align16(s.gt_bytes * ncells);
  const uint32_t ncells_r = ((1u << (3 * (L - 1))) - 1u) / 7u;  // ranks are stored for levels 0..L-2
  s.r_off = o; o += align16(2 * (ncells_r ? ncells_r : 1u));
  // the finest grid also hosts the general parse path's summaries (9 NT words, padded)
  s.fg_off = o; o += align16(std::max<uint32_t>(s.gt_bytes * b * b * b, 4u * (9u * threads + 64u)));
  s.list_off = o; o += align16(2u << (3 * (L - 1)));  // rank -> cell of the stop-0 level-(L-1) cells
  const uint32_t fixed = o;
  uint32_t stage = align16(v.max_stage) + 16u;  // slack for 8-nibble windows at the end
  if (fixed + nstage * stage > (uint32_t)optin) stage = 0;
  s.stage_bytes = stage;
  s.nstage = nstage;
  s.stage_off = o; o += nstage * stage;
  s.total = o;
  if (s.total > (uint32_t)optin) return VC_ERR_UNSUPPORTED;
  // rANS symbol kernel: table + one coded-word buffer per warp
  s.ws_stride = align16((v.max_sym + 1u) / 2u) + 16u;
  s.a_buf = align16(4u * v.max_rec_words);
  if (4u * kRansM + kRansWarps * s.a_buf > (uint32_t)optin) s.a_buf = 0;
  s.a_smem = 4u * kRansM + kRansWarps * s.a_buf;
  *out = s;
  return VC_OK;
}

vc_status launch_decode(const Volume& v, const uint32_t* ids, uint32_t n, const uint32_t* slots, uint32_t* cache,
                        uint32_t lod, uint32_t mode, int32_t* status, cudaStream_t stream) {
  if (n == 0) return VC_OK;
  const bool rans = v.coder == 1;
  const bool batched = mode == VC_MODE_BATCHED;
  const uint32_t nt = v.sched.threads;
  void* k = pick_kernel(v.L, nt, v.dv.sm.gt_bytes == 2, rans, batched);
  if (!k) return VC_ERR_UNSUPPORTED;
  const uint32_t smem = v.dv.sm.total;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return VC_ERR_CUDA;
  Params P;
  P.v = v.dv;
  P.ids = ids;
  P.slots = slots;
  P.n = n;
  P.cache = cache;
  P.lod = lod;
  P.status = status;
  P.item_base = 0;
  P.ws = nullptr;
  uint8_t* ws = nullptr;
  if (rans) {
    if (cudaMallocAsync(reinterpret_cast<void**>(&ws), (size_t)n * v.dv.sm.ws_stride, stream) != cudaSuccess) {
      cudaGetLastError();
      return VC_ERR_OOM;
    }
    P.ws = ws;
    void* ka = reinterpret_cast<void*>(&rans_symbols_kernel);
    if (cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.dv.sm.a_smem) != cudaSuccess) {
      cudaFreeAsync(ws, stream);
      return VC_ERR_CUDA;
    }
  }
  vc_status rc = VC_OK;
  auto run_symbols = [&](uint32_t base, uint32_t count) -> bool {
    if (!rans) return true;
    Params PA = P;
    PA.item_base = base;
    PA.n = base + count;
    void* args[] = {&PA, &ws};
    const uint32_t blocks = (count + kRansWarps - 1) / kRansWarps;
    return cudaLaunchKernel(reinterpret_cast<void*>(&rans_symbols_kernel), dim3(blocks), dim3(32 * kRansWarps), args,
                            v.dv.sm.a_smem, stream) == cudaSuccess;
  };
  void* args[] = {&P};
  if (mode == VC_MODE_PLAIN) {
    for (uint32_t i = 0; i < n && rc == VC_OK; ++i) {
      P.item_base = i;
      if (!run_symbols(i, 1) || cudaLaunchKernel(k, dim3(1), dim3(nt), args, smem, stream) != cudaSuccess)
        rc = VC_ERR_CUDA;
    }
  } else if (mode == VC_MODE_GRID) {
    if (!run_symbols(0, n) || cudaLaunchKernel(k, dim3(n), dim3(nt), args, smem, stream) != cudaSuccess)
      rc = VC_ERR_CUDA;
  } else {
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, v.device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)nt, smem) != cudaSuccess) {
      rc = VC_ERR_CUDA;
    } else if (per_sm < 1) {
      rc = VC_ERR_UNSUPPORTED;
    } else {
      if (v.sched.blocks_per_sm) per_sm = std::min<int>(per_sm, (int)v.sched.blocks_per_sm);
      const uint32_t grid = std::min<uint32_t>(n, (uint32_t)(sms * per_sm));
      if (!run_symbols(0, n) ||
          cudaMemsetAsync(reinterpret_cast<uint32_t*>(status) + 2, 0, sizeof(uint32_t), stream) != cudaSuccess ||
          cudaLaunchKernel(k, dim3(grid), dim3(nt), args, smem, stream) != cudaSuccess)
        rc = VC_ERR_CUDA;
    }
  }
  if (ws) cudaFreeAsync(ws, stream);
  return rc;
}

}  // namespace vc
