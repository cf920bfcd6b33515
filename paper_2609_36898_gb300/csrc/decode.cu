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
#include <cuda_runtime.h>

#include <algorithm>

#include "vc_internal.h"

namespace vc {

namespace {

constexpr uint16_t NONE16 = 0xFFFFu;
enum : uint32_t { OP_PARENT = 0, OP_NX = 1, OP_NY = 2, OP_NZ = 3, OP_ADV = 4, OP_LAST = 5, OP_DELTA = 6 };

struct Params {
  DevVolume v;
  const uint32_t* ids;
  const uint32_t* slots;
  uint32_t n;
  uint32_t* cache;
  uint32_t lod;
  int32_t* status;
  uint32_t item_base;
  const uint8_t* ws;  // decoded rANS symbols, ws_stride bytes per item (nullptr for plain volumes)
};

template <typename GT>
struct GridT {
  static constexpr uint32_t MARK = sizeof(GT) == 1 ? 0xFDu : 0xFFFDu;  // MARK + axis: pending copy
};

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // bit i -> bit 3i
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0xFF0000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__device__ __forceinline__ uint32_t compact3(uint32_t v) {  // bit 3i -> bit i
  v &= 0x09249249u;
  v = (v ^ (v >> 2)) & 0x030C30C3u;
  v = (v ^ (v >> 4)) & 0x0300F00Fu;
  v = (v ^ (v >> 8)) & 0xFF0000FFu;
  v = (v ^ (v >> 16)) & 0x000003FFu;
  return v;
}
// Morton code m minus one step along axis a (the coordinate must be > 0).
__device__ __forceinline__ uint32_t morton_dec(uint32_t m, uint32_t a) {
  const uint32_t ma = 0x09249249u << a;
  return (((m & ma) - 1u) & ma) | (m & ~ma);
}

__device__ __forceinline__ void set_err(int* s_err, int code) { *s_err = code; }

__device__ void report(int32_t* status, int code, uint32_t item) {
  if (atomicCAS(reinterpret_cast<int*>(status), 0, code) == 0) atomicExch(reinterpret_cast<int*>(status) + 1, (int)item);
}

__device__ __forceinline__ uint32_t nib_at(const uint32_t* w, uint32_t i) { return (w[i >> 3] >> ((i & 7u) << 2)) & 15u; }

// 8 nibbles starting at nibble j of a packed array (two aligned loads and a funnel shift).
__device__ __forceinline__ uint32_t nib8_at(const uint32_t* w, uint32_t j) {
  const uint32_t lo = w[j >> 3], hi = w[(j >> 3) + 1];
  return __funnelshift_r(lo, hi, (j & 7u) << 2);
}
// 8 bits starting at bit j of a bit array.
__device__ __forceinline__ uint32_t bits8_at(const uint32_t* w, uint32_t j) {
  const uint32_t lo = w[j >> 5], hi = w[(j >> 5) + 1];
  return __funnelshift_r(lo, hi, j & 31u) & 0xFFu;
}
// bit i set iff (nibble i & 7) == v, for the 8 nibbles of x
__device__ __forceinline__ uint32_t nib_eq8(uint32_t x, uint32_t v) {
  const uint32_t t = (x & 0x77777777u) ^ (v * 0x11111111u);
  uint32_t z = ~(t + 0x77777777u) & 0x88888888u;
  z >>= 3;
  z = (z | (z >> 3)) & 0x03030303u;
  z = (z | (z >> 6)) & 0x000F000Fu;
  z = (z | (z >> 12)) & 0xFFu;
  return z;
}

// Inclusive warp scan of two counters.
__device__ __forceinline__ void warp_scan2(uint32_t& a, uint32_t& b, uint32_t lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t na = __shfl_up_sync(0xFFFFFFFFu, a, off), nb = __shfl_up_sync(0xFFFFFFFFu, b, off);
    if (lane >= (uint32_t)off) { a += na; b += nb; }
  }
}

// Exclusive block scan of (a, b); tmp holds 2 * NW + 2 words. Ends with a barrier.
template <int NT>
__device__ __forceinline__ void block_scan2(uint32_t a, uint32_t b, uint32_t& pa, uint32_t& pb, uint32_t& ta,
                                            uint32_t& tb, uint32_t* tmp) {
  constexpr uint32_t NW = NT / 32;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t ia = a, ib = b;
  warp_scan2(ia, ib, lane);
  if (lane == 31) { tmp[warp] = ia; tmp[NW + warp] = ib; }
  __syncthreads();
  if (warp == 0) {
    const uint32_t va = lane < NW ? tmp[lane] : 0u, vb = lane < NW ? tmp[NW + lane] : 0u;
    uint32_t sa = va, sb = vb;
    warp_scan2(sa, sb, lane);
    if (lane < NW) { tmp[lane] = sa - va; tmp[NW + lane] = sb - vb; }
    if (lane == 31) { tmp[2 * NW] = sa; tmp[2 * NW + 1] = sb; }
  }
  __syncthreads();
  pa = tmp[warp] + ia - a;
  pb = tmp[NW + warp] + ib - b;
  ta = tmp[2 * NW];
  tb = tmp[2 * NW + 1];
  __syncthreads();
}

// ------------------------------------------------------------------------------------------
// Parse table: entry for (state, byte) after reading its low then high nibble.
// bit 0: end state (1 = a delta entry is expected next); bits 1-2: operations read;
// bits 3-4: delta operations read; bits 5-6: which nibbles are operations; bits 7-8: which nibbles
// are delta operations.
__device__ __forceinline__ uint32_t parse_entry(uint32_t st, uint32_t byte) {
  uint32_t e = 0, nops = 0, ndel = 0;
#pragma unroll
  for (uint32_t h = 0; h < 2; ++h) {
    const uint32_t v = (byte >> (4 * h)) & 15u;
    if (st == 0) {
      ++nops;
      e |= 1u << (5 + h);
      if ((v & 7u) == OP_DELTA) { ++ndel; e |= 1u << (7 + h); st = 1; }
    } else {
      st = (v >> 3) & 1u;  // another entry follows
    }
  }
  return e | st | (nops << 1) | (ndel << 3);
}

// One nibble of the automaton (for a trailing odd symbol).
__device__ __forceinline__ void parse_nibble(uint32_t& st, uint32_t v, uint32_t& nops, uint32_t& ndel) {
  if (st == 0) {
    ++nops;
    if ((v & 7u) == OP_DELTA) { ++ndel; st = 1; }
  } else {
    st = (v >> 3) & 1u;
  }
}

// delta from the entries at nibble i..; 0 when invalid (runs past S or needs an eighth entry)
__device__ __forceinline__ uint32_t read_delta(const uint32_t* sw, uint32_t i, uint32_t S) {
  uint32_t d = 0;
#pragma unroll 1
  for (uint32_t e = 0; e < 7u; ++e) {
    if (i + e >= S) return 0u;
    const uint32_t v = nib_at(sw, i + e);
    d = (d << 3) | (v & 7u);
    if (!(v & 8u)) return d;
  }
  return 0u;
}

struct ParseOut {
  uint32_t n_nodes;
  uint32_t n_delta;
};

// Builds nodes[] (8 operation symbols per u32, zero-padded) and dlist[] from the symbol stream.
template <int NT>
__device__ ParseOut parse_stream(const uint32_t* sw, uint32_t S, uint32_t* nodes, uint32_t nodes_words,
                                 uint32_t* dlist, uint32_t dcap, const uint16_t* lut, uint32_t* sum, int* s_err) {
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t T = (S + 7u) >> 3;  // stream words
  const uint32_t WP = (T + NT - 1) / NT;
  const uint32_t w0 = min(tid * WP, T), w1 = min(w0 + WP, T);
  for (uint32_t w = tid; w < nodes_words; w += NT) nodes[w] = 0u;
  // pass A: summaries for both start states
  uint32_t s0 = 0, s1 = 1, n0 = 0, n1 = 0, d0 = 0, d1 = 0;
  for (uint32_t w = w0; w < w1; ++w) {
    const uint32_t x = sw[w];
    const uint32_t left = S - 8u * w;
    const uint32_t full = left >= 8u ? 4u : (left >> 1);
    for (uint32_t k = 0; k < full; ++k) {
      const uint32_t byte = (x >> (8u * k)) & 0xFFu;
      const uint32_t e0 = lut[s0 * 256u + byte], e1 = lut[s1 * 256u + byte];
      n0 += (e0 >> 1) & 3u; d0 += (e0 >> 3) & 3u; s0 = e0 & 1u;
      n1 += (e1 >> 1) & 3u; d1 += (e1 >> 3) & 3u; s1 = e1 & 1u;
    }
    if (left < 8u && (left & 1u)) {
      const uint32_t v = (x >> (8u * full)) & 15u;
      parse_nibble(s0, v, n0, d0);
      parse_nibble(s1, v, n1, d1);
    }
  }
  // sum layout: [0,NT) end states, then n0, n1, d0, d1, then start state / node base / delta base
  sum[tid] = s0 | (s1 << 1);
  sum[NT + tid] = n0;
  sum[2 * NT + tid] = n1;
  sum[3 * NT + tid] = d0;
  sum[4 * NT + tid] = d1;
  __syncthreads();
  if (warp == 0) {
    constexpr uint32_t PER = NT / 32;
    uint32_t E0 = 0, E1 = 1, N0 = 0, N1 = 0, D0 = 0, D1 = 0;  // identity
    for (uint32_t t = lane * PER; t < lane * PER + PER; ++t) {
      const uint32_t te = sum[t];
      const uint32_t a0 = E0 ? sum[2 * NT + t] : sum[NT + t], b0 = E0 ? sum[4 * NT + t] : sum[3 * NT + t];
      const uint32_t a1 = E1 ? sum[2 * NT + t] : sum[NT + t], b1 = E1 ? sum[4 * NT + t] : sum[3 * NT + t];
      N0 += a0; D0 += b0; E0 = (te >> E0) & 1u;
      N1 += a1; D1 += b1; E1 = (te >> E1) & 1u;
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t pE0 = __shfl_up_sync(0xFFFFFFFFu, E0, off), pE1 = __shfl_up_sync(0xFFFFFFFFu, E1, off);
      const uint32_t pN0 = __shfl_up_sync(0xFFFFFFFFu, N0, off), pN1 = __shfl_up_sync(0xFFFFFFFFu, N1, off);
      const uint32_t pD0 = __shfl_up_sync(0xFFFFFFFFu, D0, off), pD1 = __shfl_up_sync(0xFFFFFFFFu, D1, off);
      if (lane >= (uint32_t)off) {
        // prefix p, then this lane's function c from p's end state
        const uint32_t cE0 = E0, cE1 = E1, cN0 = N0, cN1 = N1, cD0 = D0, cD1 = D1;
        N0 = pN0 + (pE0 ? cN1 : cN0); D0 = pD0 + (pE0 ? cD1 : cD0); E0 = pE0 ? cE1 : cE0;
        N1 = pN1 + (pE1 ? cN1 : cN0); D1 = pD1 + (pE1 ? cD1 : cD0); E1 = pE1 ? cE1 : cE0;
      }
    }
    uint32_t xs = __shfl_up_sync(0xFFFFFFFFu, E0, 1), xn = __shfl_up_sync(0xFFFFFFFFu, N0, 1),
             xd = __shfl_up_sync(0xFFFFFFFFu, D0, 1);
    if (lane == 0) { xs = 0; xn = 0; xd = 0; }
    for (uint32_t t = lane * PER; t < lane * PER + PER; ++t) {
      const uint32_t te = sum[t];
      const uint32_t tn = xs ? sum[2 * NT + t] : sum[NT + t], td = xs ? sum[4 * NT + t] : sum[3 * NT + t];
      sum[5 * NT + t] = xs;
      sum[6 * NT + t] = xn;
      sum[7 * NT + t] = xd;
      xn += tn; xd += td; xs = (te >> xs) & 1u;
    }
    if (lane == 31) {
      sum[8 * NT] = xn;
      sum[8 * NT + 1] = xd;
      if (xs != 0) set_err(s_err, VC_ERR_CORRUPT);  // the stream ends inside a delta entry chain
    }
  }
  __syncthreads();
  // pass B: node symbols and delta values
  uint32_t st = sum[5 * NT + tid];
  const uint32_t jstart = sum[6 * NT + tid];
  uint32_t j = jstart, d = sum[7 * NT + tid], acc = 0;
  auto append = [&](uint32_t v) {
    acc |= v << ((j & 7u) << 2);
    ++j;
    if ((j & 7u) == 0u) {
      const uint32_t wi = (j >> 3) - 1u;
      if (wi < nodes_words) {
        if (wi == (jstart >> 3) && (jstart & 7u)) atomicOr(&nodes[wi], acc);
        else nodes[wi] = acc;
      }
      acc = 0;
    }
  };
  auto delta_at = [&](uint32_t pos) {
    if (d < dcap) dlist[d] = read_delta(sw, pos + 1, S);
    ++d;
  };
  for (uint32_t w = w0; w < w1; ++w) {
    const uint32_t x = sw[w];
    const uint32_t left = S - 8u * w;
    const uint32_t full = left >= 8u ? 4u : (left >> 1);
    for (uint32_t k = 0; k < full; ++k) {
      const uint32_t byte = (x >> (8u * k)) & 0xFFu;
      const uint32_t e = lut[st * 256u + byte];
      const uint32_t opm = (e >> 5) & 3u, delm = (e >> 7) & 3u;
      if (opm & 1u) {
        append(byte & 15u);
        if (delm & 1u) delta_at(8u * w + 2u * k);
      }
      if (opm & 2u) {
        append(byte >> 4);
        if (delm & 2u) delta_at(8u * w + 2u * k + 1u);
      }
      st = e & 1u;
    }
    if (left < 8u && (left & 1u)) {
      const uint32_t v = (x >> (8u * full)) & 15u;
      if (st == 0) {
        append(v);
        if ((v & 7u) == OP_DELTA) { delta_at(8u * w + 2u * full); st = 1; }
      } else {
        st = (v >> 3) & 1u;
      }
    }
  }
  if ((j & 7u) && (j >> 3) < nodes_words) atomicOr(&nodes[j >> 3], acc);
  ParseOut out;
  out.n_nodes = sum[8 * NT];
  out.n_delta = sum[8 * NT + 1];
  __syncthreads();
  return out;
}

struct BrickCtx {
  const uint32_t* pal;
  uint32_t n_pal;
  const uint32_t* nodes;  // 8 operation symbols per u32
  uint32_t n_nodes;
  const uint32_t* adv_mask;
  const uint32_t* del_mask;
  const uint32_t* adv_pre;
  const uint32_t* del_pre;
  const uint32_t* dlist;
  uint32_t dlist_cap;
  uint32_t op_mask;
  int* s_err;
};

// Palette index of node j with operation o in {ADV, LAST, DELTA}.
__device__ __forceinline__ uint32_t pal_index(const BrickCtx& c, uint32_t j, uint32_t o) {
  const uint32_t w = j >> 5, lt = (1u << (j & 31u)) - 1u;
  const uint32_t k = c.adv_pre[w] + __popc(c.adv_mask[w] & lt);
  if (o == OP_ADV) {
    if (k >= c.n_pal) { set_err(c.s_err, VC_ERR_CORRUPT); return 0; }
    return k;
  }
  if (o == OP_LAST) {
    if (k == 0) { set_err(c.s_err, VC_ERR_CORRUPT); return 0; }
    return k - 1;
  }
  const uint32_t d = c.del_pre[w] + __popc(c.del_mask[w] & lt);
  const uint32_t delta = d < c.dlist_cap ? c.dlist[d] : 0u;
  if (delta == 0 || delta > k) { set_err(c.s_err, VC_ERR_CORRUPT); return 0; }
  return k - delta;
}

__device__ __forceinline__ uint32_t label_of(const BrickCtx& c, uint32_t idx) {
  return idx < c.n_pal ? c.pal[idx] : 0u;
}

// Follows neighbour marks (at most three hops) in a level grid indexed by Morton code.
template <typename GT>
__device__ __forceinline__ uint32_t resolve_morton(const GT* G, uint32_t m, uint32_t g, int* s_err) {
#pragma unroll 1
  for (int hop = 0; hop < 3 && g >= GridT<GT>::MARK; ++hop) {
    m = morton_dec(m, g - GridT<GT>::MARK);
    g = G[m];
  }
  if (g >= GridT<GT>::MARK) { set_err(s_err, VC_ERR_CORRUPT); g = 0; }
  return g;
}

__device__ __forceinline__ void store16(uint32_t* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  *reinterpret_cast<uint4*>(p) = make_uint4(a, b, c, d);
}

template <typename GT>
__device__ __forceinline__ void store_pair(GT* fg, uint32_t pos, uint32_t lo, uint32_t hi) {
  if constexpr (sizeof(GT) == 1) *reinterpret_cast<uint16_t*>(fg + pos) = (uint16_t)(lo | (hi << 8));
  else *reinterpret_cast<uint32_t*>(fg + pos) = lo | (hi << 16);
}

// ------------------------------------------------------------------------------------------
// Decode one brick. head: the record (header, [states], palette) in shared or global memory;
// sw: its symbols as packed nibbles (u32 aligned); out: destination of (b >> lod)^3 labels.
template <int L, typename GT, bool RANS, int NT>
__device__ void decode_brick(const Params& P, const uint32_t* head, const uint32_t* sw, uint32_t* out,
                             unsigned char* sm, int* s_err) {
  constexpr uint32_t NW = NT / 32;
  constexpr uint32_t MARK = GridT<GT>::MARK;
  const SmemLayout& SL = P.v.sm;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  uint32_t* misc = reinterpret_cast<uint32_t*>(sm + SL.misc_off);
  uint32_t* wtot = misc + 16;      // NW warp totals (words 16..47)
  uint32_t* scan_tmp = misc + 48;  // 2 NW + 2 words (48..113); the parse summaries start at 128

  const uint32_t n_pal = head[0], S = head[1], nd = head[3];
  const uint32_t ns = RANS ? (S < 32u ? S : 32u) : 0u;

  BrickCtx c;
  c.pal = head + 4 + ns;
  c.n_pal = n_pal;
  c.op_mask = P.v.op_mask;
  c.s_err = s_err;
  uint32_t* dlist = reinterpret_cast<uint32_t*>(sm + SL.dlist_off);
  c.dlist = dlist;
  c.dlist_cap = nd < SL.dlist_cap ? nd : SL.dlist_cap;

  // 1. operations per node
  if (nd == 0) {
    c.nodes = sw;
    c.n_nodes = S;
  } else {
    uint32_t* nodes = reinterpret_cast<uint32_t*>(sm + SL.nodes_off);
    const ParseOut po = parse_stream<NT>(sw, S, nodes, SL.nodes_words, dlist, c.dlist_cap,
                                         reinterpret_cast<const uint16_t*>(sm + SL.lut_off), misc + 128, s_err);
    c.nodes = nodes;
    c.n_nodes = po.n_nodes;
    if (po.n_delta != nd) set_err(s_err, VC_ERR_CORRUPT);
  }

  // 2. palette-cursor masks and prefix counts (32 nodes per word)
  uint32_t* adv_mask = reinterpret_cast<uint32_t*>(sm + SL.mask_off);
  uint32_t* del_mask = adv_mask + SL.nwords;
  uint32_t* adv_pre = adv_mask + 2 * SL.nwords;
  uint32_t* del_pre = adv_mask + 3 * SL.nwords;
  c.adv_mask = adv_mask; c.del_mask = del_mask; c.adv_pre = adv_pre; c.del_pre = del_pre;
  {
    const uint32_t nw32 = (c.n_nodes + 31u) >> 5;
    const uint32_t per = (nw32 + NT - 1) / NT;
    const uint32_t a0 = min(tid * per, nw32), a1 = min(a0 + per, nw32);
    uint32_t sa = 0, sd = 0;
    for (uint32_t w = a0; w < a1; ++w) {
      uint32_t am = 0, dm = 0;
#pragma unroll
      for (uint32_t k = 0; k < 4; ++k) {
        const uint32_t x = c.nodes[4u * w + k];
        am |= nib_eq8(x, OP_ADV) << (8u * k);
        dm |= nib_eq8(x, OP_DELTA) << (8u * k);
      }
      const uint32_t left = c.n_nodes - 32u * w;
      if (left < 32u) { const uint32_t valid = (1u << left) - 1u; am &= valid; dm &= valid; }
      adv_mask[w] = am; del_mask[w] = dm;
      sa += __popc(am); sd += __popc(dm);
    }
    if (tid == 0) { adv_mask[nw32] = 0; del_mask[nw32] = 0; }  // read by 8-bit windows at the end
    uint32_t pa, pd, ta, td;
    block_scan2<NT>(sa, sd, pa, pd, ta, td, scan_tmp);
    for (uint32_t w = a0; w < a1; ++w) {
      adv_pre[w] = pa; del_pre[w] = pd;
      pa += __popc(adv_mask[w]); pd += __popc(del_mask[w]);
    }
    if (tid == 0 && (ta != n_pal || td != nd)) set_err(s_err, VC_ERR_CORRUPT);
  }
  __syncthreads();

  // 3. coarse levels
  const uint32_t Lout = (uint32_t)L - P.lod;
  const uint32_t last_coarse = Lout < (uint32_t)L ? Lout : (uint32_t)L - 1u;
  GT* G = reinterpret_cast<GT*>(sm + SL.g_off);
  uint16_t* R = reinterpret_cast<uint16_t*>(sm + SL.r_off);
  const bool no_stop = (P.v.flags & kFlagNoStop) != 0;
  uint32_t off = 0, Nl = 1, gofs = 0, gofs_prev = 0;
  for (uint32_t l = 0; l <= last_coarse; ++l) {
    const uint32_t cells = 1u << (3u * l);
    const uint32_t nwa = cells <= 32u ? 1u : min(NW, cells >> 5);
    const uint32_t cpw = cells <= 32u ? 32u : cells / nwa;
    GT* Gl = G + gofs;
    uint16_t* Rl = R + gofs;
    const GT* Gp = G + gofs_prev;
    const uint16_t* Rp = R + gofs_prev;
    if (warp < nwa) {
      uint32_t running = 0;
      for (uint32_t base = warp * cpw; base < (warp + 1) * cpw; base += 32u) {
        const uint32_t m = base + lane;
        bool nonstop = false;
        if (m < cells) {
          bool emitted = true;
          uint32_t j = 0;
          if (l > 0) {
            const uint32_t r = Rp[m >> 3];
            emitted = r != NONE16;
            j = off + 8u * r + (m & 7u);
          }
          uint32_t g = 0;
          if (!emitted) {
            g = Gp[m >> 3];
          } else if (j >= c.n_nodes) {
            set_err(s_err, VC_ERR_CORRUPT);
          } else {
            const uint32_t s = nib_at(c.nodes, j), o = s & 7u, stop = s >> 3;
            if (o == 7u || !((c.op_mask >> o) & 1u) || (stop && no_stop)) set_err(s_err, VC_ERR_CORRUPT);
            if (o == OP_PARENT) {
              if (l == 0) set_err(s_err, VC_ERR_CORRUPT);
              else g = Gp[m >> 3];
            } else if (o <= OP_NZ) {
              const uint32_t a = o - OP_NX;
              if (((m >> a) & 1u) || (m & (0x09249249u << a)) == 0) set_err(s_err, VC_ERR_CORRUPT);
              else g = MARK + a;
            } else if (o != 7u) {
              g = pal_index(c, j, o);
            }
            nonstop = !stop;
          }
          Gl[m] = (GT)g;
        }
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, nonstop);
        if (m < cells) Rl[m] = nonstop ? (uint16_t)(running + __popc(bal & lanemask_lt())) : NONE16;
        running += __popc(bal);
      }
      if (lane == 0) wtot[warp] = running;
    }
    __syncthreads();
    uint32_t total = 0, before = 0;
    for (uint32_t w = 0; w < nwa; ++w) {
      const uint32_t t = wtot[w];
      if (w < warp) before += t;
      total += t;
    }
    if (warp < nwa) {
      for (uint32_t m = warp * cpw + lane; m < min((warp + 1) * cpw, cells); m += 32u) {
        if (before) {
          const uint32_t r = Rl[m];
          if (r != NONE16) Rl[m] = (uint16_t)(r + before);
        }
        const uint32_t g = Gl[m];
        if (g >= MARK) Gl[m] = (GT)resolve_morton<GT>(Gl, m, g, s_err);
      }
    }
    __syncthreads();
    off += Nl;
    Nl = 8u * total;
    gofs_prev = gofs;
    gofs += cells;
  }

  constexpr uint32_t b = 1u << L;
  if (Lout == (uint32_t)L) {
    // 4. finest level
    if (tid == 0 && off + Nl != c.n_nodes) set_err(s_err, VC_ERR_CORRUPT);
    const GT* Gp = G + gofs_prev;
    const uint16_t* Rp = R + gofs_prev;
    GT* fg = reinterpret_cast<GT*>(sm + SL.fg_off);
    constexpr uint32_t pcells = 1u << (3 * (L - 1));
    for (uint32_t m = tid; m < pcells; m += NT) {
      const uint32_t px = compact3(m), py = compact3(m >> 1), pz = compact3(m >> 2);
      const uint32_t f0 = ((2u * pz) * b + 2u * py) * b + 2u * px;
      const uint32_t r = Rp[m];
      const uint32_t gp = Gp[m];
      uint32_t v[8];
      if (r == NONE16) {
#pragma unroll
        for (int o = 0; o < 8; ++o) v[o] = gp;
      } else {
        const uint32_t j0 = off + 8u * r;
        if (j0 + 8u > c.n_nodes) {
          set_err(s_err, VC_ERR_CORRUPT);
#pragma unroll
          for (int o = 0; o < 8; ++o) v[o] = 0;
        } else {
          const uint32_t ops = nib8_at(c.nodes, j0);
          if (ops & 0x88888888u) set_err(s_err, VC_ERR_CORRUPT);  // stop bit at the finest level
          const uint32_t adv8 = bits8_at(adv_mask, j0), del8 = bits8_at(del_mask, j0);
          const uint32_t w = j0 >> 5, lt = (1u << (j0 & 31u)) - 1u;
          const uint32_t k0 = adv_pre[w] + __popc(adv_mask[w] & lt);
          const uint32_t dd0 = del_pre[w] + __popc(del_mask[w] & lt);
#pragma unroll
          for (uint32_t o = 0; o < 8; ++o) {
            const uint32_t op = (ops >> (4u * o)) & 7u;
            const uint32_t below = (1u << o) - 1u;
            uint32_t val = 0;
            if (op == 7u || !((c.op_mask >> op) & 1u)) {
              set_err(s_err, VC_ERR_CORRUPT);
            } else if (op == OP_PARENT) {
              val = gp;
            } else if (op <= OP_NZ) {
              const uint32_t a = op - OP_NX;
              const uint32_t pc = a == 0 ? px : (a == 1 ? py : pz);
              if (((o >> a) & 1u) || pc == 0) set_err(s_err, VC_ERR_CORRUPT);
              else val = MARK + a;
            } else {
              const uint32_t k = k0 + __popc(adv8 & below);
              if (op == OP_ADV) {
                if (k >= n_pal) set_err(s_err, VC_ERR_CORRUPT);
                else val = k;
              } else if (op == OP_LAST) {
                if (k == 0) set_err(s_err, VC_ERR_CORRUPT);
                else val = k - 1u;
              } else {
                const uint32_t di = dd0 + __popc(del8 & below);
                const uint32_t delta = di < c.dlist_cap ? dlist[di] : 0u;
                if (delta == 0 || delta > k) set_err(s_err, VC_ERR_CORRUPT);
                else val = k - delta;
              }
            }
            v[o] = val;
          }
        }
      }
      store_pair<GT>(fg, f0, v[0], v[1]);
      store_pair<GT>(fg, f0 + b, v[2], v[3]);
      store_pair<GT>(fg, f0 + b * b, v[4], v[5]);
      store_pair<GT>(fg, f0 + b * b + b, v[6], v[7]);
    }
    __syncthreads();
    constexpr uint32_t quads = b * b * b / 4u;
    for (uint32_t q = tid; q < quads; q += NT) {
      uint32_t idx[4];
      if constexpr (sizeof(GT) == 1) {
        const uint32_t x = reinterpret_cast<const uint32_t*>(fg)[q];
#pragma unroll
        for (int i = 0; i < 4; ++i) idx[i] = (x >> (8 * i)) & 0xFFu;
      } else {
        const uint2 x = reinterpret_cast<const uint2*>(fg)[q];
        idx[0] = x.x & 0xFFFFu; idx[1] = x.x >> 16; idx[2] = x.y & 0xFFFFu; idx[3] = x.y >> 16;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (idx[i] >= MARK) {
          uint32_t pos = 4u * q + (uint32_t)i, g = idx[i];
#pragma unroll 1
          for (int hop = 0; hop < 3 && g >= MARK; ++hop) {
            const uint32_t a = g - MARK;
            pos -= a == 0 ? 1u : (a == 1 ? b : b * b);
            g = fg[pos];
          }
          if (g >= MARK) { set_err(s_err, VC_ERR_CORRUPT); g = 0; }
          idx[i] = g;
        }
      }
      store16(out + 4u * q, label_of(c, idx[0]), label_of(c, idx[1]), label_of(c, idx[2]), label_of(c, idx[3]));
    }
  } else {
    // coarse level of detail: the level-Lout grid, x fastest
    const GT* Gl = G + gofs_prev;
    const uint32_t n = 1u << Lout;
    const uint32_t total = n * n * n;
    if (total >= 4u) {
      for (uint32_t q = tid; q < total / 4u; q += NT) {
        const uint32_t li = q << 2;
        uint32_t v[4];
#pragma unroll
        for (uint32_t i = 0; i < 4; ++i) {
          const uint32_t t = li + i;
          const uint32_t x = t & (n - 1u), y = (t >> Lout) & (n - 1u), z = t >> (2 * Lout);
          v[i] = label_of(c, Gl[spread3(x) | (spread3(y) << 1) | (spread3(z) << 2)]);
        }
        store16(out + li, v[0], v[1], v[2], v[3]);
      }
    } else if (tid == 0) {
      out[0] = label_of(c, Gl[0]);
    }
  }
}

// ------------------------------------------------------------------------------------------
// TMA bulk copies into shared memory, completion on an mbarrier.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after 2^22 polls (far beyond any copy's latency) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 22); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

template <int NT>
__device__ __forceinline__ void init_parse_lut(unsigned char* sm, const SmemLayout& SL) {
  uint16_t* lut = reinterpret_cast<uint16_t*>(sm + SL.lut_off);
  for (uint32_t i = threadIdx.x; i < 512u; i += NT) lut[i] = (uint16_t)parse_entry(i >> 8, i & 0xFFu);
}

// Where one request item's data lives: the record, and the bytes to stage in shared memory.
struct ItemSrc {
  const uint32_t* rec;     // record in global memory
  const uint32_t* stream;  // symbols in global memory (record for plain, workspace for rANS)
  uint32_t head_bytes;     // staged head (whole record for plain)
  uint32_t stream_bytes;   // staged symbols after the head (rANS only)
};

template <bool RANS>
__device__ __forceinline__ ItemSrc item_src(const Params& P, uint32_t item, uint32_t brick) {
  ItemSrc s;
  const uint32_t a = P.v.starts[brick], e = P.v.starts[brick + 1];
  s.rec = P.v.records + a;
  if (RANS) {
    const uint32_t np = s.rec[0], S = s.rec[1];
    const uint32_t ns = S < 32u ? S : 32u;
    s.head_bytes = (16u + 4u * ns + 4u * np + 15u) & ~15u;
    s.stream = reinterpret_cast<const uint32_t*>(P.ws + (size_t)item * P.v.sm.ws_stride);
    s.stream_bytes = (((S + 1u) >> 1) + 15u) & ~15u;
  } else {
    s.head_bytes = (e - a) * 4u;
    s.stream = s.rec + 4u + s.rec[0];
    s.stream_bytes = 0;
  }
  return s;
}

// One thread block per request item (grid and per-brick schedules).
template <int L, typename GT, bool RANS, int NT>
__global__ void __launch_bounds__(NT) decode_grid_kernel(const __grid_constant__ Params P) {
  extern __shared__ __align__(128) unsigned char sm[];
  const SmemLayout& SL = P.v.sm;
  int* s_err = reinterpret_cast<int*>(sm + SL.misc_off);
  const uint32_t item = P.item_base + blockIdx.x;
  if (item >= P.n) return;
  const uint32_t brick = P.ids[item];
  if (brick >= P.v.n_bricks) {
    if (threadIdx.x == 0) report(P.status, VC_ERR_ARG, item);
    return;
  }
  if (threadIdx.x == 0) *s_err = 0;
  init_parse_lut<NT>(sm, SL);
  const ItemSrc src = item_src<RANS>(P, item, brick);
  const uint32_t* head = src.rec;
  const uint32_t* sw = src.stream;
  if (src.head_bytes + src.stream_bytes <= SL.stage_bytes) {
    uint4* dst = reinterpret_cast<uint4*>(sm + SL.stage_off);
    const uint4* h = reinterpret_cast<const uint4*>(src.rec);
    for (uint32_t i = threadIdx.x; i < src.head_bytes / 16u; i += NT) dst[i] = h[i];
    const uint4* s = reinterpret_cast<const uint4*>(src.stream);
    for (uint32_t i = threadIdx.x; i < src.stream_bytes / 16u; i += NT) dst[src.head_bytes / 16u + i] = s[i];
    // the staged copies' offsets come from the global record (the stage is complete only after
    // the barrier below)
    head = reinterpret_cast<const uint32_t*>(sm + SL.stage_off);
    sw = reinterpret_cast<const uint32_t*>(reinterpret_cast<const unsigned char*>(head) +
                                           (RANS ? src.head_bytes : 16u + 4u * src.rec[0]));
  }
  __syncthreads();
  const uint32_t edge = (1u << L) >> P.lod;
  uint32_t* out = P.cache + (size_t)P.slots[item] * edge * edge * edge;
  decode_brick<L, GT, RANS, NT>(P, head, sw, out, sm, s_err);
  __syncthreads();
  if (threadIdx.x == 0 && *s_err) report(P.status, *s_err, item);
}

// Persistent thread blocks pull items from the work counter in status[2]; while one brick is
// decoded, the next brick's record (and symbols) are already being copied into the other stage
// buffer by the TMA engine.
template <int L, typename GT, bool RANS, int NT>
__global__ void __launch_bounds__(NT) decode_batched_kernel(const __grid_constant__ Params P) {
  extern __shared__ __align__(128) unsigned char sm[];
  const SmemLayout& SL = P.v.sm;
  uint32_t* misc = reinterpret_cast<uint32_t*>(sm + SL.misc_off);
  int* s_err = reinterpret_cast<int*>(misc);
  uint64_t* bar = reinterpret_cast<uint64_t*>(misc + 4);  // two mbarriers at byte 16
  uint32_t* counter = reinterpret_cast<uint32_t*>(P.status) + 2;
  unsigned char* stage[2] = {sm + SL.stage_off, sm + SL.stage_off + SL.stage_bytes};
  const uint32_t tid = threadIdx.x;

  // thread 0: claims the next item and, if it fits, starts copying its data into stage[buf]
  auto claim_and_issue = [&](uint32_t buf) {
    const uint32_t item = atomicAdd(counter, 1u);
    misc[1 + buf] = item;
    uint32_t bytes = 0;
    ItemSrc src{};
    if (item < P.n) {
      const uint32_t brick = P.ids[item];
      if (brick < P.v.n_bricks) {
        src = item_src<RANS>(P, item, brick);
        bytes = src.head_bytes + src.stream_bytes;
        if (bytes > SL.stage_bytes) bytes = 0;
      }
    }
    if (bytes) {
      fence_proxy_async();
      mbar_arrive_tx(&bar[buf], bytes);
      bulk_g2s(stage[buf], src.rec, src.head_bytes, &bar[buf]);
      if (src.stream_bytes) bulk_g2s(stage[buf] + src.head_bytes, src.stream, src.stream_bytes, &bar[buf]);
    } else {
      mbar_arrive_tx(&bar[buf], 0);
    }
  };

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  init_parse_lut<NT>(sm, SL);
  __syncthreads();
  if (tid == 0) claim_and_issue(0);
  uint32_t parity[2] = {0, 0};
  uint32_t buf = 0;
  for (;;) {
    __syncthreads();
    const uint32_t item = misc[1 + buf];
    if (item >= P.n) break;
    if (tid == 0) { *s_err = 0; claim_and_issue(buf ^ 1u); }
    const bool ok = mbar_wait_bounded(&bar[buf], parity[buf]);
    parity[buf] ^= 1u;
    // the decision to give up is taken by the whole block (a barrier follows either way)
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        report(P.status, VC_ERR_TIMEOUT, item);
        mbar_wait_bounded(&bar[buf ^ 1u], parity[buf ^ 1u]);  // the prefetch may still be in flight
      }
      return;
    }
    const uint32_t brick = P.ids[item];
    if (brick >= P.v.n_bricks) {
      if (tid == 0) report(P.status, VC_ERR_ARG, item);
    } else {
      const ItemSrc src = item_src<RANS>(P, item, brick);
      const bool staged = src.head_bytes + src.stream_bytes <= SL.stage_bytes;
      const uint32_t* head = staged ? reinterpret_cast<const uint32_t*>(stage[buf]) : src.rec;
      const uint32_t* sw = !staged ? src.stream
                                   : (RANS ? reinterpret_cast<const uint32_t*>(stage[buf] + src.head_bytes)
                                           : head + 4u + head[0]);
      const uint32_t edge = (1u << L) >> P.lod;
      uint32_t* out = P.cache + (size_t)P.slots[item] * edge * edge * edge;
      decode_brick<L, GT, RANS, NT>(P, head, sw, out, sm, s_err);
      __syncthreads();
      if (tid == 0 && *s_err) report(P.status, *s_err, item);
    }
    buf ^= 1u;
  }
}

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
constexpr int kThreadsB = 256;

template <int L, typename GT, bool RANS>
void* kernel_for(bool batched) {
  return batched ? reinterpret_cast<void*>(&decode_batched_kernel<L, GT, RANS, kThreadsB>)
                 : reinterpret_cast<void*>(&decode_grid_kernel<L, GT, RANS, kThreadsB>);
}

void* pick_kernel(uint32_t L, bool gt16, bool rans, bool batched) {
#define VC_PICK(LL)                                                                                         \
  case LL:                                                                                                  \
    if (gt16) return rans ? kernel_for<LL, uint16_t, true>(batched) : kernel_for<LL, uint16_t, false>(batched); \
    return rans ? kernel_for<LL, uint8_t, true>(batched) : kernel_for<LL, uint8_t, false>(batched);
  switch (L) {
    VC_PICK(1)
    VC_PICK(2)
    VC_PICK(3)
    VC_PICK(4)
    VC_PICK(5)
    default:
      return nullptr;
  }
#undef VC_PICK
}

uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

}  // namespace

vc_status compute_layout(const Volume& v, int device, uint32_t threads, uint32_t nstage, SmemLayout* out) {
  const uint32_t L = v.L;
  if (L < 1 || L > 5) return VC_ERR_UNSUPPORTED;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess)
    return VC_ERR_CUDA;
  SmemLayout s{};
  s.gt_bytes = v.max_pal < kMaxIdx8 ? 1u : 2u;
  const uint32_t b = 1u << L;
  const uint32_t ncells = ((1u << (3 * L)) - 1u) / 7u;  // levels 0..L-1
  const uint32_t stream_words = (v.max_sym + 7u) / 8u;
  uint32_t o = 0;
  s.misc_off = o; o += align16(4 * (128 + 8 * threads + 2));
  s.lut_off = o; o += 1024;
  s.nwords = (v.max_sym + 31u) / 32u + 2u;
  s.mask_off = o; o += align16(4 * 4 * s.nwords);
  s.nodes_words = stream_words + 4u;
  s.nodes_off = o; o += v.max_delta ? align16(4 * s.nodes_words) : 0u;
  s.dlist_cap = v.max_delta;
  s.dlist_off = o; o += align16(4 * (v.max_delta ? v.max_delta : 1u));
  s.g_off = o; o += align16(s.gt_bytes * ncells);
  s.r_off = o; o += align16(2 * ncells);
  s.fg_off = o; o += align16(s.gt_bytes * b * b * b);
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
  void* k = pick_kernel(v.L, v.dv.sm.gt_bytes == 2, rans, batched);
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
      if (!run_symbols(i, 1) || cudaLaunchKernel(k, dim3(1), dim3(kThreadsB), args, smem, stream) != cudaSuccess)
        rc = VC_ERR_CUDA;
    }
  } else if (mode == VC_MODE_GRID) {
    if (!run_symbols(0, n) || cudaLaunchKernel(k, dim3(n), dim3(kThreadsB), args, smem, stream) != cudaSuccess)
      rc = VC_ERR_CUDA;
  } else {
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, v.device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreadsB, smem) != cudaSuccess) {
      rc = VC_ERR_CUDA;
    } else if (per_sm < 1) {
      rc = VC_ERR_UNSUPPORTED;
    } else {
      const uint32_t grid = std::min<uint32_t>(n, (uint32_t)(sms * per_sm));
      if (!run_symbols(0, n) ||
          cudaMemsetAsync(reinterpret_cast<uint32_t*>(status) + 2, 0, sizeof(uint32_t), stream) != cudaSuccess ||
          cudaLaunchKernel(k, dim3(grid), dim3(kThreadsB), args, smem, stream) != cudaSuccess)
        rc = VC_ERR_CUDA;
    }
  }
  if (ws) cudaFreeAsync(ws, stream);
  return rc;
}

}  // namespace vc
