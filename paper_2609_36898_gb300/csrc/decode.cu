// Brick decoder kernels for sm_103a: CSGV operation streams -> uint32 label bricks.
//
// One thread block decodes one brick at a time (Results, "GPU-based rendering pipeline": the
// Decompress stage works on all requested bricks in parallel; here, in parallel over bricks and
// inside each brick). The sequential definition (levels coarse to fine, Morton order inside a
// level, a palette cursor that advances with every palette-advance operation) is evaluated in
// parallel as follows:
//   1. symbols: plain records are read in place; rANS records are decoded by one warp, 32
//      interleaved states per step, renormalisation words handed out with ballot + popc;
//   2. operations: bricks with delta operations go through a two-state parse (operation or delta
//      entry) evaluated as a chunked scan of state-transition summaries; the node-indexed
//      operation array and the delta values come out of it;
//   3. palette cursor: per 32 nodes, ballot masks of advance / delta operations and their
//      exclusive prefix counts, so that any node's cursor k_j is one popc away;
//   4. coarse levels 0..L-1: a dense grid per level (Morton indexed) of palette indices G and of
//      ranks R among the level's nodes with stop bit 0 (the next level's emitted nodes are the 8
//      children of each, in rank order). Neighbour copies form chains of at most three hops
//      (each hop turns one even coordinate odd, and a node needs an even coordinate to copy), so
//      they resolve in three rounds by the number of odd coordinates;
//   5. finest level: every thread owns groups of four consecutive x voxels, resolves each voxel
//      through its parent's rank, its operation and at most three neighbour hops, maps palette
//      indices to labels and writes 16 bytes with one vector store.
// Every check of the format is made on the way (op legality, neighbour parity, palette bounds,
// delta range, stream length); the first error of a brick goes to the caller's status buffer.
#include <cuda_runtime.h>

#include <algorithm>

#include "vc_internal.h"

namespace vc {

namespace {

constexpr uint32_t NT = kThreads;
constexpr uint32_t NW = NT / 32;
constexpr uint16_t NONE16 = 0xFFFFu;
constexpr uint32_t PEND = 0xFFF8u;  // G marks of pending neighbour copies: PEND + axis

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
};

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // bit i -> bit 3i (v < 1024)
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0xFF0000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
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

// Operation symbols of the brick's nodes: either the coded stream itself (no delta entries, two
// symbols per byte) or the node-indexed byte array made by the parse.
struct OpSrc {
  const uint8_t* p;
  bool packed;
  __device__ __forceinline__ uint32_t operator()(uint32_t j) const {
    return packed ? (uint32_t)(p[j >> 1] >> ((j & 1u) << 2)) & 15u : (uint32_t)p[j];
  }
};

struct BrickCtx {
  const uint32_t* pal;
  uint32_t n_pal;
  OpSrc ops;
  uint32_t n_nodes;
  const uint32_t* adv_mask;
  const uint32_t* del_mask;
  const uint32_t* adv_pre;
  const uint32_t* del_pre;
  const uint32_t* dlist;
  uint32_t dlist_cap;  // delta values available (the record's n_delta)
  uint32_t op_mask;
  int* s_err;
};

// Palette index of node j whose operation o is ADV, LAST or DELTA (Supplementary Fig. "CSGV
// ablation" caption: advance reads the next entry, last re-reads it, delta re-reads delta back).
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
  if (d >= c.dlist_cap) { set_err(c.s_err, VC_ERR_CORRUPT); return 0; }
  const uint32_t delta = c.dlist[d];
  if (delta == 0 || delta > k) { set_err(c.s_err, VC_ERR_CORRUPT); return 0; }
  return k - delta;
}

__device__ __forceinline__ uint32_t label_of(const BrickCtx& c, uint32_t idx) {
  return idx < c.n_pal ? c.pal[idx] : 0u;
}

// Inclusive warp scan of two counters.
__device__ __forceinline__ void warp_scan2(uint32_t& a, uint32_t& b, uint32_t lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t na = __shfl_up_sync(0xFFFFFFFFu, a, off), nb = __shfl_up_sync(0xFFFFFFFFu, b, off);
    if (lane >= (uint32_t)off) { a += na; b += nb; }
  }
}

// Exclusive block scan of (a, b); tmp holds 2 * NW + 2 words. Ends with a barrier.
__device__ __forceinline__ void block_scan2(uint32_t a, uint32_t b, uint32_t& pa, uint32_t& pb, uint32_t& ta,
                                            uint32_t& tb, uint32_t* tmp) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t ia = a, ib = b;
  warp_scan2(ia, ib, lane);
  if (lane == 31) { tmp[warp] = ia; tmp[NW + warp] = ib; }
  __syncthreads();
  if (warp == 0) {
    uint32_t va = lane < NW ? tmp[lane] : 0u, vb = lane < NW ? tmp[NW + lane] : 0u;
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

// ---------------------------------------------------------------------------------------------
// rANS symbols (one warp). Symbol i uses state i mod 32; after each step the lanes whose state fell
// below 2^16 take the next 16-bit words in lane order (ballot + popc ranks).
__device__ void rans_decode_warp(const uint32_t* states, const uint16_t* words, uint32_t nw, uint32_t S,
                                 const uint8_t* slot_sym, const uint32_t* fc, uint8_t* nib, int* s_err) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t ns = S < 32u ? S : 32u;
  uint32_t x = lane < ns ? states[lane] : (1u << 16);
  if (lane < ns && x < (1u << 16)) set_err(s_err, VC_ERR_CORRUPT);
  uint32_t ptr = 0;
  const uint32_t* freq = fc;
  const uint32_t* cum = fc + 16;
  for (uint32_t base = 0; base < S; base += 32u) {
    const uint32_t i = base + lane;
    const bool active = i < S;
    uint32_t s = 0;
    if (active) {
      const uint32_t slot = x & (kRansM - 1u);
      s = slot_sym[slot];
      x = freq[s] * (x >> 12) + slot - cum[s];
    }
    const bool need = active && x < (1u << 16);
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, need);
    if (need) {
      const uint32_t at = ptr + __popc(m & lanemask_lt());
      if (at < nw) x = (x << 16) | (uint32_t)words[at];
      else set_err(s_err, VC_ERR_CORRUPT);
    }
    ptr += __popc(m);
    const uint32_t hi = __shfl_xor_sync(0xFFFFFFFFu, s, 1);
    if (active && !(lane & 1u)) nib[i >> 1] = (uint8_t)(s | (i + 1 < S ? hi << 4 : 0u));
  }
  if (ptr != nw) set_err(s_err, VC_ERR_CORRUPT);
  if (lane < ns && x != (1u << 16)) set_err(s_err, VC_ERR_CORRUPT);
}

// ---------------------------------------------------------------------------------------------
// Delta-entry parse. The symbol stream alternates between operations and the entries that follow
// a delta operation (Methods, "Compressed segmentation volumes"). Each thread summarises its chunk
// for both start states; a warp scan composes the summaries; a second pass writes node symbols
// and delta values.
struct ParseOut {
  uint32_t n_nodes;
  uint32_t n_delta;
};

__device__ __forceinline__ uint32_t nib_at(const uint8_t* nib, uint32_t i) {
  return (uint32_t)(nib[i >> 1] >> ((i & 1u) << 2)) & 15u;
}

__device__ __forceinline__ uint32_t read_delta(const uint8_t* nib, uint32_t i, uint32_t S) {
  uint32_t d = 0;
#pragma unroll 1
  for (uint32_t e = 0; e < 7u; ++e) {
    if (i + e >= S) return 0u;
    const uint32_t v = nib_at(nib, i + e);
    d = (d << 3) | (v & 7u);
    if (!(v & 8u)) return d;
  }
  return 0u;  // an eighth entry would follow: invalid
}

__device__ ParseOut parse_deltas(const uint8_t* nib, uint32_t S, uint8_t* node_op, uint32_t* dlist, uint32_t dcap,
                                 uint32_t* sum, int* s_err) {
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t C = (S + NT - 1) / NT;
  const uint32_t i0 = min(tid * C, S), i1 = min(i0 + C, S);
  // summary per start state s in {0 = expecting an operation, 1 = expecting a delta entry}:
  // end state, operations seen, delta operations seen
  uint32_t e[2], no[2], nd[2];
#pragma unroll
  for (uint32_t s0 = 0; s0 < 2; ++s0) {
    uint32_t st = s0, n = 0, d = 0;
    for (uint32_t i = i0; i < i1; ++i) {
      const uint32_t v = nib_at(nib, i);
      if (st == 0) {
        ++n;
        if ((v & 7u) == OP_DELTA) { ++d; st = 1; }
      } else if (!(v & 8u)) {
        st = 0;
      }
    }
    e[s0] = st; no[s0] = n; nd[s0] = d;
  }
  // sum layout: [0..NT) e bits, [NT..2NT) n0, [2NT..3NT) n1, [3NT..4NT) d0, [4NT..5NT) d1
  sum[tid] = e[0] | (e[1] << 1);
  sum[NT + tid] = no[0];
  sum[2 * NT + tid] = no[1];
  sum[3 * NT + tid] = nd[0];
  sum[4 * NT + tid] = nd[1];
  __syncthreads();
  if (warp == 0) {
    // each lane composes the summaries of threads [8 lane, 8 lane + 8)
    constexpr uint32_t PER = NT / 32;
    uint32_t E0 = 0, E1 = 1, N0 = 0, N1 = 0, D0 = 0, D1 = 0;  // identity
    for (uint32_t t = lane * PER; t < lane * PER + PER; ++t) {
      const uint32_t te = sum[t];
      const uint32_t tn[2] = {sum[NT + t], sum[2 * NT + t]}, td[2] = {sum[3 * NT + t], sum[4 * NT + t]};
      N0 += tn[E0]; D0 += td[E0]; E0 = (te >> E0) & 1u;
      N1 += tn[E1]; D1 += td[E1]; E1 = (te >> E1) & 1u;
    }
    // inclusive scan of the composed functions across lanes (A then B)
    uint32_t iE0 = E0, iE1 = E1, iN0 = N0, iN1 = N1, iD0 = D0, iD1 = D1;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t pE0 = __shfl_up_sync(0xFFFFFFFFu, iE0, off), pE1 = __shfl_up_sync(0xFFFFFFFFu, iE1, off);
      const uint32_t pN0 = __shfl_up_sync(0xFFFFFFFFu, iN0, off), pN1 = __shfl_up_sync(0xFFFFFFFFu, iN1, off);
      const uint32_t pD0 = __shfl_up_sync(0xFFFFFFFFu, iD0, off), pD1 = __shfl_up_sync(0xFFFFFFFFu, iD1, off);
      if (lane >= (uint32_t)off) {
        // prefix p then current c: start s -> p, then c from p's end state
        const uint32_t cE[2] = {iE0, iE1}, cN[2] = {iN0, iN1}, cD[2] = {iD0, iD1};
        iN0 = pN0 + cN[pE0]; iD0 = pD0 + cD[pE0]; iE0 = cE[pE0];
        iN1 = pN1 + cN[pE1]; iD1 = pD1 + cD[pE1]; iE1 = cE[pE1];
      }
    }
    // exclusive prefix applied to start state 0
    uint32_t xs = __shfl_up_sync(0xFFFFFFFFu, iE0, 1), xn = __shfl_up_sync(0xFFFFFFFFu, iN0, 1),
             xd = __shfl_up_sync(0xFFFFFFFFu, iD0, 1);
    if (lane == 0) { xs = 0; xn = 0; xd = 0; }
    // walk the lane's threads and store their start state and bases in place
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
  uint32_t st = sum[5 * NT + tid], j = sum[6 * NT + tid], d = sum[7 * NT + tid];
  for (uint32_t i = i0; i < i1; ++i) {
    const uint32_t v = nib_at(nib, i);
    if (st == 0) {
      node_op[j++] = (uint8_t)v;
      if ((v & 7u) == OP_DELTA) {
        if (d < dcap) dlist[d] = read_delta(nib, i + 1, S);
        ++d;
        st = 1;
      }
    } else if (!(v & 8u)) {
      st = 0;
    }
  }
  ParseOut out;
  out.n_nodes = sum[8 * NT];
  out.n_delta = sum[8 * NT + 1];
  __syncthreads();
  return out;
}

// ---------------------------------------------------------------------------------------------
// Finest-level voxel: parent rank -> operation -> label, following at most three neighbour hops.
template <int L>
__device__ __forceinline__ uint32_t resolve_voxel(const BrickCtx& c, const uint16_t* Gp, const uint16_t* Rp,
                                                  uint32_t offL, uint32_t x, uint32_t y, uint32_t z) {
#pragma unroll 1
  for (int hop = 0; hop < 4; ++hop) {
    const uint32_t pm = spread3(x >> 1) | (spread3(y >> 1) << 1) | (spread3(z >> 1) << 2);
    const uint32_t r = Rp[pm];
    if (r == NONE16) return Gp[pm];
    const uint32_t j = offL + 8u * r + ((x & 1u) | ((y & 1u) << 1) | ((z & 1u) << 2));
    if (j >= c.n_nodes) { set_err(c.s_err, VC_ERR_CORRUPT); return 0; }
    const uint32_t s = c.ops(j), o = s & 7u;
    if ((s & 8u) || o == 7u || !((c.op_mask >> o) & 1u)) { set_err(c.s_err, VC_ERR_CORRUPT); return 0; }
    if (o == OP_PARENT) return Gp[pm];
    if (o >= OP_ADV) return pal_index(c, j, o);
    const uint32_t a = o - OP_NX;
    const uint32_t ca = a == 0 ? x : (a == 1 ? y : z);
    if ((ca & 1u) || ca == 0) { set_err(c.s_err, VC_ERR_CORRUPT); return 0; }
    if (a == 0) --x; else if (a == 1) --y; else --z;
  }
  set_err(c.s_err, VC_ERR_CORRUPT);
  return 0;
}

__device__ __forceinline__ void store16(uint32_t* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  *reinterpret_cast<uint4*>(p) = make_uint4(a, b, c, d);
}

// ---------------------------------------------------------------------------------------------
// Decode one brick whose record is at `rec` (shared or global memory) into `out`.
template <int L, bool RANS>
__device__ void decode_brick(const Params& P, const uint32_t* rec, uint32_t* out, unsigned char* sm, int* s_err) {
  const SmemLayout& SL = P.v.sm;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  uint32_t* misc = reinterpret_cast<uint32_t*>(sm + SL.misc_off);
  uint32_t* scan_tmp = misc + 16;

  const uint32_t n_pal = rec[0], S = rec[1], cb = rec[2], nd = rec[3];
  const uint32_t ns = RANS ? (S < 32u ? S : 32u) : 0u;
  const uint32_t* pal = rec + 4 + ns;
  const uint8_t* coded = reinterpret_cast<const uint8_t*>(pal + n_pal);

  // 1. symbols
  const uint8_t* nib = coded;
  if (RANS) {
    uint8_t* dst = sm + SL.nib_off;
    if (warp == 0)
      rans_decode_warp(rec + 4, reinterpret_cast<const uint16_t*>(coded), cb >> 1, S, sm + SL.rans_off,
                          reinterpret_cast<const uint32_t*>(sm + SL.rans_off + 4096), dst, s_err);
    __syncthreads();
    nib = dst;
  }

  // 2. operations
  BrickCtx c;
  c.pal = pal;
  c.n_pal = n_pal;
  c.op_mask = P.v.op_mask;
  c.s_err = s_err;
  uint32_t* masks = reinterpret_cast<uint32_t*>(sm + SL.mask_off);
  uint32_t* dlist = reinterpret_cast<uint32_t*>(sm + SL.dlist_off);
  if (nd == 0) {
    c.ops.p = nib;
    c.ops.packed = true;
    c.n_nodes = S;
  } else {
    uint8_t* node_op = sm + SL.op_off;
    ParseOut po =
        parse_deltas(nib, S, node_op, dlist, nd, reinterpret_cast<uint32_t*>(sm + SL.parse_off), s_err);
    c.ops.p = node_op;
    c.ops.packed = false;
    c.n_nodes = po.n_nodes;
    if (po.n_delta != nd) set_err(s_err, VC_ERR_CORRUPT);
  }
  const uint32_t nwords = (c.n_nodes + 31u) >> 5;
  uint32_t* adv_mask = masks;
  uint32_t* del_mask = masks + SL.nwords;
  uint32_t* adv_pre = masks + 2 * SL.nwords;
  uint32_t* del_pre = masks + 3 * SL.nwords;
  c.adv_mask = adv_mask; c.del_mask = del_mask; c.adv_pre = adv_pre; c.del_pre = del_pre; c.dlist = dlist;
  c.dlist_cap = nd;

  // 3. palette-cursor masks and prefix counts
  for (uint32_t w = warp; w < nwords; w += NW) {
    const uint32_t j = (w << 5) + lane;
    const uint32_t o = j < c.n_nodes ? (c.ops(j) & 7u) : 7u;
    const uint32_t am = __ballot_sync(0xFFFFFFFFu, o == OP_ADV), dm = __ballot_sync(0xFFFFFFFFu, o == OP_DELTA);
    if (lane == 0) { adv_mask[w] = am; del_mask[w] = dm; }
  }
  __syncthreads();
  {
    const uint32_t per = (nwords + NT - 1) / NT;
    const uint32_t w0 = min(tid * per, nwords), w1 = min(w0 + per, nwords);
    uint32_t sa = 0, sd = 0;
    for (uint32_t w = w0; w < w1; ++w) { sa += __popc(adv_mask[w]); sd += __popc(del_mask[w]); }
    uint32_t pa, pd, ta, td;
    block_scan2(sa, sd, pa, pd, ta, td, scan_tmp);
    for (uint32_t w = w0; w < w1; ++w) {
      adv_pre[w] = pa; del_pre[w] = pd;
      pa += __popc(adv_mask[w]); pd += __popc(del_mask[w]);
    }
    if (tid == 0 && (ta != n_pal || td != nd)) set_err(s_err, VC_ERR_CORRUPT);
  }
  __syncthreads();

  // 4. coarse levels
  const uint32_t Lout = (uint32_t)L - P.lod;
  const uint32_t last_coarse = Lout < (uint32_t)L ? Lout : (uint32_t)L - 1u;
  uint16_t* G = reinterpret_cast<uint16_t*>(sm + SL.grid_off);
  uint16_t* R = G + SL.ncells;
  uint32_t* chunk_mask = reinterpret_cast<uint32_t*>(sm + SL.chunk_off);
  uint32_t* chunk_pre = chunk_mask + SL.nchunks;
  uint32_t off = 0, Nl = 1, gofs = 0, gofs_prev = 0;
  const bool no_stop = (P.v.flags & kFlagNoStop) != 0;
  for (uint32_t l = 0; l <= last_coarse; ++l) {
    const uint32_t cells = 1u << (3u * l);
    const uint32_t nch = (cells + 31u) >> 5;
    uint16_t* Gl = G + gofs;
    uint16_t* Rl = R + gofs;
    const uint16_t* Gp = G + gofs_prev;
    const uint16_t* Rp = R + gofs_prev;
    // pass A: every cell of the level
    for (uint32_t ch = warp; ch < nch; ch += NW) {
      const uint32_t m = (ch << 5) + lane;
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
          const uint32_t s = c.ops(j), o = s & 7u, stop = s >> 3;
          if (o == 7u || !((c.op_mask >> o) & 1u) || (stop && no_stop)) set_err(s_err, VC_ERR_CORRUPT);
          if (o == OP_PARENT) {
            if (l == 0) set_err(s_err, VC_ERR_CORRUPT);
            else g = Gp[m >> 3];
          } else if (o <= OP_NZ) {
            const uint32_t a = o - OP_NX;
            const uint32_t ma = 0x09249249u << a;
            if ((m >> a) & 1u || (m & ma) == 0) set_err(s_err, VC_ERR_CORRUPT);
            else g = PEND + a;
          } else if (o != 7u) {
            g = pal_index(c, j, o);
          }
          nonstop = !stop;
        }
        Gl[m] = (uint16_t)g;
      }
      const uint32_t bm = __ballot_sync(0xFFFFFFFFu, nonstop);
      if (lane == 0) chunk_mask[ch] = bm;
    }
    __syncthreads();
    // neighbour copies: three rounds, from two odd coordinates down to none
    if (l > 0) {
      for (int rnd = 2; rnd >= 0; --rnd) {
        for (uint32_t m = tid; m < cells; m += NT) {
          const uint32_t g = Gl[m];
          if (g >= PEND && __popc(m & 7u) == rnd) Gl[m] = Gl[morton_dec(m, g - PEND)];
        }
        __syncthreads();
      }
    }
    // ranks of the stop-0 nodes: exclusive prefix over the chunk masks (one warp)
    if (warp == 0) {
      const uint32_t per = (nch + 31u) >> 5;
      const uint32_t c0 = min(lane * per, nch), c1 = min(c0 + per, nch);
      uint32_t s = 0, dummy = 0;
      for (uint32_t ch = c0; ch < c1; ++ch) s += __popc(chunk_mask[ch]);
      uint32_t is = s;
      warp_scan2(is, dummy, lane);
      uint32_t p = is - s;
      for (uint32_t ch = c0; ch < c1; ++ch) { chunk_pre[ch] = p; p += __popc(chunk_mask[ch]); }
      if (lane == 31) misc[8] = is;
    }
    __syncthreads();
    const uint32_t nonstop_total = misc[8];
    if (l < last_coarse || (Lout == (uint32_t)L && l == (uint32_t)L - 1u)) {
      for (uint32_t m = tid; m < cells; m += NT) {
        const uint32_t ch = m >> 5, bit = 1u << (m & 31u);
        const uint32_t msk = chunk_mask[ch];
        Rl[m] = (msk & bit) ? (uint16_t)(chunk_pre[ch] + __popc(msk & (bit - 1u))) : NONE16;
      }
    }
    __syncthreads();
    off += Nl;
    Nl = 8u * nonstop_total;
    gofs_prev = gofs;
    gofs += cells;
  }

  constexpr uint32_t b = 1u << L;
  if (Lout == (uint32_t)L) {
    // 5. finest level
    if (tid == 0 && off + Nl != c.n_nodes) set_err(s_err, VC_ERR_CORRUPT);
    const uint16_t* Gp = G + gofs_prev;
    const uint16_t* Rp = R + gofs_prev;
    constexpr uint32_t quads = b * b * b / 4u;
    for (uint32_t q = tid; q < quads; q += NT) {
      const uint32_t li = q << 2;
      uint32_t v[4];
#pragma unroll
      for (uint32_t i = 0; i < 4; ++i) {
        const uint32_t t = li + i;
        const uint32_t x = t & (b - 1u), y = (t >> L) & (b - 1u), z = t >> (2 * L);
        v[i] = label_of(c, resolve_voxel<L>(c, Gp, Rp, off, x, y, z));
      }
      store16(out + li, v[0], v[1], v[2], v[3]);
    }
  } else {
    // coarse level of detail: the level-Lout grid, x fastest
    const uint16_t* Gl = G + gofs_prev;
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

// ---------------------------------------------------------------------------------------------
// TMA bulk copy of a record into shared memory, completion on an mbarrier.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
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
// Bounded wait: gives up after ~2^22 polls (far beyond any copy's latency) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 22); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void load_rans_tables(const Params& P, unsigned char* sm) {
  const SmemLayout& SL = P.v.sm;
  const uint4* src = reinterpret_cast<const uint4*>(P.v.rans_sym);
  uint4* dst = reinterpret_cast<uint4*>(sm + SL.rans_off);
  for (uint32_t i = threadIdx.x; i < 4096u / 16u; i += NT) dst[i] = src[i];
  uint32_t* fc = reinterpret_cast<uint32_t*>(sm + SL.rans_off + 4096);
  for (uint32_t i = threadIdx.x; i < 33u; i += NT) fc[i] = P.v.rans_fc[i];
}

// Copies a record into shared memory with all threads (16-byte loads); returns where to read it.
__device__ __forceinline__ const uint32_t* stage_record(const Params& P, uint32_t brick, unsigned char* stage) {
  const uint32_t a = P.v.starts[brick], e = P.v.starts[brick + 1];
  const uint32_t* g = P.v.records + a;
  const uint32_t bytes = (e - a) * 4u;
  if (bytes > P.v.sm.stage_bytes) return g;
  const uint4* src = reinterpret_cast<const uint4*>(g);
  uint4* dst = reinterpret_cast<uint4*>(stage);
  for (uint32_t i = threadIdx.x; i < bytes / 16u; i += NT) dst[i] = src[i];
  __syncthreads();
  return reinterpret_cast<const uint32_t*>(stage);
}

// One thread block per brick: blockIdx.x + item_base is the request item.
template <int L, bool RANS>
__global__ void __launch_bounds__(NT) decode_grid_kernel(const __grid_constant__ Params P) {
  extern __shared__ __align__(128) unsigned char sm[];
  const SmemLayout& SL = P.v.sm;
  int* s_err = reinterpret_cast<int*>(sm + SL.misc_off);
  const uint32_t item = P.item_base + blockIdx.x;
  if (item >= P.n) return;
  if (threadIdx.x == 0) *s_err = 0;
  if (RANS) load_rans_tables(P, sm);
  const uint32_t brick = P.ids[item];
  if (brick >= P.v.n_bricks) {
    if (threadIdx.x == 0) report(P.status, VC_ERR_ARG, item);
    return;
  }
  __syncthreads();
  const uint32_t* rec = stage_record(P, brick, sm + SL.stage_off);
  const uint32_t edge = (1u << L) >> P.lod;
  uint32_t* out = P.cache + (size_t)P.slots[item] * edge * edge * edge;
  decode_brick<L, RANS>(P, rec, out, sm, s_err);
  __syncthreads();
  if (threadIdx.x == 0 && *s_err) report(P.status, *s_err, item);
}

// Persistent thread blocks: pull items from the work counter in status[2]; while a brick is being
// decoded, the next brick's record is already on its way into the other stage buffer (bulk copy
// completing on an mbarrier).
template <int L, bool RANS>
__global__ void __launch_bounds__(NT) decode_batched_kernel(const __grid_constant__ Params P) {
  extern __shared__ __align__(128) unsigned char sm[];
  const SmemLayout& SL = P.v.sm;
  uint32_t* misc = reinterpret_cast<uint32_t*>(sm + SL.misc_off);
  int* s_err = reinterpret_cast<int*>(misc);
  uint64_t* bar = reinterpret_cast<uint64_t*>(misc + 4);  // two mbarriers at misc + 16 bytes
  uint32_t* counter = reinterpret_cast<uint32_t*>(P.status) + 2;
  unsigned char* stage[2] = {sm + SL.stage_off, sm + SL.stage_off + SL.stage_bytes};
  const uint32_t tid = threadIdx.x;

  // thread 0: claims an item and, if its record fits, starts copying it into stage[buf].
  // misc[1 + buf] receives the item (or >= n when the queue is empty).
  auto claim_and_issue = [&](uint32_t buf) {
    const uint32_t item = atomicAdd(counter, 1u);
    misc[1 + buf] = item;
    uint32_t bytes = 0;
    const void* src = nullptr;
    if (item < P.n) {
      const uint32_t brick = P.ids[item];
      if (brick < P.v.n_bricks) {
        const uint32_t a = P.v.starts[brick], e = P.v.starts[brick + 1];
        bytes = (e - a) * 4u;
        src = P.v.records + a;
        if (bytes > SL.stage_bytes) bytes = 0;
      }
    }
    if (bytes) {
      fence_proxy_async();
      mbar_arrive_tx(&bar[buf], bytes);
      bulk_g2s(stage[buf], src, bytes, &bar[buf]);
    } else {
      mbar_arrive_tx(&bar[buf], 0);
    }
  };

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  if (RANS) load_rans_tables(P, sm);
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
      const uint32_t a = P.v.starts[brick], e = P.v.starts[brick + 1];
      const bool staged = (e - a) * 4u <= SL.stage_bytes;
      const uint32_t* rec = staged ? reinterpret_cast<const uint32_t*>(stage[buf]) : P.v.records + a;
      const uint32_t edge = (1u << L) >> P.lod;
      uint32_t* out = P.cache + (size_t)P.slots[item] * edge * edge * edge;
      decode_brick<L, RANS>(P, rec, out, sm, s_err);
      __syncthreads();
      if (tid == 0 && *s_err) report(P.status, *s_err, item);
    }
    buf ^= 1u;
  }
}

template <int L, bool RANS>
struct KernelSet {
  static void* grid() { return reinterpret_cast<void*>(&decode_grid_kernel<L, RANS>); }
  static void* batched() { return reinterpret_cast<void*>(&decode_batched_kernel<L, RANS>); }
};

void* pick_kernel(uint32_t L, bool rans, bool batched) {
#define VC_PICK(LL)                                                                        \
  case LL:                                                                                 \
    return rans ? (batched ? KernelSet<LL, true>::batched() : KernelSet<LL, true>::grid()) \
                : (batched ? KernelSet<LL, false>::batched() : KernelSet<LL, false>::grid());
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

vc_status compute_layout(uint32_t L, uint32_t coder, uint32_t max_sym, uint32_t max_pal, uint32_t max_delta,
                         uint32_t max_rec_words, int device, SmemLayout* out) {
  (void)max_pal;
  if (L < 1 || L > 5) return VC_ERR_UNSUPPORTED;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess)
    return VC_ERR_CUDA;
  SmemLayout s{};
  const uint32_t ncells = ((1u << (3 * L)) - 1u) / 7u;  // levels 0..L-1
  const uint32_t largest_coarse = 1u << (3 * (L - 1));
  uint32_t o = 0;
  s.misc_off = o; o += 256;
  s.rans_off = o; o += coder == 1 ? align16(4096 + 33 * 4) : 0;
  s.nwords = (max_sym + 31u) / 32u;
  s.mask_off = o; o += align16(4 * 4 * s.nwords);
  s.nib_off = o; o += coder == 1 ? align16((max_sym + 1) / 2) : 0;
  s.op_off = o; o += max_delta ? align16(max_sym) : 0;
  s.dlist_off = o; o += align16(4 * (max_delta ? max_delta : 1));
  s.ncells = ncells;
  s.grid_off = o; o += align16(2 * 2 * ncells);
  s.nchunks = (largest_coarse + 31u) / 32u;
  s.chunk_off = o; o += align16(2 * 4 * s.nchunks);
  s.parse_off = o; o += max_delta ? align16(4 * (8 * NT + 2)) : 0;
  const uint32_t fixed = o;
  // stage two record buffers if they fit next to the fixed regions
  uint32_t stage = align16(4 * max_rec_words);
  if (fixed + 2 * stage > (uint32_t)optin) stage = 0;
  s.stage_bytes = stage;
  s.stage_off = o; o += 2 * stage;
  s.total = o;
  if (s.total > (uint32_t)optin) return VC_ERR_UNSUPPORTED;
  *out = s;
  return VC_OK;
}

vc_status launch_decode(const Volume& v, const uint32_t* ids, uint32_t n, const uint32_t* slots, uint32_t* cache,
                        uint32_t lod, uint32_t mode, int32_t* status, cudaStream_t stream) {
  if (n == 0) return VC_OK;
  const bool rans = v.coder == 1;
  const bool batched = mode == VC_MODE_BATCHED;
  void* k = pick_kernel(v.L, rans, batched);
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
  void* args[] = {&P};
  if (mode == VC_MODE_PLAIN) {
    for (uint32_t i = 0; i < n; ++i) {
      P.item_base = i;
      if (cudaLaunchKernel(k, dim3(1), dim3(NT), args, smem, stream) != cudaSuccess) return VC_ERR_CUDA;
    }
    return VC_OK;
  }
  if (mode == VC_MODE_GRID) {
    if (cudaLaunchKernel(k, dim3(n), dim3(NT), args, smem, stream) != cudaSuccess) return VC_ERR_CUDA;
    return VC_OK;
  }
  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, v.device) != cudaSuccess) return VC_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem) != cudaSuccess) return VC_ERR_CUDA;
  if (per_sm < 1) return VC_ERR_UNSUPPORTED;
  const uint32_t grid = std::min<uint32_t>(n, (uint32_t)(sms * per_sm));
  if (cudaMemsetAsync(reinterpret_cast<uint32_t*>(status) + 2, 0, sizeof(uint32_t), stream) != cudaSuccess)
    return VC_ERR_CUDA;
  if (cudaLaunchKernel(k, dim3(grid), dim3(NT), args, smem, stream) != cudaSuccess) return VC_ERR_CUDA;
  return VC_OK;
}

}  // namespace vc
