// Device code of the brick decoder (templates), shared by the per-thread-count translation
// units. See decode.cu for the design.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "vc_internal.h"

namespace vc {
namespace dev {
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
  uint32_t ws_item0;  // the workspaces hold items ws_item0 .. (a chunk of the request)
  uint32_t out_words; // u32 words per cache slot
  uint32_t pal_bits;  // 0: labels; else cache paletting: pal_bits-bit palette indices,
  uint32_t pal_per;   //   pal_per of them per u32 word (none straddles a word)
  const uint32_t* order;  // size-aware order: the k-th scheduled item is order[k] (nullptr: k)
  const uint32_t* n_dev;  // persistent schedules: the item count in device memory, read at launch
                          // (min(n, *n_dev) items; nullptr: n), for work sized on the device
};

// Items of a launch of a persistent schedule.
__device__ __forceinline__ uint32_t launch_items(const Params& P) {
  return P.n_dev ? min(P.n, *P.n_dev) : P.n;
}

// The item scheduled k-th (k < P.n).
__device__ __forceinline__ uint32_t scheduled_item(const Params& P, uint32_t k) { return P.order ? P.order[k] : k; }

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
// Offset in the finest grid (x fastest, edge 2^L) of child (0,0,0) of level-(L-1) cell m; additive
// over disjoint bit sets of m.
template <int L>
__device__ __forceinline__ uint32_t flin(uint32_t m) {
  constexpr uint32_t b = 1u << L;
  return 2u * ((compact3(m >> 2) * b + compact3(m >> 1)) * b + compact3(m));
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
// bits 4i of z gathered into bits i (8 bits)
__device__ __forceinline__ uint32_t gather_nib_bits(uint32_t z) {
  z = (z | (z >> 3)) & 0x03030303u;
  z = (z | (z >> 6)) & 0x000F000Fu;
  z = (z | (z >> 12)) & 0xFFu;
  return z;
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

// The 4 nibbles in bits 0..15 of x spread to the 4 bytes of the result (nibble i -> byte i).
__device__ __forceinline__ uint32_t nib4_to_bytes(uint32_t x) {
  x = (x | (x << 8)) & 0x00FF00FFu;
  return (x | (x << 4)) & 0x0F0F0F0Fu;
}
// The most significant bits of the 4 bytes of x gathered into bits 0..3 (byte i -> bit i).
__device__ __forceinline__ uint32_t byte_msbs(uint32_t x) { return ((x & 0x80808080u) * 0x00204081u) >> 28; }

// The 8 cells of one sibling group (children 0..7 of a parent, child o = x | y << 1 | z << 2):
// palette indices or neighbour marks, gt_bytes each, as u32 words (8-bit grids: child o in byte
// o & 3 of word o >> 2; 16-bit grids: child o in half o & 1 of word o >> 1).
template <typename GT>
struct Cells8 {
  uint32_t w[sizeof(GT) == 1 ? 2 : 4];
};
template <typename GT>
__device__ __forceinline__ void store_cells8(GT* dst, const Cells8<GT>& v) {
  if constexpr (sizeof(GT) == 1) *reinterpret_cast<uint2*>(dst) = make_uint2(v.w[0], v.w[1]);
  else *reinterpret_cast<uint4*>(dst) = make_uint4(v.w[0], v.w[1], v.w[2], v.w[3]);
}
template <typename GT>
__device__ __forceinline__ Cells8<GT> load_cells8(const GT* src) {
  Cells8<GT> v;
  if constexpr (sizeof(GT) == 1) {
    const uint2 t = *reinterpret_cast<const uint2*>(src);
    v.w[0] = t.x; v.w[1] = t.y;
  } else {
    const uint4 t = *reinterpret_cast<const uint4*>(src);
    v.w[0] = t.x; v.w[1] = t.y; v.w[2] = t.z; v.w[3] = t.w;
  }
  return v;
}
template <typename GT>
__device__ __forceinline__ uint32_t cell_of(const Cells8<GT>& v, uint32_t o) {
  if constexpr (sizeof(GT) == 1) return (v.w[o >> 2] >> (8u * (o & 3u))) & 0xFFu;
  else return (v.w[o >> 1] >> (16u * (o & 1u))) & 0xFFFFu;
}
template <typename GT>
__device__ __forceinline__ void set_cell(Cells8<GT>& v, uint32_t o, uint32_t x) {
  if constexpr (sizeof(GT) == 1) {
    const uint32_t sh = 8u * (o & 3u);
    if (o < 4u) v.w[0] = (v.w[0] & ~(0xFFu << sh)) | (x << sh);
    else v.w[1] = (v.w[1] & ~(0xFFu << sh)) | (x << sh);
  } else {
    const uint32_t sh = 16u * (o & 1u);
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i)
      if ((o >> 1) == i) v.w[i] = (v.w[i] & ~(0xFFFFu << sh)) | (x << sh);
  }
}

// Bit o set iff child o of v holds a neighbour mark (8-bit grids: >= 0xFD; 16-bit: >= 0xFFFD).
template <typename GT>
__device__ __forceinline__ uint32_t mark_bits(const Cells8<GT>& v) {
  if constexpr (sizeof(GT) == 1) {
    const uint32_t a = ((v.w[0] & 0x7F7F7F7Fu) + 0x03030303u) & v.w[0];
    const uint32_t b = ((v.w[1] & 0x7F7F7F7Fu) + 0x03030303u) & v.w[1];
    return byte_msbs(a) | (byte_msbs(b) << 4);
  } else {
    uint32_t m = 0u;
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) {
      const uint32_t t = ((v.w[i] & 0x7FFF7FFFu) + 0x00030003u) & v.w[i] & 0x80008000u;
      m |= (((t >> 15) & 1u) | ((t >> 30) & 2u)) << (2u * i);
    }
    return m;
  }
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
// Parse of the symbol stream: which nibbles are operations and which are delta entries. It is a
// 2-state automaton (state 1 = "a delta entry comes next"): from state 0 a nibble is an operation
// and the state becomes 1 iff it is a delta operation (low 3 bits = 6); from state 1 the nibble is
// an entry and the state stays 1 iff its bit 3 ("another entry follows") is set.

// delta from the entries at nibble i..; 0 when invalid (runs past S or needs an eighth entry).
// short_delta: one entry holding delta - 1 (2 <= delta <= 16; entry 0 is invalid).
__device__ __forceinline__ uint32_t read_delta(const uint32_t* sw, uint32_t i, uint32_t S, bool short_delta) {
  if (short_delta) {
    const uint32_t v = i < S ? nib_at(sw, i) : 0u;
    return v ? v + 1u : 0u;
  }
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

// For the 8 nibbles of stream word x: D = nibbles whose low 3 bits are 6 (delta operations if they
// are operations); A / B = bit i holds the state after nibble i when the word is entered in state
// 0 / 1. The per-nibble transitions are composed by prefix doubling on 8-bit masks. An entry is
// followed by another while its bit 3 is set, or never (short_delta: one entry per delta).
__device__ __forceinline__ void word_states(uint32_t x, uint32_t& D, uint32_t& A, uint32_t& B, bool short_delta) {
  D = nib_eq8(x, OP_DELTA);
  uint32_t a = D, e = short_delta ? 0u : gather_nib_bits((x >> 3) & 0x11111111u);  // after nibble i from 0 / 1
#pragma unroll
  for (uint32_t k = 1; k < 8; k <<= 1) {
    const uint32_t ha = a << k, hb = (e << k) | ((1u << k) - 1u);  // identity below bit k
    const uint32_t na = (ha & e) | (~ha & a), nb = (hb & e) | (~hb & a);
    a = na & 0xFFu;
    e = nb & 0xFFu;
  }
  A = a;
  B = e;
}

// Operation nibbles of a word entered in state st (nv valid nibbles); *end = the state after it.
__device__ __forceinline__ uint32_t word_ops(uint32_t A, uint32_t B, uint32_t st, uint32_t nv, uint32_t* end) {
  const uint32_t F = st ? B : A;
  *end = (F >> (nv - 1u)) & 1u;
  const uint32_t entering = ((F << 1) | st) & 0xFFu;
  return ~entering & ((1u << nv) - 1u);
}

// The nibbles of x selected by m, packed from nibble 0 upwards.
__device__ __forceinline__ uint32_t pack_nibbles(uint32_t x, uint32_t m) {
  // remove the unselected nibbles (few: delta entries, or past the stream's end), highest first,
  // so that the positions below stay put; zeros shift in at the top
  uint32_t drop = ~m & 0xFFu;
  while (drop) {
    const uint32_t p = 31u - __clz(drop);
    const uint32_t low = (1u << (4u * p)) - 1u;
    x = (x & low) | ((x >> 4) & ~low);
    drop &= ~(1u << p);
  }
  return x;
}

// A chunk summary for both entering states: bit s of e = the state after the chunk entered in
// state s; nd_s = nodes | delta operations << K counted from entering state s. ND is uint32_t with
// K = 16 while node counts stay below 2^16 (b <= 32) and uint64_t with K = 32 beyond.
template <typename ND>
struct Fn2 {
  uint32_t e;
  ND nd0, nd1;
};
template <typename ND>
__device__ __forceinline__ Fn2<ND> fn_id() {
  return Fn2<ND>{2u, 0, 0};
}
template <typename ND>
__device__ __forceinline__ Fn2<ND> fn_then(const Fn2<ND>& p, const Fn2<ND>& c) {  // p, then c
  const uint32_t p0 = p.e & 1u, p1 = (p.e >> 1) & 1u;
  const uint32_t c0 = c.e & 1u, c1 = (c.e >> 1) & 1u;
  Fn2<ND> r;
  r.nd0 = p.nd0 + (p0 ? c.nd1 : c.nd0);
  r.nd1 = p.nd1 + (p1 ? c.nd1 : c.nd0);
  r.e = (p0 ? c1 : c0) | ((p1 ? c1 : c0) << 1);
  return r;
}
template <typename ND>
__device__ __forceinline__ Fn2<ND> fn_shfl_up(const Fn2<ND>& f, uint32_t d) {
  return Fn2<ND>{__shfl_up_sync(0xFFFFFFFFu, f.e, d), __shfl_up_sync(0xFFFFFFFFu, f.nd0, d),
                 __shfl_up_sync(0xFFFFFFFFu, f.nd1, d)};
}

// Builds nodes[] (8 operation symbols per u32) and dlist[] (first-entry nibble index of each delta
// operation) from the symbol stream. Each thread takes a contiguous run of stream words: it
// summarises the run for both entering states, a block-wide scan of the summaries gives every run
// its entering state and its node and delta bases, and the runs then write their operation
// nibbles. scan_tmp: 5 (NT / 32) + 5 words (8-byte aligned). wst (may be NULL): one word per
// stream word, where the first pass leaves each word's automaton masks for the second. WIDE counts
// nodes in 32 bits (needed from 2^16 nodes on, b = 64), otherwise in 16.
template <int NT, bool WIDE>
__device__ ParseOut parse_stream(const uint32_t* sw, uint32_t S, uint32_t* nodes, uint32_t nodes_words,
                                 uint32_t* dlist, uint32_t dcap, uint32_t* scan_tmp, uint32_t* wst, int* s_err,
                                 bool short_delta) {
  using ND = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
  using F = Fn2<ND>;
  constexpr uint32_t K = WIDE ? 32u : 16u;
  constexpr ND NMASK = WIDE ? (ND)0xFFFFFFFFu : (ND)0xFFFFu;
  constexpr uint32_t NW = NT / 32;
  ND* tnd = reinterpret_cast<ND*>(scan_tmp);  // [2 (NW + 1)] node / delta counts
  uint32_t* te = scan_tmp + 2 * (NW + 1) * (sizeof(ND) / 4);  // [NW + 1] exit states
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t T = (S + 7u) >> 3;  // stream words
  const uint32_t WP = (T + NT - 1) / NT;
  const uint32_t w0 = min(tid * WP, T), w1 = min(w0 + WP, T);
  // 1. this run's summary for entering state 0 and 1
  F f = fn_id<ND>();
  {
    uint32_t s0 = 0, s1 = 1;
    for (uint32_t w = w0; w < w1; ++w) {
      const uint32_t x = sw[w];
      const uint32_t nv = min(8u, S - 8u * w);
      uint32_t D, A, B, e0, e1;
      word_states(x, D, A, B, short_delta);
      const uint32_t m0 = word_ops(A, B, s0, nv, &e0), m1 = word_ops(A, B, s1, nv, &e1);
      if (wst) wst[w] = m0 | (m1 << 8) | (D << 16);  // this word's operations on both paths
      f.nd0 += (ND)__popc(m0) | ((ND)__popc(m0 & D) << K);
      f.nd1 += (ND)__popc(m1) | ((ND)__popc(m1 & D) << K);
      s0 = e0;
      s1 = e1;
    }
    f.e = s0 | (s1 << 1);
  }
  // 2. exclusive scan of the summaries over the block (warp shuffles, then the warp totals)
  F inc = f;
#pragma unroll
  for (uint32_t d = 1; d < 32; d <<= 1) {
    const F p = fn_shfl_up(inc, d);
    if (lane >= d) inc = fn_then(p, inc);
  }
  if (lane == 31) { te[warp] = inc.e; tnd[2 * warp] = inc.nd0; tnd[2 * warp + 1] = inc.nd1; }
  __syncthreads();
  if (warp == 0) {
    F v = lane < NW ? F{te[lane], tnd[2 * lane], tnd[2 * lane + 1]} : fn_id<ND>();
    F vi = v;
#pragma unroll
    for (uint32_t d = 1; d < NW; d <<= 1) {
      const F p = fn_shfl_up(vi, d);
      if (lane >= d) vi = fn_then(p, vi);
    }
    F ex = fn_shfl_up(vi, 1);
    if (lane == 0) ex = fn_id<ND>();
    __syncwarp();
    if (lane < NW) { te[lane] = ex.e; tnd[2 * lane] = ex.nd0; tnd[2 * lane + 1] = ex.nd1; }
    if (lane == NW - 1) { te[NW] = vi.e; tnd[2 * NW] = vi.nd0; }
  }
  __syncthreads();
  F pre = fn_shfl_up(inc, 1);
  if (lane == 0) pre = fn_id<ND>();
  pre = fn_then(F{te[warp], tnd[2 * warp], tnd[2 * warp + 1]}, pre);
  uint32_t st = pre.e & 1u;  // the stream starts in state 0
  const uint32_t path = st;  // which of the two paths of the first pass this run takes
  uint32_t j = (uint32_t)(pre.nd0 & NMASK), d = (uint32_t)(pre.nd0 >> K);
  const uint32_t total_e = te[NW] & 1u;
  const ND total_nd = tnd[2 * NW];
  // the node words this run shares with its neighbours start at zero
  const uint32_t jend = j + (uint32_t)((st ? f.nd1 : f.nd0) & NMASK);
  if ((j >> 3) < nodes_words) nodes[j >> 3] = 0u;
  if ((jend >> 3) < nodes_words) nodes[jend >> 3] = 0u;
  __syncthreads();
  // 3. write this run's operation nibbles and delta positions
  const uint32_t jstart = j;
  uint64_t acc = 0;
  for (uint32_t w = w0; w < w1; ++w) {
    const uint32_t x = sw[w];
    const uint32_t nv = min(8u, S - 8u * w);
    uint32_t D, m;
    if (wst) {
      const uint32_t v = wst[w];
      m = (v >> (8u * path)) & 0xFFu;
      D = v >> 16;
    } else {
      uint32_t A, B, end;
      word_states(x, D, A, B, short_delta);
      m = word_ops(A, B, st, nv, &end);
      st = end;
    }
    const uint32_t cnt = __popc(m);
    const uint32_t p = j & 7u;
    acc |= (uint64_t)pack_nibbles(x, m) << (4u * p);
    j += cnt;
    if (p + cnt >= 8u) {  // node word (j - cnt) / 8 is complete
      const uint32_t wi = (j - cnt) >> 3;
      if (wi < nodes_words) {
        if (wi == (jstart >> 3)) atomicOr(&nodes[wi], (uint32_t)acc);
        else nodes[wi] = (uint32_t)acc;
      }
      acc >>= 32;
    }
    uint32_t dm = m & D;
    while (dm) {
      const uint32_t b = __ffs(dm) - 1u;
      dm &= dm - 1u;
      if (d < dcap) dlist[d] = 8u * w + b + 1u;  // first entry; resolved after the parse
      ++d;
    }
  }
  if ((j & 7u) && (j >> 3) < nodes_words) atomicOr(&nodes[j >> 3], (uint32_t)acc);
  if (tid == 0 && total_e != 0) set_err(s_err, VC_ERR_CORRUPT);  // the stream ends inside a delta entry chain
  ParseOut out;
  out.n_nodes = (uint32_t)(total_nd & NMASK);
  out.n_delta = (uint32_t)(total_nd >> K);
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
  const uint32_t* dlist;
  uint32_t dlist_cap;
  uint32_t op_mask;
  int* s_err;
};

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
// sw: its symbols as packed nibbles (u32 aligned); out: the slot, (b >> lod)^3 labels or packed
// palette indices (P.pal_bits).
// on_stage_free() is called by every thread exactly once, as soon as the staged record is no longer
// read: right after the finest grid is filled when the palette fits its shared copy, else at the end.
// S_use: symbols to parse (0: all; fewer: a coarser level of detail needs only the stream's
// prefix up to its level, and the counts of the whole stream are then upper bounds).
template <int L, typename GT, bool RANS, int NT, typename Hook>
__device__ void decode_brick(const Params& P, const uint32_t* head, const uint32_t* sw, uint32_t* out,
                             unsigned char* sm, unsigned char* gm, int* s_err, uint32_t S_use, Hook&& on_stage_free) {
  constexpr uint32_t NW = NT / 32;
  constexpr uint32_t MARK = GridT<GT>::MARK;
  const SmemLayout& SL = P.v.sm;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  uint32_t* misc = reinterpret_cast<uint32_t*>(sm + SL.misc_off);
  uint32_t* wtot = misc + 16;      // NW warp totals (words 16..47)
  uint32_t* scan_tmp = misc + 48;  // 5 NW + 5 words (48..255), 8-byte aligned

  // large regions: the scratch slice (gm), or shared memory for those the layout put there (b = 64)
  auto big = [&](uint32_t bit) -> unsigned char* { return (L >= 6 && (SL.big_sm & bit)) ? sm : gm; };
  const uint32_t n_pal = head[0], S_rec = head[1], nd = head[3];
  const bool truncated = S_use != 0u && S_use < S_rec;
  const uint32_t S = truncated ? S_use : S_rec;
  const bool short_delta = (P.v.flags & kFlagShortDelta) != 0;
  const uint32_t ns = RANS ? head_words(S_rec, runs_k(P.v.flags)) : 0u;  // rANS states and run starts

  BrickCtx c;
  c.pal = head + 4 + ns;
  c.n_pal = n_pal;
  const bool pal_copied = n_pal <= SL.pal_cap;
  if (pal_copied) {  // a private copy of the palette frees the stage before the output pass; byte
                     // grids get 256 entries (zero padded) so that any byte index stays in bounds
    uint32_t* pc = reinterpret_cast<uint32_t*>(sm + SL.pal_off);
    for (uint32_t i = tid; i < SL.pal_cap; i += NT) pc[i] = i < n_pal ? c.pal[i] : 0u;
    c.pal = pc;  // read after the barriers of the steps below
  }
  c.op_mask = P.v.op_mask;
  c.s_err = s_err;
  uint32_t* dlist = reinterpret_cast<uint32_t*>(big(kBigDelta) + SL.dlist_off);
  c.dlist = dlist;
  c.dlist_cap = nd < SL.dlist_cap ? nd : SL.dlist_cap;

  // 1. operations per node
  if (nd == 0 && SL.stage_alias) {
    // the symbols are the operations; copied out of the stage, which step 2 overwrites
    uint32_t* nodes = reinterpret_cast<uint32_t*>(big(kBigNodes) + SL.nodes_off);
    const uint32_t nw = min((S + 7u) / 8u + 2u, SL.nodes_words);
    for (uint32_t i = tid; i < nw; i += NT) nodes[i] = sw[i];
    c.nodes = nodes;
    c.n_nodes = S;
    __syncthreads();
  } else if (nd == 0) {
    c.nodes = sw;
    c.n_nodes = S;
  } else {
    uint32_t* nodes = reinterpret_cast<uint32_t*>(big(kBigNodes) + SL.nodes_off);
    // the finest grid's region is idle during the parse: it keeps the per-word automaton masks
    uint32_t* wst = ((S + 7u) >> 3) * 4u <= SL.wst_bytes ? reinterpret_cast<uint32_t*>(big(kBigFg) + SL.wst_off) : nullptr;
    const ParseOut po = parse_stream<NT, (L >= 6)>(sw, S, nodes, SL.nodes_words, dlist, c.dlist_cap, scan_tmp, wst, s_err,
                                                   short_delta);
    // a stream whose delta count is off may claim more nodes than the layout holds (it is sized
    // for the volume's largest S - n_delta): flagged, and cut to what the regions hold
    const uint32_t ncap = 32u * (SL.nwords - 2u);
    c.nodes = nodes;
    c.n_nodes = min(po.n_nodes, ncap);
    if ((truncated ? po.n_delta > nd : po.n_delta != nd) || po.n_nodes > ncap) set_err(s_err, VC_ERR_CORRUPT);
    // delta values from their entries, one delta operation per thread (visible after the barriers
    // of step 2)
    for (uint32_t d = tid; d < c.dlist_cap; d += NT) dlist[d] = read_delta(sw, dlist[d], S, short_delta);
    if (SL.stage_alias) __syncthreads();  // the stage is read up to here; step 2 overwrites it
  }

  // 2. palette-cursor masks and prefix counts (32 nodes per word)
  uint32_t* adv_mask = reinterpret_cast<uint32_t*>(big(kBigMasks) + SL.mask_off);
  uint32_t* del_mask = adv_mask + SL.nwords;
  // prefix counts: 16 bits while a brick has fewer than 2^16 nodes (b <= 32), 32 bits beyond
  using Pre = typename std::conditional<(L >= 6), uint32_t, uint16_t>::type;
  Pre* adv_pre = reinterpret_cast<Pre*>(adv_mask + 2 * SL.nwords);
  Pre* del_pre = adv_pre + SL.nwords;
  c.adv_mask = adv_mask; c.del_mask = del_mask;
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
      adv_pre[w] = (Pre)pa; del_pre[w] = (Pre)pd;
      pa += __popc(adv_mask[w]); pd += __popc(del_mask[w]);
    }
    if (tid == 0 && (truncated ? (ta > n_pal || td > nd) : (ta != n_pal || td != nd))) set_err(s_err, VC_ERR_CORRUPT);
  }
  __syncthreads();

  // 3. coarse levels 0..L-1, parent-major. G: palette index per cell (Morton order, levels
  // 0..L-1). NS: for level l >= 1, one byte per level-(l-1) cell whose bit o says that child o
  // was emitted with stop bit 0. The stop-0 cells of a level, in rank (= stream) order, go to one
  // of two lists; the next level's children of rank r are nodes off + 8 r .. off + 8 r + 7.
  const uint32_t Lout = (uint32_t)L - P.lod;
  const uint32_t last_coarse = Lout < (uint32_t)L ? Lout : (uint32_t)L - 1u;
  GT* G = reinterpret_cast<GT*>(sm + SL.g_off);
  uint8_t* NS = sm + SL.ns_off;
  uint16_t* lists[2] = {reinterpret_cast<uint16_t*>(sm + SL.list_off),
                        reinterpret_cast<uint16_t*>(sm + SL.list_off) + SL.list0_cap};
  const bool no_stop = (P.v.flags & kFlagNoStop) != 0;
  constexpr uint32_t b = 1u << L;
  const bool finest = Lout == (uint32_t)L;
  GT* fg = reinterpret_cast<GT*>(big(kBigFg) + SL.fg_off);

  // the 8 children (nodes j0 .. j0+7) of a stop-0 cell with index gp at coordinates (px, py, pz):
  // palette indices or neighbour marks into v, returns the children emitted with stop bit 0
  auto decode8 = [&](uint32_t j0, uint32_t gp, uint32_t px, uint32_t py, uint32_t pz, bool at_finest,
                     uint32_t (&v)[8]) -> uint32_t {
    if (j0 + 8u > c.n_nodes) {
      set_err(s_err, VC_ERR_CORRUPT);
#pragma unroll
      for (int o = 0; o < 8; ++o) v[o] = 0;
      return 0;
    }
    const uint32_t ops = nib8_at(c.nodes, j0);
    // per-child class masks (SWAR over the 8 operation nibbles)
    const uint32_t m_nx = nib_eq8(ops, OP_NX), m_ny = nib_eq8(ops, OP_NY), m_nz = nib_eq8(ops, OP_NZ);
    const uint32_t m_7 = nib_eq8(ops, 7u);
    const uint32_t m_pal = gather_nib_bits((ops & 0x44444444u) >> 2) & ~m_7;  // advance, last, delta
    bool bad = ((ops & 0x88888888u) != 0 && (at_finest || no_stop)) || m_7 != 0;
    // a neighbour copy needs that coordinate even (child bit 0) and > 0
    bad |= (m_nx & ~(px ? 0x55u : 0u)) | (m_ny & ~(py ? 0x33u : 0u)) | (m_nz & ~(pz ? 0x0Fu : 0u));
    if (c.op_mask != 0x7Fu) {
#pragma unroll
      for (uint32_t o = 0; o < 7; ++o)
        if (!((c.op_mask >> o) & 1u)) bad |= nib_eq8(ops, o) != 0;
    }
    // parent copies and neighbour marks
#pragma unroll
    for (uint32_t o = 0; o < 8; ++o) {
      const uint32_t op = (ops >> (4u * o)) & 7u;
      v[o] = op == OP_PARENT ? gp : MARK + op - OP_NX;
    }
    if (m_pal) {  // palette reads (a minority of nodes): cursor from the masks
      const uint32_t adv8 = bits8_at(adv_mask, j0), del8 = bits8_at(del_mask, j0);
      const uint32_t w = j0 >> 5, lt = (1u << (j0 & 31u)) - 1u;
      const uint32_t k0 = adv_pre[w] + __popc(adv_mask[w] & lt);
      const uint32_t dd0 = del_pre[w] + __popc(del_mask[w] & lt);
      // the group's cursor stays within the palette: its advances read entries k0 .. k0 + na - 1,
      // last / delta children read below the cursor (a corrupt cursor may run past the palette,
      // and an index out of range could pass for a neighbour mark)
      bad |= k0 + (uint32_t)__popc(adv8) > n_pal;
#pragma unroll
      for (uint32_t o = 0; o < 8; ++o) {
        if ((m_pal >> o) & 1u) {
          const uint32_t op = (ops >> (4u * o)) & 7u;
          const uint32_t below = (1u << o) - 1u;
          const uint32_t k = k0 + __popc(adv8 & below);
          if (op == OP_ADV) {
            v[o] = k;
          } else if (op == OP_LAST) {
            bad |= k == 0u;
            v[o] = k - 1u;
          } else {
            const uint32_t di = dd0 + __popc(del8 & below);
            const uint32_t delta = di < c.dlist_cap ? dlist[di] : 0u;
            bad |= delta == 0u || delta > k;
            v[o] = k - delta;
          }
        }
      }
    }
    if (bad) {
      set_err(s_err, VC_ERR_CORRUPT);
#pragma unroll
      for (int o = 0; o < 8; ++o) v[o] = 0;  // keep invalid indices out of the grids
    }
    return gather_nib_bits((~ops & 0x88888888u) >> 3);  // children with stop bit 0
  };
  auto store8 = [&](GT* dst, const uint32_t (&v)[8]) {  // 8 consecutive cells
    if constexpr (sizeof(GT) == 1) {
      *reinterpret_cast<uint2*>(dst) = make_uint2(v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24),
                                                  v[4] | (v[5] << 8) | (v[6] << 16) | (v[7] << 24));
    } else {
      *reinterpret_cast<uint4*>(dst) = make_uint4(v[0] | (v[1] << 16), v[2] | (v[3] << 16), v[4] | (v[5] << 16),
                                                  v[6] | (v[7] << 16));
    }
  };

  // The same decode as decode8 for parent cell p (Morton code) with the children's cells packed
  // (Cells8) and the neighbour legality, class masks and marks taken by SWAR over op bytes; the
  // children emitted with stop bit 0 go to open8.
  // Palette reads of the sibling group at nodes j0 .. j0+7 (operations ops; e: child o's
  // operation in byte o & 3 of e[o >> 2]): the cursor k0 (advances before node j0) and the delta
  // operations dd0 before it come from the masks; per child, exclusive prefix counts within the
  // group. The advance / last / delta children of v get their palette indices.
  auto palette8 = [&](uint32_t j0, uint32_t ops, const uint32_t (&e)[2], Cells8<GT>& v, bool& bad) {
    uint32_t adv[2], lst[2], del[2], palm[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t x = e[h];
      const uint32_t ge4 = (x + 0x7C7C7C7Cu) & 0x80808080u, ge5 = (x + 0x7B7B7B7Bu) & 0x80808080u;
      const uint32_t ge6 = (x + 0x7A7A7A7Au) & 0x80808080u, eq7 = (x + 0x79797979u) & 0x80808080u;
      adv[h] = (ge4 & ~ge5) >> 7;  // 0x01 per advance byte
      lst[h] = (ge5 & ~ge6) >> 7;
      del[h] = (ge6 & ~eq7) >> 7;
      palm[h] = ((ge4 & ~eq7) >> 7) * 0xFFu;
    }
    const uint32_t w = j0 >> 5, lt = (1u << (j0 & 31u)) - 1u;
    const uint32_t k0 = adv_pre[w] + __popc(adv_mask[w] & lt);
    const uint32_t dd0 = del_pre[w] + __popc(del_mask[w] & lt);
    const uint32_t na0 = (adv[0] * 0x01010101u) >> 24, nd0 = (del[0] * 0x01010101u) >> 24;
    // Both paths below check that the cursor stays within the palette: an advance reads entry
    // k < |P|, last / delta children read below the cursor k <= |P| (a corrupt cursor may run
    // past the palette, and an index out of range could pass for a neighbour mark).
    const uint32_t ndel = nd0 + ((del[1] * 0x01010101u) >> 24);
    bool bytewise = false;
    if constexpr (sizeof(GT) == 1) bytewise = ndel <= 4u;
    if (bytewise) {
      // 8-bit grids: the cursor stays below 252 (checked next, in full width: it also keeps every
      // cursor byte of the bytewise computation from wrapping), so all eight children are
      // computed bytewise: k per byte, the group's delta values by byte permutation (up to four
      // of them; more in one group take the loop below)
      const uint32_t K[2] = {k0 * 0x01010101u + adv[0] * 0x01010100u,
                             (k0 + na0) * 0x01010101u + adv[1] * 0x01010100u};
      const uint32_t Dp[2] = {del[0] * 0x01010100u, nd0 * 0x01010101u + del[1] * 0x01010100u};
      bad |= k0 + na0 + ((adv[1] * 0x01010101u) >> 24) > n_pal;  // the cursor after the group <= |P|
      uint32_t d4 = 0u;
#pragma unroll
      for (uint32_t i = 0; i < 4; ++i) {
        const uint32_t di = dd0 + i;
        if (i < ndel) d4 |= (di < c.dlist_cap ? min(dlist[di], 255u) : 0u) << (8u * i);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t t = Dp[h] | (Dp[h] >> 4);
        t &= 0x00FF00FFu;
        const uint32_t sel = (t | (t >> 8)) & 0xFFFFu;  // byte i of Dp -> nibble i
        const uint32_t delm = del[h] * 0xFFu, lstm = lst[h] * 0xFFu;
        const uint32_t D = __byte_perm(d4, 0u, sel) & delm;
        bad |= (__vcmpeq4(K[h], 0u) & lstm) != 0u;                        // last: k >= 1
        bad |= ((__vcmpeq4(D, 0u) | __vcmpgtu4(D, K[h])) & delm) != 0u;   // delta: 1 <= delta <= k
        const uint32_t idx = K[h] - lst[h] - D;
        v.w[h] = (v.w[h] & ~palm[h]) | (idx & palm[h]);
      }
    } else {
      // 16-bit grids, or more than four delta operations in the group: child by child
      const uint32_t adv8 = byte_msbs(adv[0] << 7) | (byte_msbs(adv[1] << 7) << 4);
      const uint32_t del8 = byte_msbs(del[0] << 7) | (byte_msbs(del[1] << 7) << 4);
      uint32_t mp = byte_msbs(palm[0]) | (byte_msbs(palm[1]) << 4);
      while (mp) {
        const uint32_t o = __ffs(mp) - 1u;
        mp &= mp - 1u;
        const uint32_t op = (ops >> (4u * o)) & 7u;
        const uint32_t below = (1u << o) - 1u;
        const uint32_t k = k0 + __popc(adv8 & below);
        uint32_t idx;
        if (op == OP_ADV) {
          idx = k;
        } else if (op == OP_LAST) {
          bad |= k == 0u;
          idx = k - 1u;
        } else {
          const uint32_t di = dd0 + __popc(del8 & below);
          const uint32_t delta = di < c.dlist_cap ? dlist[di] : 0u;
          bad |= delta == 0u || delta > k;
          idx = k - delta;
        }
        set_cell<GT>(v, o, idx & (sizeof(GT) == 1 ? 0xFFu : 0xFFFFu));
        bad |= k + ((adv8 >> o) & 1u) > n_pal;  // advance: k < |P|; last / delta: k <= |P|
      }
    }
  };
  // The same decode as decode8 for parent cell p (Morton code), with the children's cells packed
  // (Cells8): the checks run on the 8 operation nibbles at once, parent copies and neighbour
  // marks are merged bytewise. The children emitted with stop bit 0 go to open8. With defer_pal
  // the palette reads are left to the caller (has_pal: the group has some; their cells hold gp).
  auto decode8p = [&](uint32_t j0, uint32_t gp, uint32_t p, bool at_finest, bool defer_pal, uint32_t& open8,
                      bool& has_pal) -> Cells8<GT> {
    Cells8<GT> v;
    if (j0 + 8u > c.n_nodes) {
      set_err(s_err, VC_ERR_CORRUPT);
#pragma unroll
      for (auto& x : v.w) x = 0u;
      open8 = 0u;
      has_pal = false;
      return v;
    }
    const uint32_t ops = nib8_at(c.nodes, j0);
    if (!at_finest) open8 = gather_nib_bits((~ops & 0x88888888u) >> 3);
    bool bad = (ops & 0x88888888u) != 0u && (at_finest || no_stop);
    // per operation nibble (low 3 bits): >= 1, >= 4, == 7
    const uint32_t x = ops & 0x77777777u;
    const uint32_t ge1 = (x + 0x77777777u) & 0x88888888u, ge4 = (x + 0x44444444u) & 0x88888888u;
    const uint32_t eq7 = (x + 0x11111111u) & 0x88888888u;
    // a neighbour copy along axis a is legal only for children whose coordinate a is even, in a
    // parent whose coordinate a is > 0: allowed axes of child o = (7 - o) & (positive axes of p)
    const uint32_t axm = ((p & 0x09249249u) ? 1u : 0u) | ((p & 0x12492492u) ? 2u : 0u) | ((p & 0x24924924u) ? 4u : 0u);
    const uint32_t axis_bit = x + (x & (x >> 1) & 0x11111111u);  // ops 1, 2, 3 -> 1, 2, 4
    const uint32_t nbn = ((ge1 & ~ge4) >> 3) * 0xFu;            // nibbles of neighbour copies
    bad |= (axis_bit & ~(0x01234567u & (axm * 0x11111111u)) & nbn) != 0u || eq7 != 0u;
    has_pal = (ge4 & ~eq7) != 0u;
    // child o's operation in byte o & 3 of e[o >> 2]
    const uint32_t e[2] = {nib4_to_bytes(x & 0xFFFFu), nib4_to_bytes(x >> 16)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t xb = e[h];
      const uint32_t nbm = ((((xb + 0x7F7F7F7Fu) & ~(xb + 0x7C7C7C7Cu)) & 0x80808080u) >> 7) * 0xFFu;
      if constexpr (sizeof(GT) == 1) {
        v.w[h] = ((gp * 0x01010101u) & ~nbm) | ((xb | 0xFCFCFCFCu) & nbm);  // MARK + axis = 0xFC | op
      } else {
        // 16-bit cells: two children per word
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const uint32_t lo = (xb >> (16 * q)) & 0xFFu, hi = (xb >> (16 * q + 8)) & 0xFFu;
          const uint32_t vlo = (lo >= 1u && lo <= 3u) ? 0xFFFCu | lo : gp;
          const uint32_t vhi = (hi >= 1u && hi <= 3u) ? 0xFFFCu | hi : gp;
          v.w[2 * h + q] = vlo | (vhi << 16);
        }
      }
    }
    if (c.op_mask != 0x7Fu) {
#pragma unroll
      for (uint32_t o = 0; o < 7; ++o)
        if (!((c.op_mask >> o) & 1u)) bad |= nib_eq8(ops, o) != 0;
    }
    if (has_pal && !defer_pal) palette8(j0, ops, e, v, bad);
    if (bad) {
      set_err(s_err, VC_ERR_CORRUPT);
#pragma unroll
      for (auto& w : v.w) w = 0u;  // keep invalid indices out of the grids
      has_pal = false;
    }
    return v;
  };

  // level 0: the root (node 0) must be a palette advance
  if (tid == 0) {
    uint32_t ns0 = 0, g0 = 0;
    if (c.n_nodes == 0) {
      set_err(s_err, VC_ERR_CORRUPT);
    } else {
      const uint32_t s0 = nib_at(c.nodes, 0);
      if ((s0 & 7u) != OP_ADV || n_pal == 0 || ((s0 >> 3) && no_stop)) set_err(s_err, VC_ERR_CORRUPT);
      ns0 = (s0 >> 3) ? 0u : 1u;
    }
    G[0] = (GT)g0;
    lists[0][0] = 0;
    misc[8] = ns0;
    misc[9] = 0u;  // finest level, label output: open cells queued for palette reads
  }
  __syncthreads();
  const bool root_open = misc[8] != 0;
  // level grids: the root at 0, level l >= 1 at 8 + (8^l - 8) / 7, so that every 8 siblings are
  // one aligned 8-cell group (stored with one vector store)
  uint32_t off = 1, npar = root_open ? 1u : 0u, gofs_prev = 0, gofs = 8, nsofs_prev = 0, nsofs = 0;
  // is level-l cell p emitted with stop bit 0?  (l >= 1: from the level's NS bytes)
  auto open_cell = [&](uint32_t l, uint32_t p, uint32_t nso) -> bool {
    return l == 0 ? root_open : ((NS[nso + (p >> 3)] >> (p & 7u)) & 1u) != 0;
  };
  for (uint32_t l = 1; l <= last_coarse; ++l) {
    const uint32_t parents = 1u << (3u * (l - 1u));
    GT* Gl = G + gofs;
    const GT* Gp = G + gofs_prev;
    uint8_t* NSl = NS + nsofs;  // this level's bytes (indexed by parent)
    const uint16_t* list_prev = lists[(l - 1u) & 1u];
    uint16_t* list_cur = lists[l & 1u];
    // children of stopped (or not emitted) parents inherit the parent's index
    for (uint32_t p = tid; p < parents; p += NT) {
      if (!open_cell(l - 1u, p, nsofs_prev)) {
        const uint32_t g = Gp[p];
        const uint32_t v[8] = {g, g, g, g, g, g, g, g};
        store8(Gl + 8u * p, v);
        NSl[p] = 0;
      }
    }
    // children of stop-0 parents: a contiguous run of ranks per thread
    const uint32_t per = (npar + NT - 1u) / NT;
    const uint32_t r0 = min(tid * per, npar), r1 = min(r0 + per, npar);
    uint32_t cnt = 0;
    for (uint32_t r = r0; r < r1; ++r) {
      const uint32_t p = list_prev[r];
      uint32_t open8;
      bool has_pal;
      store_cells8<GT>(Gl + 8u * p, decode8p(off + 8u * r, Gp[p], p, false, false, open8, has_pal));
      NSl[p] = (uint8_t)open8;
      cnt += __popc(open8);
    }
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= (uint32_t)o) inc += t;
    }
    if (lane == 31) wtot[warp] = inc;
    __syncthreads();
    // the warp totals, scanned by every warp with shuffles
    uint32_t wt = lane < NW ? wtot[lane] : 0u;
#pragma unroll
    for (uint32_t o = 1; o < NW; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, wt, o);
      if (lane >= o) wt += t;
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, wt, NW - 1u);
    uint32_t base = inc - cnt + (warp ? __shfl_sync(0xFFFFFFFFu, wt, warp - 1u) : 0u);
    // list this level's stop-0 cells by rank (a corrupt stream may claim more than the buffer
    // holds: flagged, and the list is cut); resolve the neighbour marks among the children
    const uint32_t lcap = (l & 1u) ? SL.list1_cap : SL.list0_cap;
    for (uint32_t r = r0; r < r1; ++r) {
      const uint32_t p = list_prev[r];
      uint32_t open8 = NSl[p];
      while (open8) {
        const uint32_t o = __ffs(open8) - 1u;
        open8 &= open8 - 1u;
        if (base < lcap) {
          list_cur[base] = (uint16_t)(8u * p + o);
        } else {  // cut: the cell counts as stopped from here on, so that every cell of the next
                  // levels is still written (inherited) and the stop bits match the ranks
          set_err(s_err, VC_ERR_CORRUPT);
          NSl[p] &= (uint8_t)~(1u << o);
        }
        ++base;
      }
    }
    // one child per thread: the chains are short, dependent loads, so spread them out
    for (uint32_t cc = tid; cc < 8u * npar; cc += NT) {
      const uint32_t m = 8u * list_prev[cc >> 3] + (cc & 7u);
      const uint32_t g = Gl[m];
      if (g >= MARK) Gl[m] = (GT)resolve_morton<GT>(Gl, m, g, s_err);
    }
    __syncthreads();
    off += 8u * npar;
    npar = min(total, lcap);
    gofs_prev = gofs;
    gofs += 1u << (3u * l);
    nsofs_prev = nsofs;
    nsofs += (parents + 3u) & ~3u;  // the next level's bytes start 4-byte aligned
  }

  bool cells_path = false;
  if constexpr (L >= 2 && L <= 6) {
    if (finest && !P.pal_bits) {
      // 4'. finest level with label output. The finest voxels of a level-(L-1) cell that was not
      // emitted with stop bit 0 all hold that cell's index (in the level grid); only the open
      // cells' 8 children are decoded, into a buffer by rank (Cells8 each). The output pass then
      // reads, per pair of x-adjacent cells, the level grid or the children, and writes 4 rows
      // of 4 labels.
      cells_path = true;
      if (tid == 0 && off + 8u * npar != c.n_nodes) set_err(s_err, VC_ERR_CORRUPT);
      const GT* Gp = G + gofs_prev;  // level L-1, neighbour marks resolved
      // open level-(L-1) cells as a bit array in Morton order (the level's stop bytes)
      const uint32_t* ns32 = reinterpret_cast<const uint32_t*>(NS + nsofs_prev);
      uint16_t* rpre = reinterpret_cast<uint16_t*>(sm + SL.rank_off);  // rank of the first open cell of each 32
      const uint16_t* plist = lists[(L - 1u) & 1u];
      GT* cb = reinterpret_cast<GT*>(big(kBigFg) + SL.fg_off);
      // rank of open cell m (bit m of ns32 set)
      auto rank_of = [&](uint32_t m, uint32_t w) -> uint32_t {
        return rpre[m >> 5] + __popc(w & ((1u << (m & 31u)) - 1u));
      };
      // 8-bit grids leave the palette reads to a pass over the queued cells only (about a third
      // of them), so that the warps do not all run them; cells beyond the queue's capacity read
      // the palette here
      uint16_t* pq = reinterpret_cast<uint16_t*>(sm + SL.pq_off);
      constexpr bool defer = sizeof(GT) == 1;
      for (uint32_t r = tid; r < npar; r += NT) {
        const uint32_t p = plist[r];
        if ((ns32[p >> 5] & ((1u << (p & 31u)) - 1u)) == 0u) rpre[p >> 5] = (uint16_t)r;
        uint32_t open8;
        bool has_pal;
        const uint32_t j0 = off + 8u * r;
        Cells8<GT> v = decode8p(j0, Gp[p], p, true, defer, open8, has_pal);
        if (defer) {
          const uint32_t act = __activemask();
          const uint32_t bal = __ballot_sync(act, has_pal);
          if (bal) {
            const uint32_t leader = __ffs(act) - 1u;
            uint32_t base = 0u;
            if (lane == leader) base = atomicAdd(misc + 9, (uint32_t)__popc(bal));
            base = __shfl_sync(act, base, leader);
            const uint32_t at = base + __popc(bal & lanemask_lt());
            if (has_pal && at < SL.pq_cap) {
              pq[at] = (uint16_t)r;
            } else if (has_pal) {
              const uint32_t ops = nib8_at(c.nodes, j0);
              const uint32_t x = ops & 0x77777777u;
              const uint32_t e[2] = {nib4_to_bytes(x & 0xFFFFu), nib4_to_bytes(x >> 16)};
              bool bad = false;
              palette8(j0, ops, e, v, bad);
              if (bad) {
                set_err(s_err, VC_ERR_CORRUPT);
#pragma unroll
                for (auto& w : v.w) w = 0u;
              }
            }
          }
        }
        store_cells8<GT>(cb + 8u * r, v);
      }
      __syncthreads();
      if constexpr (defer) {
        const uint32_t nq = min(misc[9], SL.pq_cap);
        for (uint32_t i = tid; i < nq; i += NT) {
          const uint32_t r = pq[i], j0 = off + 8u * r;
          const uint32_t ops = nib8_at(c.nodes, j0);
          const uint32_t x = ops & 0x77777777u;
          const uint32_t e[2] = {nib4_to_bytes(x & 0xFFFFu), nib4_to_bytes(x >> 16)};
          Cells8<GT> v = load_cells8<GT>(cb + 8u * r);
          bool bad = false;
          palette8(j0, ops, e, v, bad);
          if (bad) {
            set_err(s_err, VC_ERR_CORRUPT);
#pragma unroll
            for (auto& w : v.w) w = 0u;
          }
          store_cells8<GT>(cb + 8u * r, v);
        }
        __syncthreads();
      }
      // neighbour marks, one per lane: each warp takes 32 open cells (ranks) at a time, lists
      // their marks in its queue (lane << 3 | child) and its lanes take them in turn. Child o of
      // cell p copying along axis a takes child o | 1 << a of cell p - e_a (a mark again at most
      // twice more: the chain is followed); cells that are not open hold their level-grid value.
      // Marks are replaced in place: a chain that meets a replaced value stops there, with the
      // same result.
      uint8_t* mq = big(kBigQueues) + SL.mq_off + 224u * warp;
      for (uint32_t r0 = warp * 32u; r0 < npar; r0 += NT) {
        const uint32_t r = r0 + lane;
        const uint32_t mm = r < npar ? mark_bits<GT>(load_cells8<GT>(cb + 8u * r)) : 0u;
        const uint32_t cnt = __popc(mm);
        uint32_t inc = cnt;
#pragma unroll
        for (uint32_t d = 1; d < 32u; d <<= 1) {
          const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, d);
          if (lane >= d) inc += t;
        }
        const uint32_t T = __shfl_sync(0xFFFFFFFFu, inc, 31);
        uint32_t pos = inc - cnt;
#pragma unroll
        for (uint32_t o = 0; o < 7; ++o)  // child 7 has every coordinate odd: never a mark
          if ((mm >> o) & 1u) mq[pos++] = (uint8_t)((lane << 3) | o);
        __syncwarp();
        for (uint32_t t = lane; t < T; t += 32u) {
          const uint32_t q = mq[t];
          const uint32_t rr = r0 + (q >> 3), o = q & 7u;
          uint32_t p = plist[rr], oo = o;
          uint32_t g = cb[8u * rr + o];
#pragma unroll 1
          for (int hop = 0; hop < 3 && g >= MARK; ++hop) {
            const uint32_t a = g - MARK;
            p = morton_dec(p, a);
            oo |= 1u << a;
            const uint32_t w = ns32[p >> 5];
            g = ((w >> (p & 31u)) & 1u) ? (uint32_t)cb[8u * rank_of(p, w) + oo] : (uint32_t)Gp[p];
          }
          if (g >= MARK) { set_err(s_err, VC_ERR_CORRUPT); g = 0; }
          cb[8u * rr + o] = (GT)g;
        }
        __syncwarp();
      }
      __syncthreads();
      // output: pair q = (k, cy, cz) covers level-(L-1) cells (2k, cy, cz) and (2k + 1, cy, cz),
      // i.e. voxels x = 4k .. 4k + 3 of rows y = 2cy, 2cy + 1 and z = 2cz, 2cz + 1. Both the
      // cells' Morton code and the rows' offset are additive over disjoint bits of q, so the
      // thread's part and the (unrolled) iteration's part are computed apart.
      constexpr uint32_t n = 1u << (L - 1);           // level-(L-1) cells per axis
      constexpr uint32_t KB = L - 2;                  // bits of k
      constexpr uint32_t NPAIR = n * n * n / 2u;
      auto pair_morton = [](uint32_t q) -> uint32_t {
        const uint32_t k = q & ((n >> 1) - 1u), cy = (q >> KB) & (n - 1u), cz = q >> (KB + L - 1);
        return spread3(2u * k) | (spread3(cy) << 1) | (spread3(cz) << 2);
      };
      auto pair_offset = [](uint32_t q) -> uint32_t {
        const uint32_t k = q & ((n >> 1) - 1u), cy = (q >> KB) & (n - 1u), cz = q >> (KB + L - 1);
        return (2u * cz * b + 2u * cy) * b + 4u * k;
      };
      const uint32_t m_t = pair_morton(tid & (NT - 1u)), o_t = pair_offset(tid & (NT - 1u));
      const uint32_t pmask = pal_copied && sizeof(GT) == 1 ? SL.pal_cap - 1u : 0xFFFFFFFFu;
      auto lab = [&](uint32_t idx) -> uint32_t {
        if constexpr (sizeof(GT) == 1) {
          if (pal_copied) return c.pal[idx & pmask];
        }
        return label_of(c, idx);
      };
#pragma unroll
      for (uint32_t i = 0; i < (NPAIR + NT - 1u) / NT; ++i) {
        if (NPAIR % NT != 0u && tid + i * NT >= NPAIR) break;
        const uint32_t m0 = m_t + pair_morton(i * NT);
        uint32_t* o = out + o_t + pair_offset(i * NT);
        const uint32_t w = ns32[m0 >> 5];
        const uint32_t open2 = (w >> (m0 & 31u)) & 3u;
        const uint32_t ga = Gp[m0], gb = Gp[m0 + 1u];
        const uint32_t r0 = rank_of(m0, w);  // meaningful only if one of the two is open
        Cells8<GT> A, B;
        constexpr uint32_t rep = sizeof(GT) == 1 ? 0x01010101u : 0x00010001u;
        if (open2 & 1u) {
          A = load_cells8<GT>(cb + 8u * r0);
        } else {
#pragma unroll
          for (auto& x : A.w) x = ga * rep;
        }
        if (open2 & 2u) {
          B = load_cells8<GT>(cb + 8u * (r0 + (open2 & 1u)));
        } else {
#pragma unroll
          for (auto& x : B.w) x = gb * rep;
        }
        if constexpr (sizeof(GT) == 1) {
          if (pal_copied) {  // zero-padded power-of-two palette copy: masked bytes index it
            const uint32_t pm4 = pmask * 0x01010101u;
#pragma unroll
            for (uint32_t h = 0; h < 2; ++h) {
              A.w[h] &= pm4;
              B.w[h] &= pm4;
            }
          }
        }
#pragma unroll
        for (uint32_t row = 0; row < 4; ++row) {  // row = dy | dz << 1: children 2 row, 2 row + 1
          uint32_t* dst = o + (row & 1u) * b + (row >> 1) * b * b;
          if constexpr (sizeof(GT) == 1) {
            if (pal_copied) {
              const uint32_t wa = A.w[row >> 1], wb = B.w[row >> 1], k = 2u * (row & 1u);
              store16(dst, c.pal[__byte_perm(wa, 0u, 0x4440u | k)], c.pal[__byte_perm(wa, 0u, 0x4441u | k)],
                      c.pal[__byte_perm(wb, 0u, 0x4440u | k)], c.pal[__byte_perm(wb, 0u, 0x4441u | k)]);
              continue;
            }
          }
          store16(dst, lab(cell_of<GT>(A, 2u * row)), lab(cell_of<GT>(A, 2u * row + 1u)),
                  lab(cell_of<GT>(B, 2u * row)), lab(cell_of<GT>(B, 2u * row + 1u)));
        }
      }
    }
  }
  if (cells_path) {
  } else if (finest) {
    // 4. finest level: constant blocks of stopped level-(L-1) cells, then the 8 operations of each
    // stop-0 cell (from the rank list), the neighbour marks, the output. For b = 32 the index grid
    // holds one z half at a time (levels are in Morton order, whose top bit is z's, so the first
    // half of the level-(L-1) cells and of the rank list covers z < b / 2); the last plane of the
    // first half is kept for the -z neighbours of the second.
    if (tid == 0 && off + 8u * npar != c.n_nodes) set_err(s_err, VC_ERR_CORRUPT);
    const GT* Gp = G + gofs_prev;
    constexpr uint32_t pcells = 1u << (3 * (L - 1));
    constexpr uint32_t NH = L == 5 ? 2u : 1u;  // z halves (b = 64 works in global scratch: one)
    constexpr uint32_t hcells = pcells / NH;                 // level-(L-1) cells per half
    constexpr uint32_t hvox = b * b * b / NH;                // voxels per half
    constexpr uint32_t PC = (hcells + NT - 1) / NT;
    const uint32_t ftid = flin<L>(tid & (NT - 1u) & (hcells - 1u));
    const uint16_t* plist = lists[(L - 1u) & 1u];
    GT* plane = reinterpret_cast<GT*>(sm + SL.plane_off);  // z = b/2 - 1, resolved (NH == 2)
    // ranks of the first half: open cells are listed in increasing Morton order
    uint32_t rsplit = npar;
    if (NH == 2) {
      uint32_t lo = 0, hi = npar;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (plist[mid] < hcells) lo = mid + 1; else hi = mid;
      }
      rsplit = lo;
    }
#pragma unroll 1
    for (uint32_t h = 0; h < NH; ++h) {
      const uint32_t rb = h ? rsplit : 0u, re = (h + 1 < NH) ? rsplit : npar;
#pragma unroll(PC <= 16u ? PC : 8u)
      for (uint32_t k = 0; k < PC; ++k) {
        const uint32_t pl = tid + k * NT;  // with NT a power of two, pl's bits are tid's plus k * NT's
        const uint32_t p = h * hcells + pl;
        if (pl < hcells && !open_cell(L - 1u, p, nsofs_prev)) {
          const uint32_t g = Gp[p];
          const uint32_t f0 = hcells > NT ? ftid + flin<L>(k * NT) : flin<L>(pl);
          store_pair<GT>(fg, f0, g, g);
          store_pair<GT>(fg, f0 + b, g, g);
          store_pair<GT>(fg, f0 + b * b, g, g);
          store_pair<GT>(fg, f0 + b * b + b, g, g);
        }
      }
      for (uint32_t r = rb + tid; r < re; r += NT) {
        const uint32_t p = plist[r];
        uint32_t v[8];
        decode8(off + 8u * r, Gp[p], compact3(p), compact3(p >> 1), compact3(p >> 2), true, v);
        const uint32_t f0 = flin<L>(p) - h * hvox;
        store_pair<GT>(fg, f0, v[0], v[1]);
        store_pair<GT>(fg, f0 + b, v[2], v[3]);
        store_pair<GT>(fg, f0 + b * b, v[4], v[5]);
        store_pair<GT>(fg, f0 + b * b + b, v[6], v[7]);
      }
      __syncthreads();
      // neighbour marks of this half, resolved per decoded block (at most three hops each; a -z
      // hop out of the second half lands on the kept plane, whose values are final)
      // (one row of 2 voxels per thread, 4 threads per block: the chains are short, dependent
      // loads, so spread them out)
      for (uint32_t cc = tid; cc < 4u * (re - rb); cc += NT) {
        const uint32_t row = cc & 3u;
        const uint32_t pos0 = flin<L>(plist[rb + (cc >> 2)]) - h * hvox + (row & 1u) * b + (row >> 1) * (b * b);
#pragma unroll
        for (uint32_t i = 0; i < 2; ++i) {
          const uint32_t pos = pos0 + i;
          uint32_t g = fg[pos];
          if (g >= MARK) {
            int32_t q = (int32_t)pos;
#pragma unroll 1
            for (int hop = 0; hop < 3 && g >= MARK; ++hop) {
              const uint32_t a = g - MARK;
              q -= a == 0 ? 1 : (a == 1 ? (int32_t)b : (int32_t)(b * b));
              g = q >= 0 ? (uint32_t)fg[q] : (NH == 2 ? (uint32_t)plane[q + (int32_t)(b * b)] : MARK + 3u);
            }
            if (g >= MARK) { set_err(s_err, VC_ERR_CORRUPT); g = 0; }
            fg[pos] = (GT)g;
          }
        }
      }
      __syncthreads();
      if (pal_copied && h + 1 == NH) on_stage_free();
      constexpr uint32_t quads = hvox / 4u;
      uint32_t* outh = out + h * hvox;
      // resolves the neighbour marks of voxel pos (at most three hops)
      auto resolve_fg = [&](uint32_t pos, uint32_t g) -> uint32_t {
        int32_t q = (int32_t)pos;
#pragma unroll 1
        for (int hop = 0; hop < 3 && g >= MARK; ++hop) {
          const uint32_t a = g - MARK;
          q -= a == 0 ? 1 : (a == 1 ? (int32_t)b : (int32_t)(b * b));
          g = q >= 0 ? (uint32_t)fg[q] : (NH == 2 ? (uint32_t)plane[q + (int32_t)(b * b)] : MARK + 3u);
        }
        if (g >= MARK) { set_err(s_err, VC_ERR_CORRUPT); g = 0; }
        return g;
      };
      if (P.pal_bits) {
        // cache paletting (Methods, "Cache paletting"): pal_per indices of pal_bits bits in each
        // u32 word, voxels in x-fastest order. A word that straddles the two halves is written
        // with the second, which reads the first half's last voxels from the kept plane.
        const uint32_t E = P.pal_per, I = P.pal_bits;
        const uint32_t wlo = h ? hvox / E : 0u;
        const uint32_t whi = h + 1 < NH ? hvox / E : (b * b * b + E - 1u) / E;
        for (uint32_t w = wlo + tid; w < whi; w += NT) {
          const uint32_t v0 = w * E;
          uint32_t word = 0;
          if (sizeof(GT) == 1 && E <= 8u && v0 >= h * hvox && v0 + 8u <= (h + 1u) * hvox) {
            // byte grid, 8 indices at hand from two or three aligned words
            const uint32_t lv = v0 - h * hvox;
            const uint32_t* g32 = reinterpret_cast<const uint32_t*>(fg) + (lv >> 2);
            const uint32_t sh = (lv & 3u) * 8u;
            const uint32_t lo = __funnelshift_r(g32[0], g32[1], sh);
            const uint32_t hi = sh ? __funnelshift_r(g32[1], g32[2], sh) : g32[1];
#pragma unroll
            for (uint32_t i = 0; i < 8; ++i)
              if (i < E) word |= (((i < 4 ? lo : hi) >> (8u * (i & 3u))) & 0xFFu) << (I * i);
          } else {
            for (uint32_t i = 0; i < E; ++i) {
              const uint32_t v = v0 + i;
              if (v >= b * b * b) break;
              const uint32_t g = v >= h * hvox ? (uint32_t)fg[v - h * hvox] : (uint32_t)plane[v + b * b - hvox];
              word |= g << (I * i);
            }
          }
          out[w] = word;
        }
      } else if constexpr (sizeof(GT) == 1) {
        if (pal_copied) {
          // byte grid and a zero-padded power-of-two palette copy: masked indices stay in bounds,
          // marks are resolved
          const uint32_t* fg32 = reinterpret_cast<const uint32_t*>(fg);
          const uint32_t pm = SL.pal_cap - 1u;
#pragma unroll 4
          for (uint32_t q = tid; q < quads; q += NT) {
            const uint32_t x = fg32[q];
            store16(outh + 4u * q, c.pal[x & pm], c.pal[(x >> 8) & pm], c.pal[(x >> 16) & pm], c.pal[(x >> 24) & pm]);
          }
        } else {
          const uint32_t* fg32 = reinterpret_cast<const uint32_t*>(fg);
          for (uint32_t q = tid; q < quads; q += NT) {
            const uint32_t x = fg32[q];
            uint32_t idx[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) idx[i] = resolve_fg(4u * q + (uint32_t)i, (x >> (8 * i)) & 0xFFu);
            store16(outh + 4u * q, label_of(c, idx[0]), label_of(c, idx[1]), label_of(c, idx[2]), label_of(c, idx[3]));
          }
        }
      } else {
        for (uint32_t q = tid; q < quads; q += NT) {
          const uint2 x = reinterpret_cast<const uint2*>(fg)[q];
          const uint32_t idx[4] = {resolve_fg(4u * q, x.x & 0xFFFFu), resolve_fg(4u * q + 1u, x.x >> 16),
                                   resolve_fg(4u * q + 2u, x.y & 0xFFFFu), resolve_fg(4u * q + 3u, x.y >> 16)};
          store16(outh + 4u * q, label_of(c, idx[0]), label_of(c, idx[1]), label_of(c, idx[2]), label_of(c, idx[3]));
        }
      }
      if (h + 1 < NH) {
        // keep the last plane of this half, then the grid takes the next half
        for (uint32_t i = tid; i < b * b; i += NT) plane[i] = fg[hvox - b * b + i];
        __syncthreads();
      }
    }
  } else {
    // coarse level of detail: the level-Lout grid, x fastest
    const GT* Gl = G + gofs_prev;
    const uint32_t n = 1u << Lout;
    const uint32_t total = n * n * n;
    auto cell = [&](uint32_t t) -> uint32_t {
      const uint32_t x = t & (n - 1u), y = (t >> Lout) & (n - 1u), z = t >> (2 * Lout);
      return Gl[spread3(x) | (spread3(y) << 1) | (spread3(z) << 2)];
    };
    if (P.pal_bits) {  // cache paletting, as at the finest level
      const uint32_t E = P.pal_per, I = P.pal_bits;
      for (uint32_t w = tid; w * E < total; w += NT) {
        uint32_t word = 0;
        for (uint32_t i = 0; i < E && w * E + i < total; ++i) word |= cell(w * E + i) << (I * i);
        out[w] = word;
      }
    } else if (total >= 4u) {
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
  if (cells_path || !finest || !pal_copied) {
    __syncthreads();
    on_stage_free();
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
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// A bulk copy of a record lands within microseconds; a wait that lasts a second has failed.
constexpr uint64_t kWaitBudgetNs = 1000000000ull;
// Bounded wait: gives up once budget_ns of wall-clock time have passed (the clock is read after
// every poll; 2^22 polls at most, whatever the clock says) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t budget_ns = kWaitBudgetNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > budget_ns) break;
  }
  return false;
}


// Where one request item's data lives: the record, and the bytes to stage in shared memory.
struct ItemSrc {
  const uint32_t* rec;     // record in global memory
  const uint32_t* stream;  // symbols in global memory (record for plain, workspace for rANS)
  uint32_t head_bytes;     // staged head (whole record for plain)
  uint32_t stream_bytes;   // staged symbols after the head (rANS only)
  uint32_t S_use;          // symbols to parse: all (0), or the prefix the rANS symbol kernel decoded
                           // for a coarser level of detail
};

template <bool RANS>
__device__ __forceinline__ ItemSrc item_src(const Params& P, uint32_t item, uint32_t brick) {
  ItemSrc s;
  const uint32_t a = P.v.starts[brick], e = P.v.starts[brick + 1];
  s.rec = P.v.records + a;
  if (RANS) {
    const uint32_t np = s.rec[0], S = s.rec[1];
    const uint32_t ns = head_words(S, runs_k(P.v.flags));
    s.head_bytes = (16u + 4u * ns + 4u * np + 15u) & ~15u;
    s.stream = reinterpret_cast<const uint32_t*>(P.ws + (size_t)(item - P.ws_item0) * P.v.sm.ws_stride);
    s.S_use = P.lod >= P.v.prefix_lod ? min(s.stream[P.v.sm.ws_stride / 4u - 1u], S) : 0u;  // the slot's last word
    s.stream_bytes = ((((s.S_use ? s.S_use : S) + 1u) >> 1) + 15u) & ~15u;
  } else {
    s.head_bytes = (e - a) * 4u;
    s.stream = s.rec + 4u + s.rec[0];
    s.stream_bytes = 0;
    s.S_use = 0;
  }
  return s;
}

// One thread block per request item (grid and per-brick schedules).
// 256-thread blocks are held to 48 registers so that five fit an SM (40 warps)
constexpr int min_blocks(int NT) { return NT == 256 ? 5 : 1; }

template <int L, typename GT, bool RANS, int NT>
__global__ void __launch_bounds__(NT, min_blocks(NT)) decode_grid_kernel(const __grid_constant__ Params P) {
  extern __shared__ __align__(128) unsigned char sm[];
  const SmemLayout& SL = P.v.sm;
  int* s_err = reinterpret_cast<int*>(sm + SL.misc_off);
  const uint32_t k = P.item_base + blockIdx.x;
  if (k >= P.n) return;
  const uint32_t item = scheduled_item(P, k);
  const uint32_t brick = P.ids[item];
  if (brick >= P.v.n_bricks) {
    if (threadIdx.x == 0) report(P.status, VC_ERR_ARG, item);
    return;
  }
  if (threadIdx.x == 0) *s_err = 0;
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
  uint32_t* out = P.cache + (size_t)P.slots[item] * P.out_words;
  decode_brick<L, GT, RANS, NT>(P, head, sw, out, sm, sm, s_err, src.S_use, [] {});
  __syncthreads();
  if (threadIdx.x == 0 && *s_err) report(P.status, *s_err, item);
}

// Persistent thread blocks pull items from the work counter in status[2]; while one brick is
// decoded, the next brick's record (and symbols) are already being copied into the other stage
// buffer by the TMA engine.
template <int L, typename GT, bool RANS, int NT>
__global__ void __launch_bounds__(NT, min_blocks(NT)) decode_batched_kernel(const __grid_constant__ Params P) {
  extern __shared__ __align__(128) unsigned char sm[];
  const SmemLayout& SL = P.v.sm;
  uint32_t* misc = reinterpret_cast<uint32_t*>(sm + SL.misc_off);
  int* s_err = reinterpret_cast<int*>(misc);
  uint64_t* bar = reinterpret_cast<uint64_t*>(misc + 4);  // two mbarriers at byte 16
  uint32_t* counter = reinterpret_cast<uint32_t*>(P.status) + 2;
  unsigned char* stage[2] = {sm + SL.stage_off, sm + SL.stage_off + SL.stage_bytes};
  const uint32_t tid = threadIdx.x;
  const uint32_t n = launch_items(P);

  // thread 0: claims the next item and, if it fits, starts copying its data into stage[buf]
  auto claim_and_issue = [&](uint32_t buf) {
    const uint32_t k = atomicAdd(counter, 1u);
    const uint32_t item = k < n ? scheduled_item(P, k) : k;  // >= n: no more items
    misc[1 + buf] = item;
    uint32_t bytes = 0;
    ItemSrc src{};
    if (item < n) {
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
  __syncthreads();
  // stage depth 2: the next item is claimed (and its copy started) while this one is decoded;
  // depth 1: claimed once this one is done
  const bool prefetch = SL.nstage == 2;
  if (tid == 0) claim_and_issue(0);
  uint32_t parity[2] = {0, 0};
  uint32_t buf = 0;
  for (;;) {
    __syncthreads();
    const uint32_t item = misc[1 + buf];
    if (item >= n) break;
    if (tid == 0) {
      *s_err = 0;
      if (prefetch) claim_and_issue(buf ^ 1u);
    }
    // one warp polls the barrier; the block barrier below publishes the staged bytes to the rest
    const bool ok = (tid >> 5) != 0 || mbar_wait_bounded(&bar[buf], parity[buf]);
    parity[buf] ^= 1u;
    // the decision to give up is taken by the whole block (a barrier follows either way)
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        report(P.status, VC_ERR_TIMEOUT, item);
        if (prefetch) mbar_wait_bounded(&bar[buf ^ 1u], parity[buf ^ 1u]);  // the prefetch may be in flight
      }
      return;
    }
    const uint32_t brick = P.ids[item];
    bool released = false;
    if (brick >= P.v.n_bricks) {
      if (tid == 0) report(P.status, VC_ERR_ARG, item);
    } else {
      const ItemSrc src = item_src<RANS>(P, item, brick);
      const bool staged = src.head_bytes + src.stream_bytes <= SL.stage_bytes;
      const uint32_t* head = staged ? reinterpret_cast<const uint32_t*>(stage[buf]) : src.rec;
      const uint32_t* sw = !staged ? src.stream
                                   : (RANS ? reinterpret_cast<const uint32_t*>(stage[buf] + src.head_bytes)
                                           : head + 4u + head[0]);
      uint32_t* out = P.cache + (size_t)P.slots[item] * P.out_words;
      // depth 1: the next item's copy starts as soon as this brick's stage is free
      decode_brick<L, GT, RANS, NT>(P, head, sw, out, sm, sm, s_err, src.S_use, [&] {
        if (!prefetch && tid == 0) claim_and_issue(0);
        released = true;
      });
      __syncthreads();
      if (tid == 0 && *s_err) report(P.status, *s_err, item);
    }
    if (prefetch) {
      buf ^= 1u;
    } else if (!released) {
      __syncthreads();  // every thread is done with stage[0] before it is refilled
      if (tid == 0) claim_and_issue(0);
    }
  }
}

// b = 64: the working set of one brick (about a megabyte: nodes, masks, grids) is beyond shared
// memory, so each persistent block keeps the large regions (node operations, delta values, cursor
// masks, the 64^3 index grid) in its own slice (P.v.sm.gscratch bytes) of a global-memory
// scratch buffer, largely L2-resident, and the rest (scan scratch, palette copy, level grids, stop
// bytes, rank lists) in shared memory, or everything in the slice when those do not fit
// (P.v.sm.total = 0). It reads the record and symbols where they are. Blocks pull items from the
// work counter in status[2] (items item_base + counter).
template <int L, typename GT, bool RANS, int NT>
__global__ void __launch_bounds__(NT) decode_scratch_kernel(const __grid_constant__ Params P, uint8_t* scratch) {
  extern __shared__ __align__(128) unsigned char dyn_sm[];
  __shared__ int s_err;
  __shared__ uint32_t s_item;
  // the large regions: the block's scratch slice, or shared memory when the layout has no slice
  unsigned char* gm = P.v.sm.gscratch ? scratch + (size_t)blockIdx.x * P.v.sm.gscratch : dyn_sm;
  unsigned char* sm = P.v.sm.total ? dyn_sm : gm;
  uint32_t* counter = reinterpret_cast<uint32_t*>(P.status) + 2;
  const uint32_t n = launch_items(P);
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t k = P.item_base + atomicAdd(counter, 1u);
      s_item = k < n ? scheduled_item(P, k) : k;  // >= n: no more items
      s_err = 0;
    }
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= n) break;
    const uint32_t brick = P.ids[item];
    if (brick >= P.v.n_bricks) {
      if (threadIdx.x == 0) report(P.status, VC_ERR_ARG, item);
    } else {
      const ItemSrc src = item_src<RANS>(P, item, brick);
      uint32_t* out = P.cache + (size_t)P.slots[item] * P.out_words;
      decode_brick<L, GT, RANS, NT>(P, src.rec, src.stream, out, sm, gm, &s_err, src.S_use, [] {});
      __syncthreads();
      if (threadIdx.x == 0 && s_err) report(P.status, s_err, item);
    }
    __syncthreads();  // s_item and s_err are taken over by the next item
  }
}

}  // namespace
}  // namespace dev
}  // namespace vc
