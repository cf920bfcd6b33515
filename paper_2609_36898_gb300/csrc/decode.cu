// Brick decoder kernels for sm_103a: CSGV operation streams -> uint32 label bricks.
//
// The Decompress stage works on all requested bricks in parallel (Results, "GPU-based rendering
// pipeline"). Here the work of one brick is split into two kernels so that each runs at the
// parallelism it needs:
//
//  A. rans_symbols_kernel (rANS volumes only): one warp per brick, 4 to 16 bricks per block. The 32
//     interleaved states decode one symbol each per step; the lanes whose state fell below 2^16
//     take the next 16-bit words in lane order (ballot + popc ranks). The symbols (two per byte,
//     the same layout as the plain coder) go to a stream-ordered workspace. Decoding is a serial
//     chain per brick, so many bricks per SM hide its latency. For a level of detail of 1 or
//     more the warp also tells operations from delta entries (a shuffle scan of the 2-state
//     automaton per step) and counts each level's nodes, stops after the target level, and leaves
//     the prefix length for the reconstruction, which parses only that prefix.
//
//  B. reconstruct kernels: one thread block per brick (grid) or persistent blocks pulling bricks
//     from a work counter with a bulk-copy prefetch of the next brick's record (batched):
//       1. parse: the symbol stream alternates between operations and the delta entries that
//          follow a delta operation (Methods, "Compressed segmentation volumes"), a 2-state
//          automaton. Per 32-bit word of 8 symbols, SWAR prefix doubling on 8-bit masks gives the
//          state after every symbol for both entering states at once; each thread summarises a
//          run of words, a block scan composes the runs, and a second pass writes the operations
//          (8 per u32, node-indexed) and the delta positions. Bricks without delta operations
//          skip this: their symbols are the node operations.
//       2. palette cursor: per 32 nodes, SWAR masks of advance / delta operations and exclusive
//          prefix counts, so that any node's cursor k_j is one popc away (Supplementary Fig.
//          "CSGV ablation" caption: advance reads the next entry, last re-reads it, delta re-reads
//          the entry delta back).
//       3. coarse levels 1..L-1, parent-major: the stop-0 cells of a level are listed by rank, and
//          rank r's 8 children are the nodes at offset + 8 r (Results, "CSGV results"). Each
//          thread decodes 8 children at once (SWAR classes of the 8 operation nibbles); neighbour
//          copies are written as marks and then resolved, one child per thread, by walking at
//          most three hops (each hop turns an even coordinate odd, and a copy needs an even one).
//       4. finest level, in two z halves for b = 32: stopped cells fill their 2^3 blocks of the
//          index grid (two cells per store row), stop-0 cells decode their 8 operations, marks are
//          resolved, and the output pass maps indices to labels (16-byte stores) or packs palette
//          indices (cache paletting).
//     The pipelined schedule runs A and B on two library streams chunk by chunk, so that the
//     symbols of one chunk decode while the previous chunk is reconstructed.
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
// rANS symbols: one warp per request item. Table entry per slot: freq | (slot - cum) << 13 |
// symbol << 25. Full steps of 32 symbols run without bounds checks; the last step is guarded.
// Returns true if the stream was consumed exactly and every state ended at 2^16. The coded words
// flow through a register window: lane l holds words wb + l, wb + 32 + l (in use) and the next two
// runs of 32 (loads in flight), so the global-memory latency stays off the state chain.
__device__ __forceinline__ bool rans_steps(const uint32_t* tab, const uint16_t* words, uint32_t nw, uint32_t S,
                                           uint32_t x, uint32_t ns, uint8_t* out, uint32_t lane) {
  const uint32_t lt = lanemask_lt();
  const uint32_t full = S & ~31u;
  uint8_t* o = out + (lane >> 1);
  const bool even = !(lane & 1u);
  auto ld = [&](uint32_t i) -> uint32_t { return i < nw ? (uint32_t)__ldg(words + i) : 0u; };
  uint32_t wb = 0, w0 = ld(lane), w1 = ld(32u + lane), w2 = ld(64u + lane), w3 = ld(96u + lane);
  uint32_t ptr = 0;  // words consumed; ptr - wb < 32 between steps
  bool bad = false;
  auto step = [&](bool active, uint32_t& s) {
    if (active) {
      const uint32_t e = tab[x & (kRansM - 1u)];
      s = e >> 25;
      x = (e & 0x1FFFu) * (x >> 12) + ((e >> 13) & 0xFFFu);
    }
    const bool need = active && x < (1u << 16);
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, need);
    const uint32_t r = ptr - wb + __popc(m & lt);  // < 63
    const uint32_t v0 = __shfl_sync(0xFFFFFFFFu, w0, r & 31u), v1 = __shfl_sync(0xFFFFFFFFu, w1, r & 31u);
    if (need) x = (x << 16) | (r < 32u ? v0 : v1);  // words past the end read as 0; caught by ptr != nw
    ptr += __popc(m);
    if (ptr - wb >= 32u) {  // slide the window by one run of 32 words
      wb += 32u;
      w0 = w1;
      w1 = w2;
      w2 = w3;
      w3 = ld(wb + 96u + lane);
    }
  };
#pragma unroll 8
  for (uint32_t base = 0; base < full; base += 32u) {
    uint32_t s = 0;
    step(true, s);
    const uint32_t hi = __shfl_xor_sync(0xFFFFFFFFu, s, 1);
    if (even) o[base >> 1] = (uint8_t)(s | (hi << 4));
  }
  if (full < S) {
    const uint32_t i = full + lane;
    const bool active = i < S;
    uint32_t s = 0;
    step(active, s);
    const uint32_t hi = __shfl_xor_sync(0xFFFFFFFFu, s, 1);
    if (active && even) o[full >> 1] = (uint8_t)(s | (i + 1 < S ? hi << 4 : 0u));
  }
  bad |= ptr != nw;
  bad |= lane < ns && x != (1u << 16);
  return !__any_sync(0xFFFFFFFFu, bad);
}

// Position (0..31) of the k-th set bit (k >= 1, counted from bit 0) of m; m holds at least k.
__device__ __forceinline__ uint32_t kth_set_bit(uint32_t m, uint32_t k) {
  uint32_t lo = 0, hi = 31;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    const uint32_t le = mid == 31u ? 0xFFFFFFFFu : (2u << mid) - 1u;
    if ((uint32_t)__popc(m & le) >= k) hi = mid;
    else lo = mid + 1u;
  }
  return lo;
}

// The prefix decode's walk over the stream, carried from one rANS run to the next: the
// operation / entry automaton's state, the current level, its nodes still to come and its nodes
// emitted with stop bit 0, and whether the target level is complete (then the end is the next
// operation).
struct PrefixWalk {
  uint32_t st, level, rem, open;
  bool wait_op, done;
  uint32_t end;
};

// One run of the prefix decode: the stream's symbols s0 .. s0 + len - 1 (s0 a multiple of 32)
// from the run's states and its nw words, into the workspace slot `out` (nibbles by stream
// position). A coarser level of detail needs the levels 0 .. T only, and they come first: level
// l + 1 has 8 nodes per node of level l emitted with stop bit 0, and an operation may be followed
// by delta entries. Per step the warp finds which of its 32 symbols are operations (the 2-state
// automaton, both entering states packed in 2 bits and composed over the lanes by a shuffle
// scan) and counts the nodes of the current level. W.done once the first operation after level
// T's last node is reached (W.end: its position). false for a read past the run's words, or, when
// the run was decoded to its end, words left over or a state that does not end at 2^16.
__device__ bool prefix_run(const uint32_t* tab, const uint16_t* words, uint32_t nw, uint32_t s0, uint32_t len,
                           uint32_t x, uint32_t ns, uint8_t* out, uint32_t lane, uint32_t T, bool no_stop,
                           bool short_delta, PrefixWalk& W) {
  const uint32_t lt = lanemask_lt();
  uint8_t* o = out + (lane >> 1);
  const bool even = !(lane & 1u);
  auto ld = [&](uint32_t i) -> uint32_t { return i < nw ? (uint32_t)__ldg(words + i) : 0u; };
  uint32_t wb = 0, w0 = ld(lane), w1 = ld(32u + lane), w2 = ld(64u + lane), w3 = ld(96u + lane);
  uint32_t ptr = 0;
  for (uint32_t base = 0; base < len; base += 32u) {
    const uint32_t i = base + lane;
    const bool active = i < len;
    uint32_t s = 0;
    if (active) {
      const uint32_t e = tab[x & (kRansM - 1u)];
      s = e >> 25;
      x = (e & 0x1FFFu) * (x >> 12) + ((e >> 13) & 0xFFFu);
    }
    const bool need = active && x < (1u << 16);
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, need);
    const uint32_t r = ptr - wb + __popc(m & lt);
    const uint32_t v0 = __shfl_sync(0xFFFFFFFFu, w0, r & 31u), v1 = __shfl_sync(0xFFFFFFFFu, w1, r & 31u);
    if (need) x = (x << 16) | (r < 32u ? v0 : v1);
    ptr += __popc(m);
    if (ptr - wb >= 32u) {
      wb += 32u;
      w0 = w1;
      w1 = w2;
      w2 = w3;
      w3 = ld(wb + 96u + lane);
    }
    const uint32_t hi = __shfl_xor_sync(0xFFFFFFFFu, s, 1);
    if (active && even) o[(s0 + base) >> 1] = (uint8_t)(s | (i + 1 < len ? hi << 4 : 0u));
    // the state after this symbol entered in state 0 (bit 0) / 1 (bit 1), inactive lanes the
    // identity; composed over the lanes (p, then g: state s -> bit p(s) of g)
    uint32_t g = active ? ((s & 7u) == OP_DELTA ? 1u : 0u) | ((short_delta ? 0u : (s >> 3) & 1u) << 1) : 2u;
#pragma unroll
    for (uint32_t d = 1; d < 32u; d <<= 1) {
      const uint32_t p = __shfl_up_sync(0xFFFFFFFFu, g, d);
      if (lane >= d) g = ((g >> (p & 1u)) & 1u) | (((g >> (p >> 1)) & 1u) << 1);
    }
    uint32_t e = __shfl_up_sync(0xFFFFFFFFu, g, 1);
    if (lane == 0) e = 2u;
    const bool is_op = active && ((e >> W.st) & 1u) == 0u;
    uint32_t opm = __ballot_sync(0xFFFFFFFFu, is_op);
    const uint32_t openm = __ballot_sync(0xFFFFFFFFu, is_op && (no_stop || !(s & 8u)));
    W.st = (__shfl_sync(0xFFFFFFFFu, g, 31) >> W.st) & 1u;
    if (W.wait_op) {
      if (opm) {
        W.end = s0 + base + (__ffs(opm) - 1u);
        W.done = true;
      }
    } else if ((uint32_t)__popc(opm) < W.rem) {  // every operation of the step is in the current level
      W.open += (uint32_t)__popc(openm);
      W.rem -= (uint32_t)__popc(opm);
    } else {
      while (opm) {
        const uint32_t c = (uint32_t)__popc(opm);
        const uint32_t k = W.rem < c ? W.rem : c;
        const uint32_t p = kth_set_bit(opm, k);
        const uint32_t sel = opm & (p == 31u ? 0xFFFFFFFFu : (2u << p) - 1u);
        W.open += (uint32_t)__popc(sel & openm);
        W.rem -= k;
        opm &= ~sel;
        if (W.rem == 0u) {
          if (W.level == T || W.open == 0u) {  // the target level (or the last emitted one) is complete
            W.wait_op = true;
            if (opm) {
              W.end = s0 + base + (__ffs(opm) - 1u);
              W.done = true;
            }
            break;
          }
          ++W.level;
          W.rem = 8u * W.open;
          W.open = 0u;
        }
      }
    }
    if (W.done) return true;  // stopped inside the run: its end is not checked
  }
  bool bad = ptr != nw;
  bad |= lane < ns && x != (1u << 16);
  return !__any_sync(0xFFFFFFFFu, bad);
}

// Run `run` of the item scheduled k-th, by one warp (tab: the slot table in shared memory); the
// runs of a record are independent (vc_internal.h). With wpi = 1 at a coarse level of detail the
// warp walks the runs in order and stops after the target level; the symbols decoded go to the
// workspace slot's last word for the reconstruction kernel.
__device__ __forceinline__ void rans_symbols_item(const Params& P, const uint32_t* tab, uint8_t* ws, uint32_t k,
                                                  uint32_t run, uint32_t lane) {
  const SmemLayout& SL = P.v.sm;
  const uint32_t item = scheduled_item(P, k);
  const uint32_t brick = P.ids[item];
  if (brick >= P.v.n_bricks) return;  // reported by the reconstruction kernel
  const uint32_t* rec = P.v.records + P.v.starts[brick];
  const uint32_t np = rec[0], S = rec[1], cb = rec[2];
  const uint32_t K = runs_k(P.v.flags), nr = run_n(S, K), q = run_q(S, K), hw = head_words(S, K);
  if (run >= nr) return;
  const uint32_t nw = cb >> 1;
  const uint16_t* words =
      reinterpret_cast<const uint16_t*>(reinterpret_cast<const unsigned char*>(rec) + 16u + 4u * hw + 4u * np);
  uint8_t* out = ws + (size_t)(item - P.ws_item0) * SL.ws_stride;
  // run r: symbols r q .., states at word 4 + 32 r, words from its start to the next run's
  auto run_words = [&](uint32_t r, uint32_t& w0, uint32_t& w1) -> bool {
    w0 = r ? rec[4u + hw - (nr - 1u) + (r - 1u)] : 0u;
    w1 = r + 1u < nr ? rec[4u + hw - (nr - 1u) + r] : nw;
    return w0 <= w1 && w1 <= nw;
  };
  bool ok = true;
  if (P.lod < P.v.prefix_lod) {
    uint32_t w0, w1;
    const uint32_t len = min(q, S - run * q), ns = min(len, 32u);
    const uint32_t x0 = lane < ns ? rec[4u + 32u * run + lane] : (1u << 16);
    ok = run_words(run, w0, w1) && !__any_sync(0xFFFFFFFFu, lane < ns && x0 < (1u << 16));
    if (ok) ok = rans_steps(tab, words + w0, w1 - w0, len, x0, ns, out + ((run * q) >> 1), lane);
  } else {
    const uint32_t T = P.v.L > P.lod ? P.v.L - P.lod : 0u;
    PrefixWalk W{0u, 0u, 1u, 0u, false, false, S};
    for (uint32_t r = 0; r < nr && ok && !W.done; ++r) {
      uint32_t w0, w1;
      const uint32_t len = min(q, S - r * q), ns = min(len, 32u);
      const uint32_t x0 = lane < ns ? rec[4u + 32u * r + lane] : (1u << 16);
      ok = run_words(r, w0, w1) && !__any_sync(0xFFFFFFFFu, lane < ns && x0 < (1u << 16));
      if (ok)
        ok = prefix_run(tab, words + w0, w1 - w0, r * q, len, x0, ns, out, lane, T, (P.v.flags & kFlagNoStop) != 0,
                        (P.v.flags & kFlagShortDelta) != 0, W);
    }
    if (lane == 0) reinterpret_cast<uint32_t*>(ws + (size_t)(item - P.ws_item0 + 1u) * SL.ws_stride)[-1] = W.end;
  }
  if (!ok && lane == 0) report(P.status, VC_ERR_CORRUPT, item);
}

// wpi warps per item (the record's runs side by side; 1 at a coarse level of detail).
__global__ void __launch_bounds__(32 * kRansWarps) rans_symbols_kernel(const __grid_constant__ Params P,
                                                                      uint8_t* ws, uint32_t wpi) {
  extern __shared__ __align__(128) unsigned char sm[];
  uint32_t* tab = reinterpret_cast<uint32_t*>(sm);
  for (uint32_t i = threadIdx.x; i < kRansM; i += blockDim.x) tab[i] = P.v.rans_tab[i];
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t g = blockIdx.x * (blockDim.x >> 5) + warp;  // the block's warps take consecutive (item, run)
  const uint32_t k = P.item_base + g / wpi;
  if (k >= P.n) return;
  rans_symbols_item(P, tab, ws, k, g % wpi, lane);
}

// The same with the item count in device memory (launch_items): persistent warps stride over the
// items.
__global__ void __launch_bounds__(32 * kRansWarps) rans_symbols_dev_kernel(const __grid_constant__ Params P,
                                                                          uint8_t* ws, uint32_t wpi) {
  extern __shared__ __align__(128) unsigned char sm[];
  uint32_t* tab = reinterpret_cast<uint32_t*>(sm);
  const uint32_t n = launch_items(P) * wpi;
  if (blockIdx.x * kRansWarps >= n) return;
  for (uint32_t i = threadIdx.x; i < kRansM; i += 32u * kRansWarps) tab[i] = P.v.rans_tab[i];
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  for (uint32_t g = blockIdx.x * kRansWarps + warp; g < n; g += gridDim.x * kRansWarps)
    rans_symbols_item(P, tab, ws, g / wpi, g % wpi, lane);
}

// ------------------------------------------------------------------------------------------
// Size-aware order: the request's items sorted longest record first (a counting sort into 256
// buckets of record size, one block), so that the longest bricks do not start last and stretch
// the tail of the launch. order[k] = the item scheduled k-th; ties keep no particular order.
constexpr uint32_t kOrderBuckets = 256u;
constexpr uint32_t kOrderThreads = 1024u;
constexpr uint32_t kOrderMin = 1024u;  // smaller requests keep their own order

__global__ void __launch_bounds__(kOrderThreads) order_kernel(const __grid_constant__ Params P, uint32_t max_words,
                                                               uint32_t* order) {
  constexpr uint32_t KEEP = 8;  // buckets of a thread's first items are kept in registers
  __shared__ uint32_t cnt[kOrderBuckets];
  const uint32_t tid = threadIdx.x, lane = tid & 31u;
  for (uint32_t i = tid; i < kOrderBuckets; i += kOrderThreads) cnt[i] = 0u;
  __syncthreads();
  auto bucket = [&](uint32_t item) -> uint32_t {  // 0 = longest
    const uint32_t brick = P.ids[item];
    if (brick >= P.v.n_bricks) return kOrderBuckets - 1u;  // reported by the decode kernels
    const uint32_t w = min(P.v.starts[brick + 1] - P.v.starts[brick], max_words);
    return (uint32_t)(((uint64_t)(max_words - w) * (kOrderBuckets - 1u)) / max_words);
  };
  // one shared-memory atomic per distinct bucket in a warp (lanes with equal buckets grouped)
  auto warp_add = [&](bool valid, uint32_t bk) -> uint32_t {
    const uint32_t key = valid ? bk : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, key);
    const uint32_t leader = __ffs(peers) - 1u;
    uint32_t base = 0;
    if (valid && lane == leader) base = atomicAdd(&cnt[bk], __popc(peers));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    return base + __popc(peers & lanemask_lt());
  };
  uint32_t kept[KEEP];
  const uint32_t rounds = (P.n + kOrderThreads - 1u) / kOrderThreads;
#pragma unroll
  for (uint32_t r = 0; r < KEEP; ++r) {
    const uint32_t i = r * kOrderThreads + tid;
    kept[r] = r < rounds && i < P.n ? bucket(i) : 0u;
    if (r < rounds) warp_add(i < P.n, kept[r]);
  }
  for (uint32_t r = KEEP; r < rounds; ++r) {
    const uint32_t i = r * kOrderThreads + tid;
    warp_add(i < P.n, i < P.n ? bucket(i) : 0u);
  }
  __syncthreads();
  if (tid < 32u) {  // exclusive scan of the counts, 8 buckets per lane
    constexpr uint32_t per = kOrderBuckets / 32u;
    uint32_t v[per], sum = 0;
#pragma unroll
    for (uint32_t j = 0; j < per; ++j) { v[j] = cnt[tid * per + j]; sum += v[j]; }
    uint32_t inc = sum;
#pragma unroll
    for (uint32_t d = 1; d < 32u; d <<= 1) {
      const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, d);
      if (tid >= d) inc += t;
    }
    uint32_t base = inc - sum;
#pragma unroll
    for (uint32_t j = 0; j < per; ++j) { cnt[tid * per + j] = base; base += v[j]; }
  }
  __syncthreads();
#pragma unroll
  for (uint32_t r = 0; r < KEEP; ++r) {
    const uint32_t i = r * kOrderThreads + tid;
    if (r < rounds) {
      const uint32_t pos = warp_add(i < P.n, kept[r]);
      if (i < P.n) order[pos] = i;
    }
  }
  for (uint32_t r = KEEP; r < rounds; ++r) {
    const uint32_t i = r * kOrderThreads + tid;
    const uint32_t pos = warp_add(i < P.n, i < P.n ? bucket(i) : 0u);
    if (i < P.n) order[pos] = i;
  }
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

void palette_packing(uint32_t max_pal, uint32_t* bits, uint32_t* per_word) {
  uint32_t I = 1;
  while ((1u << I) < max_pal) ++I;  // ceil(log2 max_pal), at least 1
  *bits = I;
  *per_word = 32u / I;
}

bool schedule_supported(uint32_t L, uint32_t threads) {
  if (L < 1 || L > 6) return false;
  if (threads == 256) return true;
  return (threads == 512 || threads == 1024) && L >= 4;
}

vc_status compute_layout(const Volume& v, int device, uint32_t threads, uint32_t nstage, SmemLayout* out,
                         bool paletted) {
  const uint32_t L = v.L;
  if (!schedule_supported(L, threads) || nstage < 1 || nstage > 2) return VC_ERR_UNSUPPORTED;
  int optin = 0, per_sm = 0, reserved = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device) != cudaSuccess)
    return VC_ERR_CUDA;
  // b = 64 bricks: with label output the finest level needs only the open cells' children, so
  // every region may fit one block's shared memory (attempt -1; no scratch slice); otherwise
  // (and for packed palette indices, whose finest level is a 64^3 index grid) the large regions
  // (node operations, delta values, cursor masks, the finest grid) live in a global scratch slice
  // per block, the rest in shared memory when it fits (attempt 0), else everything in the slice
  // (attempt 1); see SmemLayout::gscratch. In attempt 0 the shared memory left over takes whole
  // large regions back, the most read first: the children (or finest grid), the node operations,
  // the cursor masks, the delta values (SmemLayout::big_sm); up to the block's share of the
  // multiprocessor when 1024 / threads blocks are resident (as many as 64 registers a thread
  // allow), so that the fill costs no occupancy.
  const bool global = L >= 6;
  SmemLayout s{};
  uint32_t o = 0, og = 0;  // shared / global scratch bytes placed
  uint32_t nodes_bytes = 0, dlist_bytes = 0, mask_bytes = 0;
  auto build = [&](int attempt, uint32_t big) {
    s = SmemLayout{};
    s.big_sm = big;
    o = 0;
    og = 0;
    const bool all_shared = attempt < 0, all_global = attempt == 1;
    // offset of a region of `bytes`; region: 0 for the small ones, else its SmemLayout::big_sm bit
    auto put = [&](uint32_t region, uint32_t bytes) -> uint32_t {
      const bool in_global = global && !all_shared && (all_global || (region && !(big & region)));
      uint32_t& c = in_global ? og : o;
      const uint32_t at = c;
      c += bytes;
      return at;
    };
    s.gt_bytes = v.max_pal < kMaxIdx8 ? 1u : 2u;
    const uint32_t b = 1u << L;
    const uint32_t ncells = ((1u << (3 * L)) - 1u) / 7u;  // levels 0..L-1
    // misc: words 0..15 (flags, items, mbarriers), 16..47 warp totals, then 5 (NT / 32) + 5 words
    // of scan scratch
    s.misc_off = put(0u, align16(4u * (48u + 5u * (threads / 32u) + 5u)));
    // a single stage may alias the regions a brick fills only after its parse (see stage_alias)
    const bool pal_always_copied = s.gt_bytes == 1 || v.max_pal <= 1024u;
    const bool may_alias = nstage == 1 && pal_always_copied && !global;
    // node operations: written by the parse; bricks without delta operations use their staged
    // symbols directly, or a copy here when the stage is aliased
    s.nodes_words = (v.max_nodes + 7u) / 8u + 4u;
    nodes_bytes = (v.max_delta || may_alias) ? align16(4 * s.nodes_words) : 0u;
    s.nodes_off = put(kBigNodes, nodes_bytes);
    s.dlist_cap = v.max_delta;
    dlist_bytes = align16(4 * (v.max_delta ? v.max_delta : 1u));
    s.dlist_off = put(kBigDelta, dlist_bytes);
    // cursor masks (2 u32 masks + 2 prefixes per word of 32 nodes), level grids, stop bytes and
    // rank lists: one contiguous span unless b = 64
    s.nwords = (v.max_nodes + 31u) / 32u + 2u;
    mask_bytes = align16((global ? 16 : 12) * s.nwords);
    s.mask_off = put(kBigMasks, mask_bytes);
    s.g_off = put(0u, align16(s.gt_bytes * (ncells + 7u)));  // level 1 starts at cell 8 (alignment)
    // per level l >= 1 below L, one byte per level-(l-1) cell: its children's stop-0 bits
    uint32_t ns_bytes = 0;
    for (uint32_t l = 1; l < L; ++l) ns_bytes += ((1u << (3 * (l - 1))) + 3u) & ~3u;
    s.ns_off = put(0u, align16(ns_bytes ? ns_bytes : 1u));
    // the stop-0 cells of each level by rank, two buffers (even / odd levels); a level's stop-0
    // cells have 8 emitted children each, so there are at most max_nodes / 8 of them
    uint32_t cap[2] = {1u, 1u};
    for (uint32_t l = 0; l + 1 <= L; ++l)
      cap[l & 1u] = std::max(cap[l & 1u], std::min(1u << (3 * l), v.max_nodes / 8u + 1u));
    s.list0_cap = (cap[0] + 7u) & ~7u;
    s.list1_cap = cap[1];
    s.list_off = put(0u, align16(2u * (s.list0_cap + cap[1])));
    // the finest index grid holds one z half at a time for b = 32 (plus the last plane of the first)
    const uint32_t nh = L == 5 ? 2u : 1u;
    // label output keeps 8 children per open level-(L-1) cell instead (b >= 4); b <= 32 then
    // needs neither the index grid nor the kept plane
    const uint32_t cap_open = (L - 1u) & 1u ? s.list1_cap : s.list0_cap;  // open level-(L-1) cells
    const uint32_t cb_bytes = L >= 2 ? s.gt_bytes * 8u * cap_open : 0u;
    const bool cells_only = all_shared || (!paletted && !global && L >= 2);
    s.fg_bytes = align16(cells_only ? cb_bytes : std::max(s.gt_bytes * b * b * b / nh, cb_bytes));
    s.fg_off = put(kBigFg, s.fg_bytes);
    s.plane_off = put(0u, nh == 2 && !cells_only ? align16(s.gt_bytes * b * b) : 0u);
    // private palette copy (frees the stage early); byte grids: a power of two >= max_pal, zero
    // padded (indices are masked with pal_cap - 1, so any byte stays in bounds)
    uint32_t p2 = 16u;
    while (p2 < v.max_pal) p2 <<= 1;
    s.pal_cap = s.gt_bytes == 1 ? p2 : (v.max_pal <= 1024u ? v.max_pal : 0u);
    s.pal_off = put(0u, align16(4u * s.pal_cap));
    s.rank_off = put(0u, align16(2u * std::max(1u, (1u << (3 * (L - 1))) / 32u)));
    // the queue of open cells with palette reads: the rank list of level L-2, no longer read then
    s.pq_off = s.list_off + (L & 1u ? 2u * s.list0_cap : 0u);
    s.pq_cap = L & 1u ? s.list1_cap : s.list0_cap;
    // per warp a queue of up to 32 x 7 neighbour marks; the node operations, delta values and
    // cursor masks are no longer read when the queues are filled: the queues go over that span
    // while it is one piece of memory (b = 64: in the scratch slice), else over the node
    // operations' region when it is large enough, else into a region of their own
    const uint32_t mq_bytes = 224u * (threads / 32u);
    const bool span_whole = !global || all_shared || all_global || (big & (kBigNodes | kBigDelta | kBigMasks)) == 0u;
    const uint32_t dead_span = s.mask_off + (global ? 16u : 12u) * s.nwords - s.nodes_off;
    if (span_whole && dead_span >= mq_bytes) {
      s.mq_off = s.nodes_off;
      if (big & kBigNodes) s.big_sm |= kBigQueues;
    } else if (nodes_bytes >= mq_bytes) {
      s.mq_off = s.nodes_off;
      if (big & kBigNodes) s.big_sm |= kBigQueues;
    } else {
      s.mq_off = put(kBigQueues, align16(mq_bytes));
    }
  };
  for (int attempt = global && !paletted ? -1 : 0; attempt < (global ? 2 : 1); ++attempt) {
    build(attempt, 0u);
    if (global && attempt == 0 && o + 64u <= (uint32_t)optin) {
      const uint32_t share = (uint32_t)per_sm / std::max(1u, 1024u / threads) - (uint32_t)reserved;
      uint32_t left = std::min<uint32_t>((uint32_t)optin, share) - 64u;
      left = left > o ? left - o : 0u;
      uint32_t big = 0;
      const uint32_t cand[4][2] = {{kBigFg, s.fg_bytes}, {kBigNodes, nodes_bytes}, {kBigMasks, mask_bytes},
                                   {kBigDelta, dlist_bytes}};
      for (const auto& c : cand)
        if (c[1] && c[1] <= left) {
          big |= c[0];
          left -= c[1];
        }
      if (big) build(attempt, big);
    }
    if (!global || o + 64u <= (uint32_t)optin) break;  // (+ the kernel's static shared words)
  }
  if (global && o + 64u > (uint32_t)optin) return VC_ERR_UNSUPPORTED;
  const uint32_t span_bytes = s.fg_off - s.mask_off;  // masks .. rank lists (b <= 32)
  if (global) {  // nothing staged: the record and symbols are read where they are
    s.stage_alias = 0;
    s.wst_off = s.fg_off;
    s.wst_bytes = s.fg_bytes;
    s.stage_bytes = 0;
    s.nstage = nstage;
    s.stage_off = o;
    s.total = o;  // shared bytes (0: everything in the slice)
    s.gscratch = (og + 255u) & ~255u;
    s.ws_stride = align16((v.max_sym + 1u) / 2u) + 16u;
    s.a_buf = 0;
    s.a_smem = 4u * kRansM;
    *out = s;
    return VC_OK;
  }
  const bool may_alias = nstage == 1 && (s.gt_bytes == 1 || v.max_pal <= 1024u);
  const uint32_t fixed = o;
  uint32_t stage = align16(v.max_stage) + 16u;  // slack for 8-nibble windows at the end
  s.wst_off = s.fg_off;
  s.wst_bytes = s.fg_bytes;
  s.nstage = nstage;
  if (may_alias && stage <= span_bytes) {
    // one stage over the masks .. rank lists span
    s.stage_alias = 1;
    s.stage_bytes = stage;
    s.stage_off = s.mask_off;
  } else {
    if (fixed + nstage * stage > (uint32_t)optin) stage = 0;
    s.stage_alias = 0;
    s.stage_bytes = stage;
    s.stage_off = o; o += nstage * stage;
  }
  s.total = o;
  if (s.total > (uint32_t)optin) return VC_ERR_UNSUPPORTED;
  // rANS symbol kernel: table + one coded-word buffer per warp
  s.ws_stride = align16((v.max_sym + 1u) / 2u) + 16u;
  s.a_buf = 0;
  s.a_smem = 4u * kRansM;  // the slot table only: many blocks per SM hide the step latency
  *out = s;
  return VC_OK;
}

namespace {

bool set_smem(void* k, uint32_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

// Bricks (warps) per block of the rANS symbol kernel for `count` bricks on `sms` multiprocessors.
// Each brick is one serial chain, so a launch lasts as long as its slowest chain, and chains that
// share a scheduler slow each other down: when the launch fits about one wave, the block size
// (16, 8 or 4 warps) that puts the fewest warps on the busiest multiprocessor wins (ties: the
// larger block, fewer copies of the slot table); 512 bricks of 64^3 then run on 128
// multiprocessors, 4 warps each, instead of 32 with 16.
uint32_t symbol_warps(uint32_t count, uint32_t sms) {
  if (sms == 0 || count > kRansWarps * sms * 4u) return kRansWarps;
  uint32_t best = kRansWarps, best_load = ~0u;
  for (uint32_t w = kRansWarps; w >= 4u; w >>= 1) {
    const uint32_t blocks = (count + w - 1) / w;
    const uint32_t load = (blocks + sms - 1) / sms * w;
    if (load < best_load) {
      best_load = load;
      best = w;
    }
  }
  return best;
}

// Warps per item of the rANS symbol kernels: one per run of the records (1 at a coarse level of
// detail, where one warp walks the runs up to the level).
uint32_t symbol_wpi(const Params& P) { return P.lod < P.v.prefix_lod ? runs_k(P.v.flags) : 1u; }

bool launch_symbols(const Params& P, uint8_t* ws, uint32_t base, uint32_t count, uint32_t smem, uint32_t sms,
                    cudaStream_t s) {
  Params PA = P;
  PA.item_base = base;
  PA.n = base + count;
  uint32_t wpi = symbol_wpi(P);
  void* args[] = {&PA, &ws, &wpi};
  const uint32_t w = symbol_warps(count * wpi, sms);
  const uint32_t blocks = (count * wpi + w - 1) / w;
  return cudaLaunchKernel(reinterpret_cast<void*>(&rans_symbols_kernel), dim3(blocks), dim3(32 * w), args, smem, s) ==
         cudaSuccess;
}

// The pipelined schedule: chunks of request items flow through the rANS symbol kernel (stream 0)
// and the reconstruction kernel (stream 1, one block per brick), so that the symbols of chunk k+1
// decode while chunk k is reconstructed; a ring of symbol workspaces is reused once the chunk that
// last used it is done. Plain-coded volumes have no symbol stage: one reconstruction launch.
vc_status launch_pipelined(Volume& v, Params P, uint32_t n, cudaStream_t stream) {
  const bool rans = v.coder == 1;
  const uint32_t nt = v.sched.threads;
  const SmemLayout& SL = v.dv.sm;
  void* kf = pick_kernel(v.L, nt, SL.gt_bytes == 2, rans, false);
  if (!kf) return VC_ERR_UNSUPPORTED;
  if (!set_smem(kf, SL.total)) return VC_ERR_CUDA;
  if (!rans) {
    void* args[] = {&P};
    if (cudaLaunchKernel(kf, dim3(n), dim3(nt), args, SL.total, stream) != cudaSuccess) return VC_ERR_CUDA;
    ++v.launches;
    return VC_OK;
  }
  if (!set_smem(reinterpret_cast<void*>(&rans_symbols_kernel), SL.a_smem)) return VC_ERR_CUDA;
  const uint32_t chunk = std::max<uint32_t>(1u, v.sched.chunk ? v.sched.chunk : 512u);
  const uint32_t nchunks = (n + chunk - 1) / chunk;
  const uint32_t ring = std::min<uint32_t>(kRing, nchunks);
  uint8_t* ws = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&ws), (size_t)ring * chunk * SL.ws_stride, stream) != cudaSuccess) {
    cudaGetLastError();
    return VC_ERR_OOM;
  }
  const cudaStream_t sA = v.aux[0], sF = v.aux[1];
  vc_status rc = VC_OK;
  auto ok = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == VC_OK) rc = VC_ERR_CUDA;
    return e == cudaSuccess;
  };
  ok(cudaEventRecord(v.ev_fork, stream));
  ok(cudaStreamWaitEvent(sA, v.ev_fork, 0));
  ok(cudaStreamWaitEvent(sF, v.ev_fork, 0));
  for (uint32_t k = 0; k < nchunks && rc == VC_OK; ++k) {
    const uint32_t base = k * chunk, cnt = std::min(chunk, n - base), slot = k % ring;
    Params Q = P;
    Q.item_base = base;
    Q.n = base + cnt;
    Q.ws_item0 = base;
    Q.ws = ws + (size_t)slot * chunk * SL.ws_stride;
    if (k >= ring) ok(cudaStreamWaitEvent(sA, v.ev_f[slot], 0));  // slot read by chunk k - ring
    ok(launch_symbols(Q, const_cast<uint8_t*>(Q.ws), base, cnt, SL.a_smem, v.sms, sA) ? cudaSuccess
                                                                                         : cudaErrorLaunchFailure);
    ok(cudaEventRecord(v.ev_a[slot], sA));
    ok(cudaStreamWaitEvent(sF, v.ev_a[slot], 0));
    void* argsF[] = {&Q};
    ok(cudaLaunchKernel(kf, dim3(cnt), dim3(nt), argsF, SL.total, sF));
    ok(cudaEventRecord(v.ev_f[slot], sF));
    v.launches += 2;
  }
  // join: the caller's stream waits for both
  ok(cudaEventRecord(v.ev_join[0], sA));
  ok(cudaEventRecord(v.ev_join[1], sF));
  for (int i = 0; i < 2; ++i) ok(cudaStreamWaitEvent(stream, v.ev_join[i], 0));
  cudaFreeAsync(ws, stream);
  return rc;
}

// b = 64: persistent blocks of the scratch kernel, before the occupancy limit (blocks_per_sm, else
// 2 per SM: each holds a scratch slice of about a megabyte)
uint32_t scratch_grid(const Volume& v, uint32_t n) {
  const uint32_t per_sm = v.sched.blocks_per_sm ? v.sched.blocks_per_sm : 2u;
  return std::min(n, std::max(1u, v.sms) * per_sm);
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing arrives at (no copy
// is issued, so nothing is in flight when it gives up) and reports VC_ERR_TIMEOUT, or VC_OK if the
// wait were to complete; the elapsed wall-clock time goes to status[2..3] (ns, low / high).
__global__ void wait_selftest_kernel(int32_t* status, uint64_t budget_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  const uint64_t t0 = globaltimer_ns();
  const bool ok = mbar_wait_bounded(&bar, 0, budget_ns);
  const uint64_t dt = globaltimer_ns() - t0;
  if (!ok) atomicCAS(reinterpret_cast<int*>(status), 0, VC_ERR_TIMEOUT);
  status[2] = (int32_t)(uint32_t)dt;
  status[3] = (int32_t)(uint32_t)(dt >> 32);
}

// The coarsest level of detail straight from the encoding: the first palette entry of each brick
// (the root is always a palette advance).
__global__ void __launch_bounds__(256) coarsest_kernel(const __grid_constant__ Params P, uint32_t* out) {
  const uint32_t i = blockIdx.x * 256u + threadIdx.x;
  if (i >= P.n) return;
  const uint32_t brick = P.ids[i];
  if (brick >= P.v.n_bricks) {
    out[i] = 0u;
    report(P.status, VC_ERR_ARG, i);
    return;
  }
  const uint32_t* rec = P.v.records + P.v.starts[brick];
  const uint32_t np = rec[0], S = rec[1];
  const uint32_t ns = P.v.coder == 1 ? head_words(S, runs_k(P.v.flags)) : 0u;
  if (np == 0u) {
    out[i] = 0u;
    report(P.status, VC_ERR_CORRUPT, i);
    return;
  }
  out[i] = rec[4u + ns];
}

}  // namespace

vc_status launch_coarsest(Volume& v, const uint32_t* ids, uint32_t n, uint32_t* out, int32_t* status,
                          cudaStream_t stream) {
  if (n == 0) return VC_OK;
  Params P{};
  P.v = v.dv;
  P.ids = ids;
  P.n = n;
  P.status = status;
  void* args[] = {&P, &out};
  if (cudaLaunchKernel(reinterpret_cast<void*>(&coarsest_kernel), dim3((n + 255u) / 256u), dim3(256), args, 0,
                       stream) != cudaSuccess)
    return VC_ERR_CUDA;
  ++v.launches;
  return VC_OK;
}

size_t decode_ws_bytes(const Volume& v, uint32_t n) {
  const SmemLayout& SL = v.dv.sm;
  const size_t sym = v.coder == 1 ? ((size_t)n * SL.ws_stride + 255u) & ~size_t(255) : 0u;
  const size_t slice = std::max(SL.gscratch, v.sm_pal.gscratch);  // labels or packed indices
  return sym + (slice ? (size_t)scratch_grid(v, n) * slice : 0u);
}

vc_status launch_decode(Volume& v, const uint32_t* ids, uint32_t n, const uint32_t* slots, uint32_t* cache,
                        uint32_t lod, uint32_t mode, int32_t* status, cudaStream_t stream, bool presorted) {
  return launch_decode_ws(v, ids, n, slots, cache, lod, mode, status, stream, nullptr, 0, presorted);
}

vc_status launch_decode_ws(Volume& v, const uint32_t* ids, uint32_t n, const uint32_t* slots, uint32_t* cache,
                           uint32_t lod, uint32_t mode, int32_t* status, cudaStream_t stream, uint8_t* ws_ext,
                           size_t ws_cap, bool presorted) {
  if (n == 0) return VC_OK;
  const bool rans = v.coder == 1;
  Params P;
  P.v = v.dv;
  if (v.split && lod == 0) {
    // the finest level is in host memory only: whole records over the host link, read with
    // plain loads (the bulk-copy prefetch of the batched kernel is not used on them)
    P.v.records = v.full_records;
    P.v.starts = v.full_starts;
    if ((mode & ~VC_MODE_PALETTED) == VC_MODE_BATCHED) mode = (mode & VC_MODE_PALETTED) | VC_MODE_GRID;
  }
  P.ids = ids;
  P.slots = slots;
  P.n = n;
  P.cache = cache;
  P.lod = lod;
  P.status = status;
  P.item_base = 0;
  P.ws = nullptr;
  P.ws_item0 = 0;
  P.order = nullptr;
  P.n_dev = nullptr;
  const uint32_t edge = (1u << v.L) >> lod;
  P.out_words = edge * edge * edge;
  P.pal_bits = P.pal_per = 0;
  if (mode & VC_MODE_PALETTED) {
    mode &= ~VC_MODE_PALETTED;
    if (mode == VC_MODE_PIPELINED) return VC_ERR_UNSUPPORTED;
    palette_packing(v.max_pal, &P.pal_bits, &P.pal_per);
    P.out_words = (edge * edge * edge + P.pal_per - 1u) / P.pal_per;
  }
  if (P.pal_bits) P.v.sm = v.sm_pal;  // b = 64: packed indices need the voxel index grid
  const SmemLayout& SL = P.v.sm;
  const bool scratch = v.L >= 6;     // b = 64: the persistent kernel with its regions in SL
  if (mode == VC_MODE_PIPELINED && ws_ext) return VC_ERR_ARG;  // it allocates its own workspaces
  // coarse levels of detail are written by the reconstruction kernel itself
  if (mode == VC_MODE_PIPELINED && lod == 0 && !scratch) return launch_pipelined(v, P, n, stream);
  // b = 64: one persistent kernel serves the grid, batched and pipelined schedules
  if (mode == VC_MODE_PIPELINED || (scratch && mode == VC_MODE_GRID)) mode = scratch ? VC_MODE_BATCHED : VC_MODE_GRID;
  const bool batched = mode == VC_MODE_BATCHED;
  const uint32_t nt = v.sched.threads;
  void* k = pick_kernel(v.L, nt, SL.gt_bytes == 2, rans, batched);
  if (!k) return VC_ERR_UNSUPPORTED;
  const uint32_t smem = SL.total;  // b = 64: the small regions in shared memory (0: all in the scratch slice)
  if (!set_smem(k, smem)) return VC_ERR_CUDA;
  if (rans && !set_smem(reinterpret_cast<void*>(&rans_symbols_kernel), SL.a_smem)) return VC_ERR_CUDA;
  // workspace: the rANS symbols of the n items, then (b = 64) one scratch slice per block
  const size_t sym_bytes = rans ? ((size_t)n * SL.ws_stride + 255u) & ~size_t(255) : 0u;
  uint32_t sgrid = 0;
  if (scratch) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)nt, smem) != cudaSuccess) return VC_ERR_CUDA;
    if (per_sm < 1) return VC_ERR_UNSUPPORTED;
    sgrid = std::min(scratch_grid(v, n), std::max(1u, v.sms) * (uint32_t)per_sm);
    if (ws_ext && SL.gscratch) {
      if (ws_cap < sym_bytes + SL.gscratch) return VC_ERR_ARG;
      sgrid = (uint32_t)std::min<size_t>(sgrid, (ws_cap - sym_bytes) / SL.gscratch);
    } else if (ws_ext && rans && sym_bytes > ws_cap) {
      return VC_ERR_ARG;
    }
  } else if (rans && ws_ext && (size_t)n * SL.ws_stride > ws_cap) {
    return VC_ERR_ARG;
  }
  // size-aware order (one-launch schedules of large requests): 4 n bytes after the rest
  const size_t base_need = sym_bytes + (size_t)sgrid * SL.gscratch;
  const bool want_order = !presorted && n >= kOrderMin && mode != VC_MODE_PLAIN &&
                          (!ws_ext || base_need + 4ull * n <= ws_cap);
  uint8_t* ws = nullptr;  // allocated here (freed at the end); none with a caller-provided workspace
  uint8_t* wsb = ws_ext;
  const size_t need = base_need + (want_order ? 4ull * n : 0ull);
  if (!ws_ext && need) {
    if (cudaMallocAsync(reinterpret_cast<void**>(&ws), need, stream) != cudaSuccess) {
      cudaGetLastError();
      return VC_ERR_OOM;
    }
    wsb = ws;
  }
  if (rans) P.ws = wsb;
  uint8_t* scr = scratch ? wsb + sym_bytes : nullptr;
  vc_status rc = VC_OK;
  if (want_order) {
    uint32_t* order = reinterpret_cast<uint32_t*>(wsb + base_need);
    void* args[] = {&P, &v.max_rec_words, &order};
    if (cudaLaunchKernel(reinterpret_cast<void*>(&order_kernel), dim3(1), dim3(kOrderThreads), args, 0, stream) !=
        cudaSuccess) {
      if (ws) cudaFreeAsync(ws, stream);
      return VC_ERR_CUDA;
    }
    ++v.launches;
    P.order = order;
  }
  // timing events of this call (grid and batched schedules), if profiling is on and a set is free
  cudaEvent_t* ev = nullptr;
  if (v.prof && mode != VC_MODE_PLAIN) {
    if (v.prof_used < kProfCalls) ev = v.prof_ev + 3 * v.prof_used++;
    else ++v.prof_dropped;
  }
  auto mark = [&](int i) { return !ev || cudaEventRecord(ev[i], stream) == cudaSuccess; };
  auto run_symbols = [&](uint32_t base, uint32_t count) -> bool {
    if (!rans) return true;
    if (!launch_symbols(P, const_cast<uint8_t*>(P.ws), base, count, v.dv.sm.a_smem, v.sms, stream)) return false;
    ++v.launches;
    return true;
  };
  auto run = [&](dim3 grid) -> bool {
    void* args[] = {&P};
    void* args_scratch[] = {&P, &scr};
    if (cudaLaunchKernel(k, grid, dim3(nt), scratch ? args_scratch : args, smem, stream) != cudaSuccess) return false;
    ++v.launches;
    return true;
  };
  auto reset_counter = [&]() {
    return cudaMemsetAsync(reinterpret_cast<uint32_t*>(status) + 2, 0, sizeof(uint32_t), stream) == cudaSuccess;
  };
  if (scratch && mode == VC_MODE_PLAIN) {
    for (uint32_t i = 0; i < n && rc == VC_OK; ++i) {
      P.item_base = i;
      P.n = i + 1u;
      if (!run_symbols(i, 1) || !reset_counter() || !run(dim3(1))) rc = VC_ERR_CUDA;
    }
    P.n = n;
  } else if (scratch) {
    if (!mark(0) || !run_symbols(0, n) || !reset_counter() || !mark(1) || !run(dim3(sgrid)) || !mark(2))
      rc = VC_ERR_CUDA;
  } else if (mode == VC_MODE_PLAIN) {
    for (uint32_t i = 0; i < n && rc == VC_OK; ++i) {
      P.item_base = i;
      if (!run_symbols(i, 1) || !run(dim3(1))) rc = VC_ERR_CUDA;
    }
  } else if (mode == VC_MODE_GRID) {
    if (!mark(0) || !run_symbols(0, n) || !mark(1) || !run(dim3(n)) || !mark(2)) rc = VC_ERR_CUDA;
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
      if (!mark(0) || !run_symbols(0, n) || !reset_counter() || !mark(1) || !run(dim3(grid)) || !mark(2))
        rc = VC_ERR_CUDA;
    }
  }
  if (ws) cudaFreeAsync(ws, stream);
  return rc;
}

// Persistent decode of the first min(cap, *n_dev) items (a count written on the device by an
// earlier kernel of the stream), without the host reading it: the rANS symbol kernel strides over
// the items, the batched (b = 64: scratch) kernel pulls them from its work counter. ws (caller's,
// 256-byte aligned) holds decode_ws_bytes(v, cap) bytes. No size-aware order, no paletting.
vc_status launch_decode_devcount(Volume& v, const uint32_t* ids, uint32_t cap, const uint32_t* n_dev,
                                 const uint32_t* slots, uint32_t* cache, uint32_t lod, int32_t* status,
                                 cudaStream_t stream, uint8_t* ws, size_t ws_cap) {
  if (cap == 0) return VC_OK;
  if (v.split && lod == 0) return VC_ERR_UNSUPPORTED;  // bulk copies cannot read the mapped host copy
  const bool rans = v.coder == 1;
  const SmemLayout& SL = v.dv.sm;
  const bool scratch = v.L >= 6;
  Params P{};
  P.v = v.dv;
  P.ids = ids;
  P.slots = slots;
  P.n = cap;
  P.n_dev = n_dev;
  P.cache = cache;
  P.lod = lod;
  P.status = status;
  const uint32_t edge = (1u << v.L) >> lod;
  P.out_words = edge * edge * edge;
  const uint32_t nt = v.sched.threads;
  void* k = pick_kernel(v.L, nt, SL.gt_bytes == 2, rans, true);
  if (!k) return VC_ERR_UNSUPPORTED;
  const uint32_t smem = SL.total;
  if (!set_smem(k, smem)) return VC_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)nt, smem) != cudaSuccess) return VC_ERR_CUDA;
  if (per_sm < 1) return VC_ERR_UNSUPPORTED;
  if (v.sched.blocks_per_sm) per_sm = std::min<int>(per_sm, (int)v.sched.blocks_per_sm);
  const uint32_t sms = std::max(1u, v.sms);
  const size_t sym_bytes = rans ? ((size_t)cap * SL.ws_stride + 255u) & ~size_t(255) : 0u;
  uint32_t grid = std::min<uint32_t>(cap, sms * (uint32_t)per_sm);
  if (scratch) grid = std::min(grid, scratch_grid(v, cap));
  if (scratch && SL.gscratch) {
    if (ws_cap < sym_bytes + SL.gscratch) return VC_ERR_ARG;
    grid = (uint32_t)std::min<size_t>(grid, (ws_cap - sym_bytes) / SL.gscratch);
  } else if (ws_cap < sym_bytes) {
    return VC_ERR_ARG;
  }
  if (rans) {
    P.ws = ws;
    if (!set_smem(reinterpret_cast<void*>(&rans_symbols_dev_kernel), SL.a_smem)) return VC_ERR_CUDA;
    uint8_t* wsp = ws;
    uint32_t wpi = symbol_wpi(P);
    void* args[] = {&P, &wsp, &wpi};
    const uint32_t sblocks = std::min<uint32_t>((cap * wpi + kRansWarps - 1) / kRansWarps, sms * 4u);
    if (cudaLaunchKernel(reinterpret_cast<void*>(&rans_symbols_dev_kernel), dim3(sblocks), dim3(32 * kRansWarps), args,
                         SL.a_smem, stream) != cudaSuccess)
      return VC_ERR_CUDA;
    ++v.launches;
  }
  if (cudaMemsetAsync(reinterpret_cast<uint32_t*>(status) + 2, 0, sizeof(uint32_t), stream) != cudaSuccess)
    return VC_ERR_CUDA;
  uint8_t* scr = scratch ? ws + sym_bytes : nullptr;
  void* args[] = {&P};
  void* args_scratch[] = {&P, &scr};
  if (cudaLaunchKernel(k, dim3(grid), dim3(nt), scratch ? args_scratch : args, smem, stream) != cudaSuccess)
    return VC_ERR_CUDA;
  ++v.launches;
  return VC_OK;
}

vc_status launch_wait_selftest(uint32_t budget_us, int32_t* status, cudaStream_t stream) {
  const uint64_t ns = (uint64_t)budget_us * 1000ull;
  void* args[] = {&status, const_cast<uint64_t*>(&ns)};
  return cudaLaunchKernel(reinterpret_cast<void*>(&wait_selftest_kernel), dim3(1), dim3(32), args, 0, stream) ==
                 cudaSuccess
             ? VC_OK
             : VC_ERR_CUDA;
}

}  // namespace vc
