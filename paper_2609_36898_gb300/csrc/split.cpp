// Detail split (Methods, "Encoding buffer optimizations": the finest level of detail, most of every
// brick's symbols, can be kept out of GPU memory and fetched only when a brick is needed at full
// resolution). The device holds, per brick, a record of the coarse levels 0 .. L-1 alone: a valid
// stream for every level of detail except the finest (its own palette prefix, symbol count and
// delta count). The whole encoding stays in pinned host memory mapped into the device's address
// space; finest-level decodes read those records over the host link (NVLink-C2C on GB300) with
// plain loads, with no copy in between.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "vc_internal.h"

using namespace vc;

namespace {

inline uint32_t le32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
inline void put32(uint8_t* p, uint32_t v) {
  p[0] = (uint8_t)v;
  p[1] = (uint8_t)(v >> 8);
  p[2] = (uint8_t)(v >> 16);
  p[3] = (uint8_t)(v >> 24);
}

struct Tables {
  uint32_t f[16], cum[17];
  std::vector<uint8_t> slot_sym;  // symbol of every rANS slot
};

Tables make_tables(const uint32_t freq[16]) {
  Tables t;
  t.cum[0] = 0;
  for (int s = 0; s < 16; ++s) {
    t.f[s] = freq[s];
    t.cum[s + 1] = t.cum[s] + freq[s];
  }
  t.slot_sym.assign(kRansM, 0);
  for (uint32_t s = 0; s < 16; ++s)
    for (uint32_t k = t.cum[s]; k < t.cum[s + 1] && k < kRansM; ++k) t.slot_sym[k] = (uint8_t)s;
  return t;
}

// The symbols of one record: plain nibbles (low nibble first), or the 32-way interleaved rANS
// stream decoded with the volume's table: in each step of 32 symbols every lane decodes one, then
// the lanes whose state fell below 2^16 read the next 16-bit word in lane order. false if the
// coded words do not decode exactly.
// One run of a rANS record: len symbols into sym from its states and its nw words.
bool run_symbols(const uint8_t* states, uint32_t len, const uint8_t* w, uint32_t nw, const Tables& t, uint8_t* sym) {
  const uint32_t ns = std::min<uint32_t>(len, kRansLanes);
  uint32_t x[32];
  for (uint32_t l = 0; l < 32; ++l) x[l] = l < ns ? le32(states + 4 * l) : (1u << 16);
  uint32_t ptr = 0;
  for (uint32_t base = 0; base < len; base += 32) {
    const uint32_t n = std::min<uint32_t>(32, len - base);
    for (uint32_t l = 0; l < n; ++l) {
      const uint32_t slot = x[l] & (kRansM - 1u), s = t.slot_sym[slot];
      x[l] = t.f[s] * (x[l] >> 12) + slot - t.cum[s];
      sym[base + l] = (uint8_t)s;
    }
    for (uint32_t l = 0; l < n; ++l) {
      if (x[l] < (1u << 16)) {
        if (ptr >= nw) return false;
        x[l] = (x[l] << 16) | (uint32_t)w[2 * ptr] | ((uint32_t)w[2 * ptr + 1] << 8);
        ++ptr;
      }
    }
  }
  return ptr == nw;
}

// The symbols of one record: plain nibbles (low nibble first), or the rANS runs (vc_internal.h)
// decoded with the volume's table: in each step of 32 symbols every lane decodes one, then the
// lanes whose state fell below 2^16 read the next 16-bit word in lane order. false if the coded
// words do not decode exactly.
bool record_symbols(const uint8_t* r, uint32_t coder, uint32_t flags, const Tables& t, std::vector<uint8_t>& sym) {
  const uint32_t n_pal = le32(r), S = le32(r + 4), cb = le32(r + 8);
  sym.resize(S);
  if (coder == 0) {
    const uint8_t* c = r + 16 + 4 * (size_t)n_pal;
    for (uint32_t i = 0; i < S; ++i) sym[i] = (uint8_t)((c[i >> 1] >> ((i & 1u) * 4u)) & 15u);
    return true;
  }
  const uint32_t K = runs_k(flags), n = run_n(S, K), q = run_q(S, K), hw = head_words(S, K);
  const uint8_t* w = r + 16 + 4 * (size_t)hw + 4 * (size_t)n_pal;
  const uint32_t nw = cb / 2;
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t w0 = k ? le32(r + 16 + 4 * ((size_t)hw - (n - 1u) + (k - 1u))) : 0u;
    const uint32_t w1 = k + 1u < n ? le32(r + 16 + 4 * ((size_t)hw - (n - 1u) + k)) : nw;
    if (w0 > w1 || w1 > nw) return false;
    if (!run_symbols(r + 16 + 4 * (size_t)(32u * k), std::min(q, S - k * q), w + 2 * (size_t)w0, w1 - w0, t,
                     sym.data() + (size_t)k * q))
      return false;
  }
  return true;
}

// Where the finest level starts. Level 0 is the root; level l + 1 holds the 8 children of every
// node of level l emitted with stop bit 0; a delta operation is followed by its entries (while
// bit 3 is set, at most 7; one with limited delta). out: the symbols before level L, and the
// palette advances and delta operations among them. false if the stream ends early.
bool coarse_prefix(const uint8_t* sym, uint32_t S, uint32_t L, bool short_delta, uint32_t* S_c, uint32_t* adv,
                   uint32_t* nd) {
  uint32_t i = 0, a = 0, d = 0;
  uint64_t count = 1;
  for (uint32_t l = 0; l < L; ++l) {
    uint64_t open = 0;
    for (uint64_t k = 0; k < count; ++k) {
      if (i >= S) return false;
      const uint32_t s = sym[i++], op = s & 7u;
      if (op == 4u) ++a;
      if (op == 6u) {
        ++d;
        if (short_delta) {
          if (i >= S) return false;
          ++i;
        } else {
          for (uint32_t e = 0;; ++e) {
            if (i >= S || e == 7u) return false;
            if (!(sym[i++] & 8u)) break;
          }
        }
      }
      if (!(s & 8u)) ++open;
    }
    count = 8u * open;
  }
  *S_c = i;
  *adv = a;
  *nd = d;
  return true;
}

template <class F>
void parallel_for(uint32_t n, F&& fn) {
  const uint32_t threads = std::max(1u, std::min<uint32_t>(std::thread::hardware_concurrency(), 64u));
  std::atomic<uint32_t> next{0};
  auto work = [&]() {
    for (;;) {
      const uint32_t i = next.fetch_add(1);
      if (i >= n) break;
      fn(i);
    }
  };
  std::vector<std::thread> pool;
  for (uint32_t k = 1; k < threads; ++k) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
}

struct CoarseRecord {
  std::vector<uint8_t> bytes;  // 16-byte padded
};

// The coarse-levels file: the same header, new Brick Starts, per brick the record of levels
// 0 .. L-1 in the volume's coder.
vc_status build_coarse(const uint8_t* p, const VolumeScan& sc, std::vector<uint8_t>& out) {
  const uint32_t n = sc.n_bricks;
  const uint8_t* st = p + kHeaderBytes;
  const uint8_t* rec = p + sc.rec_off;
  const Tables t = make_tables(sc.freq);
  const bool short_delta = (sc.flags & kFlagShortDelta) != 0;
  std::vector<CoarseRecord> recs(n);
  std::atomic<bool> bad{false};
  parallel_for(n, [&](uint32_t id) {
    const uint8_t* r = rec + 4 * (size_t)le32(st + 4 * (size_t)id);
    std::vector<uint8_t> sym;
    uint32_t S_c = 0, adv = 0, nd = 0;
    const uint32_t n_pal = le32(r);
    if (!record_symbols(r, sc.coder, sc.flags, t, sym) || !coarse_prefix(sym.data(), (uint32_t)sym.size(), sc.L, short_delta,
                                                               &S_c, &adv, &nd) ||
        adv > n_pal || S_c == 0) {
      bad = true;
      return;
    }
    const uint32_t K = runs_k(sc.flags);
    const uint32_t ns_full = sc.coder == 1 ? head_words(le32(r + 4), K) : 0u;
    const uint8_t* pal = r + 16 + 4 * (size_t)ns_full;
    // the coarse symbols re-coded with the volume's table, in runs as the volume's records are
    std::vector<uint16_t> words, w;
    std::vector<uint32_t> head, starts;
    uint32_t cb = 0;
    if (sc.coder == 1) {
      const uint32_t nr = run_n(S_c, K), q = run_q(S_c, K);
      uint32_t st[32], ns = 0;
      for (uint32_t k = 0; k < nr; ++k) {
        if (k) starts.push_back((uint32_t)words.size());
        rans_encode(sym.data() + (size_t)k * q, std::min(q, S_c - k * q), t.f, t.cum, w, st, &ns);
        head.insert(head.end(), st, st + ns);
        words.insert(words.end(), w.begin(), w.end());
      }
      head.insert(head.end(), starts.begin(), starts.end());
      cb = 2u * (uint32_t)words.size();
    } else {
      cb = (S_c + 1u) / 2u;
    }
    const uint32_t n_states = (uint32_t)head.size();
    const size_t bytes = 16 + 4 * (size_t)n_states + 4 * (size_t)adv + cb;
    std::vector<uint8_t>& o = recs[id].bytes;
    o.assign((bytes + 15) & ~(size_t)15, 0);
    put32(o.data(), adv);
    put32(o.data() + 4, S_c);
    put32(o.data() + 8, cb);
    put32(o.data() + 12, nd);
    uint8_t* q = o.data() + 16;
    for (uint32_t l = 0; l < n_states; ++l, q += 4) put32(q, head[l]);
    std::memcpy(q, pal, 4 * (size_t)adv);  // the palette prefix the coarse levels advance through
    q += 4 * (size_t)adv;
    if (sc.coder == 1) {
      for (size_t w = 0; w < words.size(); ++w) {
        q[2 * w] = (uint8_t)words[w];
        q[2 * w + 1] = (uint8_t)(words[w] >> 8);
      }
    } else {
      for (uint32_t i = 0; i < S_c; ++i) q[i >> 1] |= (uint8_t)(sym[i] << ((i & 1u) * 4u));
    }
  });
  if (bad) return VC_ERR_FORMAT;
  uint64_t words = 0;
  std::vector<uint32_t> starts((size_t)n + 1);
  for (uint32_t id = 0; id < n; ++id) {
    starts[id] = (uint32_t)words;
    words += recs[id].bytes.size() / 4;
  }
  starts[n] = (uint32_t)words;
  const size_t rec_off = (kHeaderBytes + 4 * ((size_t)n + 1) + 15) & ~(size_t)15;
  out.assign(rec_off + 4 * words, 0);
  std::memcpy(out.data(), p, kHeaderBytes);
  put32(out.data() + 112, (uint32_t)words);
  for (uint32_t id = 0; id <= n; ++id) put32(out.data() + kHeaderBytes + 4 * (size_t)id, starts[id]);
  for (uint32_t id = 0; id < n; ++id)
    std::memcpy(out.data() + rec_off + 4 * (size_t)starts[id], recs[id].bytes.data(), recs[id].bytes.size());
  return VC_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

vc_status vc_split_counts(const void* host_bytes, size_t nbytes, uint32_t brick_id, uint32_t out[4]) {
  if (!host_bytes || !out) return VC_ERR_ARG;
  const uint8_t* p = static_cast<const uint8_t*>(host_bytes);
  VolumeScan sc;
  vc_status rc = scan_volume(p, nbytes, &sc);
  if (rc != VC_OK) return rc;
  if (brick_id >= sc.n_bricks) return VC_ERR_ARG;
  const uint8_t* r = p + sc.rec_off + 4 * (size_t)le32(p + kHeaderBytes + 4 * (size_t)brick_id);
  std::vector<uint8_t> sym;
  uint32_t S_c = 0, adv = 0, nd = 0;
  if (!record_symbols(r, sc.coder, sc.flags, make_tables(sc.freq), sym) ||
      !coarse_prefix(sym.data(), (uint32_t)sym.size(), sc.L, (sc.flags & kFlagShortDelta) != 0, &S_c, &adv, &nd))
    return VC_ERR_CORRUPT;
  out[0] = (uint32_t)sym.size();
  out[1] = S_c;
  out[2] = adv;
  out[3] = nd;
  return VC_OK;
}

vc_status vc_load_compressed_split(const void* host_bytes, size_t nbytes, int device, void* cuda_stream,
                                   vc_volume** out) {
  if (!out) return VC_ERR_ARG;
  *out = nullptr;
  if (!host_bytes) return VC_ERR_ARG;
  const uint8_t* p = static_cast<const uint8_t*>(host_bytes);
  VolumeScan full;
  vc_status rc = scan_volume(p, nbytes, &full);
  if (rc != VC_OK) return rc;
  std::vector<uint8_t> coarse;
  rc = build_coarse(p, full, coarse);
  if (rc != VC_OK) return rc;
  vc_volume* h = nullptr;
  rc = vc_load_compressed(coarse.data(), coarse.size(), device, cuda_stream, &h);
  if (rc != VC_OK) return rc;
  std::vector<uint8_t>().swap(coarse);
  Volume* v = reinterpret_cast<Volume*>(h);
  DeviceGuard g(device);
  // the whole encoding in pinned host memory mapped into the device's address space (with the
  // same 64 zero bytes of slack as the device copy)
  const size_t file_bytes = full.rec_off + 4 * (size_t)full.records_words;
  void* hp = nullptr;
  if (cudaHostAlloc(&hp, file_bytes + 64, cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    vc_release(h);
    return VC_ERR_OOM;
  }
  std::memcpy(hp, p, file_bytes);
  std::memset(static_cast<uint8_t*>(hp) + file_bytes, 0, 64);
  void* dp = nullptr;
  if (cudaHostGetDevicePointer(&dp, hp, 0) != cudaSuccess || !dp) {
    cudaGetLastError();
    cudaFreeHost(hp);
    vc_release(h);
    return VC_ERR_CUDA;
  }
  v->h_full = static_cast<uint8_t*>(hp);
  v->host_bytes = file_bytes + 64;
  v->full_records = reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(dp) + full.rec_off);
  v->full_starts = reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(dp) + kHeaderBytes);
  // finest-level decodes read the whole records: the layout, workspaces and work ordering follow
  // their maxima and sizes; the request stage's palette flags follow the whole palettes
  v->max_pal = full.max_pal;
  v->max_sym = full.max_sym;
  v->max_delta = full.max_delta;
  v->max_rec_words = full.max_words;
  v->max_stage = full.max_stage;
  v->max_nodes = full.max_nodes;
  const uint8_t* st = p + kHeaderBytes;
  for (uint32_t i = 0; i < full.n_bricks; ++i)
    v->h_rec_words[i] = le32(st + 4 * ((size_t)i + 1)) - le32(st + 4 * (size_t)i);
  SmemLayout sl, sl_pal;
  rc = compute_layout(*v, device, v->sched.threads, v->sched.stage_depth, &sl);
  if (rc == VC_OK) rc = compute_layout(*v, device, v->sched.threads, v->sched.stage_depth, &sl_pal, true);
  if (rc != VC_OK) {
    vc_release(h);
    return rc;
  }
  v->dv.sm = sl;
  v->sm_pal = sl_pal;
  v->dv.prefix_lod = kPrefixMinLodSplit;  // level 1 reads the coarse records whole
  if (cudaMemcpy(v->d_flags, full.bflags.data(), full.n_bricks, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    vc_release(h);
    return VC_ERR_CUDA;
  }
  v->split = true;
  v->encoded_bytes = nbytes;
  *out = h;
  return VC_OK;
}

}  // extern "C"
