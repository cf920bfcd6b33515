// CPU encoder of the library (the paper compresses on the CPU, parallel over bricks; Methods,
// "Compressed segmentation volumes"). Bricks are encoded independently on worker threads; the
// operation of every node is the first applicable enabled one in the paper's order (parent,
// x / y / z neighbour with a different parent, last, delta, and a palette advance otherwise;
// Supplementary Fig. "CSGV ablation" caption), coarse nodes hold the mode of their 2^3 children
// (Results, "Ray marching"), constant subtrees set the stop bit (Results, "CSGV results").
// Levels are stored Morton-indexed so that the 8 children of node m are 8m .. 8m+7.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "vc.h"
#include "vc_internal.h"

namespace {

constexpr uint32_t kOpParent = 0, kOpNx = 1, kOpLast = 5, kOpDelta = 6, kOpAdv = 4;
constexpr uint32_t kShortDeltaMax = 16;  // flags bit 1: one 4-bit entry holds delta - 1, 2 <= delta <= 16
constexpr uint32_t kM = 4096;

inline void put32(uint8_t* p, uint32_t v) {
  p[0] = (uint8_t)v;
  p[1] = (uint8_t)(v >> 8);
  p[2] = (uint8_t)(v >> 16);
  p[3] = (uint8_t)(v >> 24);
}

inline uint32_t spread(uint32_t v) {
  uint32_t m = 0;
  for (int i = 0; i < 10; ++i) m |= ((v >> i) & 1u) << (3 * i);
  return m;
}

inline uint32_t step_back(uint32_t m, uint32_t axis) {
  const uint32_t am = 0x09249249u << axis;
  return (((m & am) - 1u) & am) | (m & ~am);
}

struct Brick {
  std::vector<uint8_t> sym;
  std::vector<uint32_t> pal;
  uint32_t n_delta = 0;
  std::vector<uint16_t> words;  // rANS: the runs' words one run after the other
  std::vector<uint32_t> head;   // rANS: the runs' final states, then the starts of runs 1..
  uint32_t coded_bytes = 0;
  uint32_t rec_words = 0;
};

// Palette positions by label: the two most recent positions of each label (a palette holds
// duplicates only when delta references are disabled or cannot reach them).
class PalIndex {
 public:
  void reset(size_t cap_hint) {
    size_t cap = 64;
    while (cap < 2 * cap_hint) cap <<= 1;
    keys_.assign(cap, 0);
    used_.assign(cap, 0);
    last_.assign(cap, -1);
    prev_.assign(cap, -1);
    mask_ = cap - 1;
  }
  void add(uint32_t label, int32_t pos) {
    size_t i = slot(label);
    if (!used_[i]) { used_[i] = 1; keys_[i] = label; }
    prev_[i] = last_[i];
    last_[i] = pos;
  }
  // most recent position <= limit, or -1
  int32_t recent_at_most(uint32_t label, int32_t limit) const {
    size_t i = slot(label);
    if (!used_[i]) return -1;
    if (last_[i] <= limit) return last_[i];
    return prev_[i] <= limit ? prev_[i] : -1;
  }

 private:
  size_t slot(uint32_t label) const {
    size_t i = (label * 2654435761u) & mask_;
    while (used_[i] && keys_[i] != label) i = (i + 1) & mask_;
    return i;
  }
  std::vector<uint32_t> keys_;
  std::vector<uint8_t> used_;
  std::vector<int32_t> last_, prev_;
  size_t mask_ = 0;
};

struct Scratch {
  std::vector<uint32_t> lab[7];
  std::vector<uint8_t> uni[7];
  std::vector<uint8_t> open[7];  // emitted with stop bit 0
  PalIndex idx;
};

uint32_t mode_of_8(const uint32_t* c) {
  uint32_t best = c[0];
  int best_n = 0;
  for (int i = 0; i < 8; ++i) {
    int n = 0;
    for (int j = 0; j < 8; ++j) n += c[j] == c[i];
    if (n > best_n || (n == best_n && c[i] < best)) {
      best_n = n;
      best = c[i];
    }
  }
  return best;
}

void encode_one(const uint32_t* V, const uint32_t dims[3], uint32_t L, uint32_t id, const uint32_t nb[3],
                uint32_t op_mask, bool use_stop, bool short_delta, const std::vector<uint32_t>& sp, Scratch& s,
                Brick& out) {
  const uint32_t b = 1u << L;
  const uint32_t bx = id % nb[0], by = (id / nb[0]) % nb[1], bz = id / (nb[0] * nb[1]);
  for (uint32_t l = 0; l <= L; ++l) {
    const size_t n = (size_t)1 << (3 * l);
    s.lab[l].resize(n);
    s.uni[l].resize(n);
    s.open[l].assign(n, 0);
  }
  // finest level, Morton indexed, clamp to edge beyond the volume
  for (uint32_t z = 0; z < b; ++z) {
    const size_t gz = std::min<size_t>((size_t)bz * b + z, dims[2] - 1);
    for (uint32_t y = 0; y < b; ++y) {
      const size_t gy = std::min<size_t>((size_t)by * b + y, dims[1] - 1);
      const uint32_t* row = V + (gz * dims[1] + gy) * dims[0];
      const uint32_t myz = (sp[y] << 1) | (sp[z] << 2);
      for (uint32_t x = 0; x < b; ++x) {
        const size_t gx = std::min<size_t>((size_t)bx * b + x, dims[0] - 1);
        s.lab[L][sp[x] | myz] = row[gx];
      }
    }
  }
  std::fill(s.uni[L].begin(), s.uni[L].end(), 1);
  for (uint32_t l = L; l > 0; --l) {
    const size_t n = (size_t)1 << (3 * (l - 1));
    const uint32_t* cl = s.lab[l].data();
    const uint8_t* cu = s.uni[l].data();
    for (size_t m = 0; m < n; ++m) {
      const uint32_t* c = cl + 8 * m;
      bool u = true;
      for (int i = 0; i < 8; ++i) u = u && cu[8 * m + i] && c[i] == c[0];
      s.lab[l - 1][m] = u ? c[0] : mode_of_8(c);
      s.uni[l - 1][m] = u;
    }
  }
  out.sym.clear();
  out.pal.clear();
  out.n_delta = 0;
  s.idx.reset(64);
  size_t pal_cap = 64;
  for (uint32_t l = 0; l <= L; ++l) {
    const size_t n = (size_t)1 << (3 * l);
    const uint32_t* lab = s.lab[l].data();
    for (size_t mm = 0; mm < n; ++mm) {
      const uint32_t m = (uint32_t)mm;
      if (l > 0 && !s.open[l - 1][m >> 3]) continue;
      const uint32_t t = lab[m];
      const uint32_t stop = (l < L && use_stop && s.uni[l][m]) ? 1u : 0u;
      s.open[l][m] = (l < L && !stop) ? 1 : 0;
      uint32_t op = 8;  // none yet
      uint32_t delta = 0;
      if ((op_mask & 1u) && l > 0 && s.lab[l - 1][m >> 3] == t) op = kOpParent;
      for (uint32_t a = 0; a < 3 && op == 8; ++a) {
        if (!((op_mask >> (kOpNx + a)) & 1u)) continue;
        const uint32_t am = 0x09249249u << a;
        if (((m >> a) & 1u) || (m & am) == 0) continue;  // odd or zero coordinate
        if (lab[step_back(m, a)] == t) op = kOpNx + a;
      }
      const int32_t k = (int32_t)out.pal.size();
      if (op == 8 && ((op_mask >> kOpLast) & 1u) && k >= 1 && out.pal[k - 1] == t) op = kOpLast;
      if (op == 8 && ((op_mask >> kOpDelta) & 1u)) {
        const int32_t pos = s.idx.recent_at_most(t, k - 2);
        if (pos >= 0 && (!short_delta || k - pos <= (int32_t)kShortDeltaMax)) {
          op = kOpDelta;
          delta = (uint32_t)(k - pos);
        }
      }
      if (op == 8) {
        op = kOpAdv;
        if (out.pal.size() + 1 > pal_cap / 2) {  // rebuild the index with room to spare
          pal_cap *= 4;
          s.idx.reset(pal_cap);
          for (size_t i = 0; i < out.pal.size(); ++i) s.idx.add(out.pal[i], (int32_t)i);
        }
        s.idx.add(t, k);
        out.pal.push_back(t);
      }
      out.sym.push_back((uint8_t)(op | (stop << 3)));
      if (op == kOpDelta) {
        if (short_delta) {
          out.sym.push_back((uint8_t)(delta - 1u));  // one entry holding delta - 1 (delta <= 16)
        } else {
          // octal digits of delta, most significant first; bit 3 = another entry follows
          int nd = 1;
          while ((delta >> (3 * nd)) != 0) ++nd;
          for (int i = nd - 1; i >= 0; --i) out.sym.push_back((uint8_t)(((delta >> (3 * i)) & 7u) | (i ? 8u : 0u)));
        }
        ++out.n_delta;
      }
    }
  }
}

void quantize(const uint64_t counts[16], uint32_t f[16]) {
  uint64_t total = 0;
  for (int i = 0; i < 16; ++i) total += counts[i];
  std::memset(f, 0, 16 * sizeof(uint32_t));
  if (!total) {
    f[kOpAdv] = kM;
    return;
  }
  int64_t sum = 0;
  int top = 0;
  for (int i = 0; i < 16; ++i) {
    if (counts[i] > counts[top]) top = i;
    if (!counts[i]) continue;
    f[i] = (uint32_t)std::max<uint64_t>(1, counts[i] * kM / total);
    sum += f[i];
  }
  if (sum < (int64_t)kM) f[top] += (uint32_t)((int64_t)kM - sum);
  for (; sum > (int64_t)kM; --sum) {
    int big = -1;
    for (int i = 0; i < 16; ++i)
      if (f[i] > 1 && (big < 0 || f[i] > f[big])) big = i;
    f[big] -= 1;
  }
}

// The record's rANS part: K runs (vc_internal.h), each coded on its own.
void rans_brick(Brick& br, const uint32_t f[16], const uint32_t cum[17], uint32_t K) {
  const uint32_t S = (uint32_t)br.sym.size(), q = vc::run_q(S, K), n = vc::run_n(S, K);
  br.words.clear();
  br.head.clear();
  std::vector<uint32_t> starts;
  std::vector<uint16_t> w;
  uint32_t st[32], ns = 0;
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t len = std::min(q, S - k * q);
    if (k) starts.push_back((uint32_t)br.words.size());
    vc::rans_encode(br.sym.data() + (size_t)k * q, len, f, cum, w, st, &ns);
    br.head.insert(br.head.end(), st, st + ns);
    br.words.insert(br.words.end(), w.begin(), w.end());
  }
  br.head.insert(br.head.end(), starts.begin(), starts.end());
  br.coded_bytes = 2 * (uint32_t)br.words.size();
}

template <class F>
void parallel_for(uint32_t n, uint32_t threads, F&& fn) {
  std::atomic<uint32_t> next{0};
  auto work = [&](uint32_t tid) {
    for (;;) {
      const uint32_t i = next.fetch_add(1);
      if (i >= n) break;
      fn(i, tid);
    }
  };
  std::vector<std::thread> pool;
  for (uint32_t t = 1; t < threads; ++t) pool.emplace_back(work, t);
  work(0);
  for (auto& th : pool) th.join();
}

}  // namespace

// 32-way interleaved rANS (symbol i on state i mod 32); words come out in the decoder's read order.
void vc::rans_encode(const uint8_t* sym, uint32_t S, const uint32_t f[16], const uint32_t cum[17],
                     std::vector<uint16_t>& words, uint32_t states[32], uint32_t* n_states) {
  uint32_t x[32];
  for (int l = 0; l < 32; ++l) x[l] = 1u << 16;
  words.clear();
  const uint32_t steps = (S + 31) / 32;
  for (uint32_t t = steps; t-- > 0;) {
    for (int l = 31; l >= 0; --l) {
      const uint32_t i = t * 32 + (uint32_t)l;
      if (i >= S) continue;
      const uint32_t sy = sym[i], fs = f[sy];
      if ((uint64_t)x[l] >= ((uint64_t)fs << 20)) {
        words.push_back((uint16_t)x[l]);
        x[l] >>= 16;
      }
      x[l] = ((x[l] / fs) << 12) + (x[l] % fs) + cum[sy];
    }
  }
  std::reverse(words.begin(), words.end());
  *n_states = std::min<uint32_t>(S, 32);
  for (uint32_t l = 0; l < *n_states; ++l) states[l] = x[l];
}

extern "C" {

vc_status vc_encode_volume_freq(const uint32_t* voxels, const uint32_t dims[3], uint32_t log2b, uint32_t op_mask,
                                uint32_t coder, uint32_t flags, uint32_t threads, const uint32_t* freq_in,
                                uint8_t** out_bytes, size_t* out_size) {
  if (!voxels || !dims || !out_bytes || !out_size) return VC_ERR_ARG;
  *out_bytes = nullptr;
  *out_size = 0;
  if (log2b < 1 || log2b > 6 || !(op_mask & (1u << kOpAdv)) || (op_mask & ~0x7Fu) || coder > 1 ||
      (flags & ~(3u | vc::kFlagRunsMask)) || (coder != 1 && (flags & vc::kFlagRunsMask)))
    return VC_ERR_ARG;
  if (!dims[0] || !dims[1] || !dims[2]) return VC_ERR_ARG;
  const uint32_t b = 1u << log2b;
  uint32_t nb[3];
  uint64_t n64 = 1;
  for (int a = 0; a < 3; ++a) {
    nb[a] = (dims[a] + b - 1) / b;
    n64 *= nb[a];
  }
  if (n64 >= 0xFFFFFFFFull) return VC_ERR_ARG;
  const uint32_t n = (uint32_t)n64;
  if (!threads) threads = std::max(1u, std::thread::hardware_concurrency());
  threads = std::min(threads, std::max(1u, n));
  std::vector<uint32_t> sp(b);
  for (uint32_t i = 0; i < b; ++i) sp[i] = spread(i);
  std::vector<Brick> bricks;
  std::vector<Scratch> scratch;
  try {
    bricks.resize(n);
    scratch.resize(threads);
  } catch (...) {
    return VC_ERR_OOM;
  }
  const bool use_stop = !(flags & 1u);
  const bool short_delta = (flags & 2u) != 0;  // one 4-bit entry per delta operation: delta <= 16
  parallel_for(n, threads, [&](uint32_t id, uint32_t tid) {
    encode_one(voxels, dims, log2b, id, nb, op_mask, use_stop, short_delta, sp, scratch[tid], bricks[id]);
  });
  scratch.clear();
  uint32_t freq[16] = {0}, cum[17] = {0};
  if (coder == 1) {
    uint64_t counts[16] = {0};
    for (const Brick& br : bricks)
      for (uint8_t v : br.sym) ++counts[v];
    if (freq_in) {  // the caller's table: it must sum to M and cover every symbol that occurs
      uint32_t sum = 0;
      for (int i = 0; i < 16; ++i) {
        sum += freq_in[i];
        if (counts[i] && !freq_in[i]) return VC_ERR_ARG;
      }
      if (sum != kM) return VC_ERR_ARG;
      std::memcpy(freq, freq_in, sizeof(freq));
    } else {
      quantize(counts, freq);
    }
    for (int i = 0; i < 16; ++i) cum[i + 1] = cum[i] + freq[i];
    parallel_for(n, threads, [&](uint32_t id, uint32_t) { rans_brick(bricks[id], freq, cum, vc::runs_k(flags)); });
  }
  uint64_t words = 0;
  uint32_t max_pal = 0, max_sym = 0;
  std::vector<uint32_t> starts((size_t)n + 1);
  for (uint32_t id = 0; id < n; ++id) {
    Brick& br = bricks[id];
    if (coder == 0) br.coded_bytes = ((uint32_t)br.sym.size() + 1) / 2;
    const uint64_t bytes = 16 + 4ull * (coder == 1 ? br.head.size() : 0) + 4ull * br.pal.size() + br.coded_bytes;
    br.rec_words = (uint32_t)(((bytes + 15) & ~15ull) / 4);
    starts[id] = (uint32_t)words;
    words += br.rec_words;
    if (words >= 0xFFFFFFFFull) return VC_ERR_ARG;  // 32-bit Brick Starts in words: 16 GiB
    max_pal = std::max<uint32_t>(max_pal, (uint32_t)br.pal.size());
    max_sym = std::max<uint32_t>(max_sym, (uint32_t)br.sym.size());
  }
  starts[n] = (uint32_t)words;
  const size_t rec_off = (128 + 4 * ((size_t)n + 1) + 15) & ~(size_t)15;
  const size_t size = rec_off + 4 * words;
  uint8_t* o = static_cast<uint8_t*>(std::calloc(size, 1));
  if (!o) return VC_ERR_OOM;
  const uint32_t hdr[12] = {0x315A4356u, 1u, dims[0], dims[1], dims[2], log2b, op_mask, coder, flags, n, max_pal,
                            max_sym};
  for (int i = 0; i < 12; ++i) put32(o + 4 * i, hdr[i]);
  for (int i = 0; i < 16; ++i) put32(o + 48 + 4 * i, freq[i]);
  put32(o + 112, (uint32_t)words);
  for (uint32_t id = 0; id <= n; ++id) put32(o + 128 + 4 * (size_t)id, starts[id]);
  parallel_for(n, threads, [&](uint32_t id, uint32_t) {
    const Brick& br = bricks[id];
    uint8_t* r = o + rec_off + 4 * (size_t)starts[id];
    put32(r, (uint32_t)br.pal.size());
    put32(r + 4, (uint32_t)br.sym.size());
    put32(r + 8, br.coded_bytes);
    put32(r + 12, br.n_delta);
    uint8_t* q = r + 16;
    if (coder == 1)
      for (uint32_t h : br.head) { put32(q, h); q += 4; }
    for (uint32_t v : br.pal) { put32(q, v); q += 4; }
    if (coder == 1) {
      for (size_t w = 0; w < br.words.size(); ++w) { q[2 * w] = (uint8_t)br.words[w]; q[2 * w + 1] = (uint8_t)(br.words[w] >> 8); }
    } else {
      for (size_t i = 0; i < br.sym.size(); ++i) q[i >> 1] |= (uint8_t)(br.sym[i] << ((i & 1) * 4));
    }
  });
  *out_bytes = o;
  *out_size = size;
  return VC_OK;
}

vc_status vc_encode_volume(const uint32_t* voxels, const uint32_t dims[3], uint32_t log2b, uint32_t op_mask,
                           uint32_t coder, uint32_t flags, uint32_t threads, uint8_t** out_bytes, size_t* out_size) {
  return vc_encode_volume_freq(voxels, dims, log2b, op_mask, coder, flags, threads, nullptr, out_bytes, out_size);
}

vc_status vc_concat_volumes_z(const uint8_t* const* parts, const size_t* sizes, uint32_t nparts, uint8_t** out_bytes,
                              size_t* out_size) {
  if (!parts || !sizes || !nparts || !out_bytes || !out_size) return VC_ERR_ARG;
  *out_bytes = nullptr;
  *out_size = 0;
  auto get32 = [](const uint8_t* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
  };
  uint32_t dz = 0, max_pal = 0, max_sym = 0;
  uint64_t n_total = 0, words_total = 0;
  for (uint32_t k = 0; k < nparts; ++k) {
    const uint8_t* p = parts[k];
    if (!p || sizes[k] < 128 || get32(p) != 0x315A4356u || get32(p + 4) != 1u) return VC_ERR_FORMAT;
    const uint32_t log2b = get32(p + 20), b = 1u << (log2b & 7u);
    const uint32_t n = get32(p + 36), words = get32(p + 112);
    const size_t rec_off = (128 + 4 * ((size_t)n + 1) + 15) & ~(size_t)15;
    if (log2b < 1 || log2b > 6 || sizes[k] < rec_off + 4ull * words) return VC_ERR_FORMAT;
    // the same brick size, operations, coder, flags, x / y extent and rANS table in every part;
    // every part but the last covers whole bricks in z
    if (k > 0 && (std::memcmp(p + 8, parts[0] + 8, 8) != 0 || std::memcmp(p + 20, parts[0] + 20, 16) != 0 ||
                  std::memcmp(p + 48, parts[0] + 48, 64) != 0))
      return VC_ERR_ARG;
    if (k + 1 < nparts && get32(p + 16) % b != 0) return VC_ERR_ARG;
    dz += get32(p + 16);
    n_total += n;
    words_total += words;
    max_pal = std::max(max_pal, get32(p + 40));
    max_sym = std::max(max_sym, get32(p + 44));
  }
  if (n_total >= 0xFFFFFFFFull || words_total >= 0xFFFFFFFFull) return VC_ERR_ARG;
  const uint32_t n = (uint32_t)n_total;
  const size_t rec_off = (128 + 4 * ((size_t)n + 1) + 15) & ~(size_t)15;
  const size_t size = rec_off + 4 * words_total;
  uint8_t* o = static_cast<uint8_t*>(std::calloc(size, 1));
  if (!o) return VC_ERR_OOM;
  std::memcpy(o, parts[0], 128);
  put32(o + 16, dz);
  put32(o + 36, n);
  put32(o + 40, max_pal);
  put32(o + 44, max_sym);
  put32(o + 112, (uint32_t)words_total);
  uint32_t id = 0, wbase = 0;
  size_t rpos = rec_off;
  for (uint32_t k = 0; k < nparts; ++k) {
    const uint8_t* p = parts[k];
    const uint32_t pn = get32(p + 36), words = get32(p + 112);
    const size_t prec = (128 + 4 * ((size_t)pn + 1) + 15) & ~(size_t)15;
    for (uint32_t i = 0; i < pn; ++i) put32(o + 128 + 4 * (size_t)(id + i), wbase + get32(p + 128 + 4 * (size_t)i));
    std::memcpy(o + rpos, p + prec, 4ull * words);
    id += pn;
    wbase += words;
    rpos += 4ull * words;
  }
  put32(o + 128 + 4 * (size_t)n, wbase);
  *out_bytes = o;
  *out_size = size;
  return VC_OK;
}

void vc_free_bytes(uint8_t* bytes) { std::free(bytes); }

}  // extern "C"
