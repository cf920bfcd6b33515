/*
 * CSGV oracle: a plain, slow, single-threaded CPU encoder and decoder for the compressed
 * segmentation volume encoding of Volcanite (Methods, "Compressed segmentation volumes";
 * Fig. "CSGV" caption; Supplementary Fig. "CSGV ablation" caption).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this code. It shares no code, header or table with the GPU library; the two meet
 * only in the byte format, which each side implements from its written definition.
 *
 * Everything here follows the definitions step by step, in the paper's order, with no blocking,
 * fusion or reordering:
 *   - a brick of b^3 voxels (b = 2^L) is a multi-resolution grid; level l has (2^l)^3 nodes,
 *     level L is the voxels; a coarser node holds the most frequent label of its 2^3 children
 *     (Results, "Ray marching": a mipmap of modes);
 *   - nodes are emitted level by level, coarse to fine, one operation per node; a node whose
 *     stop bit is set marks a constant subtree, whose nodes are not emitted in finer levels
 *     (Results, "CSGV results");
 *   - operations: copy the parent's label, copy the x / y / z neighbour that has a different
 *     parent, read the next palette entry (advance), re-read the previous entry (delta = 1),
 *     re-read the entry delta back (Supplementary Fig. "CSGV ablation" caption);
 *   - unlimited delta: after the delta operation come 4-bit entries holding 3 payload bits, most
 *     significant group first, and one "another entry follows" bit, with
 *     delta <- (delta << 3) | (entry & 7) (Methods, "Compressed segmentation volumes");
 *   - operations other than palette advance may be disabled at compression time (same section);
 *   - the 4-bit symbol stream is stored plain (two per byte) or range-ANS coded (Methods, "GPU
 *     rendering pipeline"; Duda's ANS) with 32 interleaved states;
 *   - Brick Starts are 32-bit offsets in 32-bit words (Methods, "Encoding buffer optimizations").
 * Where the paper is silent (op codes, traversal order inside a level, tie-breaks, the rANS
 * parameters, the record layout) this file takes the readings written down in the design notes;
 * each is restated at the point of use.
 *
 * Parity pins live in the tests: lossless round trip, palette = distinct labels, stop-bit
 * subtrees uniform, coarse levels = mode pyramid recomputed from V, delta nibble counts in closed
 * form, brute-force enumeration of every legal operation choice on tiny bricks, rANS round trip
 * and size within the entropy bound.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

/* ---- numeric constants of the byte format (written independently on each side) ---- */
#define O_MAGIC 0x315A4356u /* "VCZ1" little endian */
#define O_VERSION 1u
#define O_HEADER_BYTES 128u
#define O_OK 0
#define O_ERR_ARG (-1)
#define O_ERR_FORMAT (-2)
#define O_ERR_OOM (-3)
#define O_ERR_CORRUPT (-5)

/* operation codes (a 3-bit field; bit 3 of the symbol is the stop bit) */
#define OP_PARENT 0
#define OP_NX 1
#define OP_NY 2
#define OP_NZ 3
#define OP_ADV 4
#define OP_LAST 5
#define OP_DELTA 6
#define OP_ALL 0x7Fu

#define CODER_PLAIN 0u
#define CODER_RANS 1u
#define FLAG_NO_STOP 1u /* encoder wrote no stop bits; a set stop bit is corrupt */
/* limited back references, the earlier encoding's form (Results, "CSGV segmentation volume
 * compression", and Supplementary Fig. "CSGV ablation" caption: the original back reference
 * stores 1 < delta <= 16 in one 4-bit entry of the operation stream; Methods, "Compressed
 * segmentation volumes": that entry is limited to 4 bits). Reading of the 4 bits: the entry
 * holds delta - 1, so entries 1..15 give delta 2..16 and entry 0 (delta 1) is corrupt; bit 3
 * does not chain. A label further back than 16 entries is appended to the palette again. */
#define FLAG_SHORT_DELTA 2u
#define SHORT_DELTA_MIN 2u
#define SHORT_DELTA_MAX 16u

/* rANS runs (flags bits 2..3 = log2 K, K = 1, 2, 4 or 8; rANS volumes only): a record's S symbols
 * are cut into runs of Q = 32 ceil(S / 32K) symbols (the last may be shorter, and small records
 * have fewer than K runs), each coded on its own with 32 interleaved states, so that a decoder can
 * decode the runs side by side. Not in the paper, which leaves the coder's layout to its encoder
 * implementations; K = 1 is the single-run record. */
#define FLAG_RUNS_SHIFT 2u
#define FLAG_RUNS_MASK (3u << FLAG_RUNS_SHIFT)
#define FLAGS_ALL (FLAG_NO_STOP | FLAG_SHORT_DELTA | FLAG_RUNS_MASK)

#define RANS_BITS 12
#define RANS_M (1u << RANS_BITS)
#define RANS_L (1u << 16)
#define RANS_LANES 32u
#define MAX_DELTA_ENTRIES 7

static inline uint32_t rd32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static inline void wr32(uint8_t* p, uint32_t v) {
  p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
}

/* Morton code m of level coordinates: bit 3i of m is bit i of x, 3i+1 of y, 3i+2 of z. */
static void demorton3(uint32_t m, int bits, uint32_t c[3]) {
  c[0] = c[1] = c[2] = 0;
  for (int i = 0; i < bits; ++i) {
    c[0] |= ((m >> (3 * i)) & 1u) << i;
    c[1] |= ((m >> (3 * i + 1)) & 1u) << i;
    c[2] |= ((m >> (3 * i + 2)) & 1u) << i;
  }
}
/* linear index of a level cell (x fastest) */
static inline size_t lin(const uint32_t c[3], uint32_t n) { return ((size_t)c[2] * n + c[1]) * n + c[0]; }

/* ===================================================================================== */
/* Unlimited delta back references (Methods, "Compressed segmentation volumes").          */
/* ===================================================================================== */

/* Writes the 4-bit entries for delta >= 1 (minimal count, most significant group first, bit 3
 * set on every entry but the last). Returns the number of entries. */
int oracle_delta_nibbles(uint32_t delta, uint8_t* out) {
  int n = 1;
  while (n < 11 && (delta >> (3 * n)) != 0) ++n;
  for (int i = 0; i < n; ++i) {
    uint32_t group = (delta >> (3 * (n - 1 - i))) & 7u;
    out[i] = (uint8_t)(group | (i + 1 < n ? 8u : 0u));
  }
  return n;
}

/* ===================================================================================== */
/* rANS (Duda): 16-symbol alphabet, M = 2^12, 32-bit states in [2^16, 2^32), 16-bit words, */
/* 32 interleaved states: symbol i uses state i mod 32.                                   */
/* ===================================================================================== */

/* Quantise symbol counts to frequencies summing to M, every present symbol >= 1:
 * f = max(1, floor(count * M / total)); the shortfall goes to the most frequent symbol (lowest
 * on ties); an excess is taken one unit at a time from the largest frequency (lowest on ties). */
int oracle_rans_quantize(const uint64_t counts[16], uint32_t freq[16]) {
  uint64_t total = 0;
  for (int s = 0; s < 16; ++s) total += counts[s];
  for (int s = 0; s < 16; ++s) freq[s] = 0;
  if (total == 0) { freq[OP_ADV] = RANS_M; return 0; }
  int64_t sum = 0;
  for (int s = 0; s < 16; ++s) {
    if (counts[s] == 0) continue;
    uint64_t f = (counts[s] * RANS_M) / total;
    freq[s] = (uint32_t)(f < 1 ? 1 : f);
    sum += freq[s];
  }
  int64_t diff = (int64_t)RANS_M - sum;
  if (diff > 0) {
    int best = 0;
    for (int s = 1; s < 16; ++s) if (counts[s] > counts[best]) best = s;
    freq[best] += (uint32_t)diff;
  }
  while (diff < 0) {
    int best = -1;
    for (int s = 0; s < 16; ++s)
      if (freq[s] > 1 && (best < 0 || freq[s] > freq[best])) best = s;
    if (best < 0) return O_ERR_ARG;
    freq[best] -= 1;
    ++diff;
  }
  return 0;
}

static void rans_cum(const uint32_t freq[16], uint32_t cum[17]) {
  cum[0] = 0;
  for (int s = 0; s < 16; ++s) cum[s + 1] = cum[s] + freq[s];
}

/* Encode S symbols. Writes n_states = min(S, 32) final states and the 16-bit word stream in the
 * order the decoder reads it. Returns the word count, or -1 if a symbol has frequency 0. */
static long rans_encode(const uint8_t* sym, uint32_t S, const uint32_t freq[16], uint32_t* states,
                        uint16_t* words) {
  uint32_t cum[17];
  rans_cum(freq, cum);
  uint32_t x[RANS_LANES];
  for (uint32_t l = 0; l < RANS_LANES; ++l) x[l] = RANS_L;
  long nw = 0;
  uint32_t T = (S + RANS_LANES - 1) / RANS_LANES;
  /* the decoder reads words step by step, lanes in ascending order within a step; the encoder
   * therefore runs steps and lanes in descending order and reverses the emitted words */
  for (uint32_t t = T; t-- > 0;) {
    for (uint32_t l = RANS_LANES; l-- > 0;) {
      uint32_t i = t * RANS_LANES + l;
      if (i >= S) continue;
      uint32_t s = sym[i], f = freq[s];
      if (f == 0) return -1;
      uint64_t xmax = ((uint64_t)(RANS_L >> RANS_BITS) << 16) * f;
      if ((uint64_t)x[l] >= xmax) {
        words[nw++] = (uint16_t)(x[l] & 0xFFFFu);
        x[l] >>= 16;
      }
      x[l] = ((x[l] / f) << RANS_BITS) + (x[l] % f) + cum[s];
    }
  }
  for (long a = 0, b = nw - 1; a < b; ++a, --b) { uint16_t t2 = words[a]; words[a] = words[b]; words[b] = t2; }
  uint32_t ns = S < RANS_LANES ? S : RANS_LANES;
  for (uint32_t l = 0; l < ns; ++l) states[l] = x[l];
  return nw;
}

/* Runs of a record of S symbols (see FLAG_RUNS_SHIFT): run length Q and number of runs. */
static uint32_t runs_of(uint32_t flags) { return 1u << ((flags & FLAG_RUNS_MASK) >> FLAG_RUNS_SHIFT); }
static uint32_t run_len(uint32_t S, uint32_t K) {
  const uint32_t per = (S + 32u * K - 1u) / (32u * K);
  return 32u * (per ? per : 1u);
}
static uint32_t run_count(uint32_t S, uint32_t K) {
  const uint32_t q = run_len(S, K);
  return S ? (S + q - 1u) / q : 1u;
}
static uint32_t run_size(uint32_t S, uint32_t K, uint32_t k) {
  const uint32_t q = run_len(S, K);
  const uint32_t len = S > k * q ? S - k * q : 0u;
  return len < q ? len : q;
}
/* Words between a rANS record's header and its palette: every run's final states (min(run, 32)
 * each, run after run), then the first coded word of every run but the first. */
static uint32_t rans_head_words(uint32_t S, uint32_t K) {
  const uint32_t n = run_count(S, K);
  uint32_t w = n - 1u;
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t len = run_size(S, K, k);
    w += len < RANS_LANES ? len : RANS_LANES;
  }
  return w;
}

/* Words between a record's header and its palette, for the other oracle files (0 for plain). */
uint32_t oracle_head_words(uint32_t coder, uint32_t flags, uint32_t S) {
  return coder == CODER_RANS ? rans_head_words(S, runs_of(flags)) : 0u;
}

/* Decode S symbols from n_states initial states and nw 16-bit words (little-endian bytes).
 * Every lane decodes its symbol of the step; then, in lane order, each lane whose state fell
 * below 2^16 shifts in the next word. The stream is valid iff no read runs past the words, all
 * words are read and every state ends at 2^16. */
static int rans_decode(const uint32_t* states0, const uint8_t* wbytes, uint32_t nw, uint32_t S,
                       const uint32_t freq[16], uint8_t* sym) {
  uint32_t cum[17];
  rans_cum(freq, cum);
  uint32_t x[RANS_LANES];
  uint32_t ns = S < RANS_LANES ? S : RANS_LANES;
  for (uint32_t l = 0; l < RANS_LANES; ++l) x[l] = l < ns ? states0[l] : RANS_L;
  for (uint32_t l = 0; l < ns; ++l)
    if (x[l] < RANS_L) return O_ERR_CORRUPT;
  uint32_t ptr = 0;
  uint32_t T = (S + RANS_LANES - 1) / RANS_LANES;
  for (uint32_t t = 0; t < T; ++t) {
    for (uint32_t l = 0; l < RANS_LANES; ++l) {
      uint32_t i = t * RANS_LANES + l;
      if (i >= S) continue;
      uint32_t slot = x[l] & (RANS_M - 1);
      uint32_t s = 0;
      while (s < 15 && cum[s + 1] <= slot) ++s;
      sym[i] = (uint8_t)s;
      x[l] = freq[s] * (x[l] >> RANS_BITS) + slot - cum[s];
    }
    for (uint32_t l = 0; l < RANS_LANES; ++l) {
      uint32_t i = t * RANS_LANES + l;
      if (i >= S) continue;
      if (x[l] < RANS_L) {
        if (ptr >= nw) return O_ERR_CORRUPT;
        uint32_t w = (uint32_t)wbytes[2 * ptr] | ((uint32_t)wbytes[2 * ptr + 1] << 8);
        x[l] = (x[l] << 16) | w;
        ++ptr;
      }
    }
  }
  if (ptr != nw) return O_ERR_CORRUPT;
  for (uint32_t l = 0; l < ns; ++l)
    if (x[l] != RANS_L) return O_ERR_CORRUPT;
  return 0;
}

/* Code S symbols as run_count(S, K) runs: head[] receives rans_head_words(S, K) words (the runs'
 * states, then where runs 1.. start in the words), words[] the runs' words one run after the
 * other (room for S words). Returns the word count, or -1 if a symbol has frequency 0. */
static long rans_encode_runs(const uint8_t* sym, uint32_t S, const uint32_t freq[16], uint32_t K, uint32_t* head,
                             uint16_t* words) {
  const uint32_t n = run_count(S, K), q = run_len(S, K);
  uint32_t n_states = 0;
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t len = run_size(S, K, k);
    n_states += len < RANS_LANES ? len : RANS_LANES;
  }
  uint32_t hs = 0;
  long nw = 0;
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t len = run_size(S, K, k);
    if (k) head[n_states + k - 1u] = (uint32_t)nw;
    const long w = rans_encode(sym + (size_t)k * q, len, freq, head + hs, words + nw);
    if (w < 0) return -1;
    hs += len < RANS_LANES ? len : RANS_LANES;
    nw += w;
  }
  return nw;
}

/* Decode the runs of a record: head points at its rans_head_words(S, K) words. The run starts
 * must not decrease and stay within the nw words; every run must read exactly its words. */
static int rans_decode_runs(const uint8_t* head, uint32_t S, uint32_t K, const uint8_t* wbytes, uint32_t nw,
                            const uint32_t freq[16], uint8_t* sym) {
  const uint32_t n = run_count(S, K), q = run_len(S, K);
  uint32_t n_states = 0;
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t len = run_size(S, K, k);
    n_states += len < RANS_LANES ? len : RANS_LANES;
  }
  uint32_t hs = 0;
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t len = run_size(S, K, k);
    const uint32_t w0 = k ? rd32(head + 4 * ((size_t)n_states + k - 1u)) : 0u;
    const uint32_t w1 = k + 1u < n ? rd32(head + 4 * ((size_t)n_states + k)) : nw;
    if (w0 > w1 || w1 > nw) return O_ERR_CORRUPT;
    uint32_t st[RANS_LANES];
    const uint32_t ns = len < RANS_LANES ? len : RANS_LANES;
    for (uint32_t l = 0; l < ns; ++l) st[l] = rd32(head + 4 * ((size_t)hs + l));
    const int rc = rans_decode(st, wbytes + 2 * (size_t)w0, w1 - w0, len, freq, sym + (size_t)k * q);
    if (rc) return rc;
    hs += ns;
  }
  return 0;
}

/* ===================================================================================== */
/* Brick hierarchy and operation stream (encoder side).                                   */
/* ===================================================================================== */

typedef struct {
  int L;
  uint32_t* lab[7]; /* lab[l][lin(c, 2^l)] */
  uint8_t* uni[7];  /* all voxels below are equal */
} hierarchy;

static void hier_free(hierarchy* h) {
  for (int l = 0; l <= h->L; ++l) { free(h->lab[l]); free(h->uni[l]); }
}

/* Mode of 8 labels; ties go to the smallest label value. */
static uint32_t mode8(const uint32_t v[8]) {
  uint32_t best = 0;
  int best_n = 0;
  for (int i = 0; i < 8; ++i) {
    int n = 0;
    for (int j = 0; j < 8; ++j) n += (v[j] == v[i]);
    if (n > best_n || (n == best_n && v[i] < best)) { best = v[i]; best_n = n; }
  }
  return best;
}

/* Level L = voxels; level l-1 node = mode of its 2^3 children; uniform = 8 uniform children
 * with one label. */
static int hier_build(const uint32_t* brick, int L, hierarchy* h) {
  h->L = L;
  for (int l = 0; l <= L; ++l) { h->lab[l] = NULL; h->uni[l] = NULL; }
  for (int l = 0; l <= L; ++l) {
    size_t n = (size_t)1 << (3 * l);
    h->lab[l] = (uint32_t*)malloc(n * sizeof(uint32_t));
    h->uni[l] = (uint8_t*)malloc(n);
    if (!h->lab[l] || !h->uni[l]) { hier_free(h); return O_ERR_OOM; }
  }
  size_t nv = (size_t)1 << (3 * L);
  memcpy(h->lab[L], brick, nv * sizeof(uint32_t));
  memset(h->uni[L], 1, nv);
  for (int l = L; l > 0; --l) {
    uint32_t n = 1u << (l - 1), nc = 1u << l;
    for (uint32_t z = 0; z < n; ++z)
      for (uint32_t y = 0; y < n; ++y)
        for (uint32_t x = 0; x < n; ++x) {
          uint32_t v[8];
          int all_uni = 1;
          for (int o = 0; o < 8; ++o) {
            uint32_t c[3] = {2 * x + (o & 1), 2 * y + ((o >> 1) & 1), 2 * z + ((o >> 2) & 1)};
            v[o] = h->lab[l][lin(c, nc)];
            all_uni &= h->uni[l][lin(c, nc)];
          }
          int same = 1;
          for (int o = 1; o < 8; ++o) same &= (v[o] == v[0]);
          uint32_t p[3] = {x, y, z};
          h->lab[l - 1][lin(p, n)] = mode8(v);
          h->uni[l - 1][lin(p, n)] = (uint8_t)(all_uni && same);
        }
  }
  return 0;
}

typedef struct {
  uint8_t* sym;
  uint32_t n_sym, cap;
  uint32_t* pal;
  uint32_t n_pal, pal_cap;
  uint32_t n_delta;
} brick_stream;

static int push_sym(brick_stream* s, uint8_t v) {
  if (s->n_sym == s->cap) {
    uint32_t nc = s->cap ? 2 * s->cap : 256;
    uint8_t* p = (uint8_t*)realloc(s->sym, nc);
    if (!p) return O_ERR_OOM;
    s->sym = p; s->cap = nc;
  }
  s->sym[s->n_sym++] = v;
  return 0;
}
static int push_pal(brick_stream* s, uint32_t v) {
  if (s->n_pal == s->pal_cap) {
    uint32_t nc = s->pal_cap ? 2 * s->pal_cap : 64;
    uint32_t* p = (uint32_t*)realloc(s->pal, nc * sizeof(uint32_t));
    if (!p) return O_ERR_OOM;
    s->pal = p; s->pal_cap = nc;
  }
  s->pal[s->n_pal++] = v;
  return 0;
}

/* Encode one brick: levels 0..L, Morton order inside a level, only nodes without a stopped
 * ancestor; per node the first applicable enabled operation in the paper's order
 * (parent, x, y, z neighbour, last, delta) and palette advance otherwise. */
static int encode_brick(const uint32_t* brick, int L, uint32_t op_mask, uint32_t flags, brick_stream* out) {
  hierarchy h;
  int rc = hier_build(brick, L, &h);
  if (rc) return rc;
  memset(out, 0, sizeof(*out));
  const int use_stop = !(flags & FLAG_NO_STOP);
  const int short_delta = (flags & FLAG_SHORT_DELTA) != 0;
  uint8_t* expanded[7]; /* emitted with stop = 0 */
  for (int l = 0; l <= L; ++l) {
    expanded[l] = (uint8_t*)calloc((size_t)1 << (3 * l), 1);
    if (!expanded[l]) { for (int q = 0; q < l; ++q) free(expanded[q]); hier_free(&h); return O_ERR_OOM; }
  }
  for (int l = 0; l <= L && !rc; ++l) {
    uint32_t n = 1u << l;
    uint32_t cnt = 1u << (3 * l);
    for (uint32_t m = 0; m < cnt && !rc; ++m) {
      uint32_t c[3];
      demorton3(m, l, c);
      uint32_t pc[3] = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
      if (l > 0 && !expanded[l - 1][lin(pc, n >> 1)]) continue; /* inside a stopped subtree */
      uint32_t label = h.lab[l][lin(c, n)];
      int stop = (l < L && use_stop) ? h.uni[l][lin(c, n)] : 0;
      expanded[l][lin(c, n)] = (uint8_t)(l < L && !stop);
      int op = -1;
      uint32_t delta = 0;
      if ((op_mask >> OP_PARENT & 1) && l > 0 && h.lab[l - 1][lin(pc, n >> 1)] == label) op = OP_PARENT;
      for (int a = 0; a < 3 && op < 0; ++a) {
        if (!(op_mask >> (OP_NX + a) & 1)) continue;
        if ((c[a] & 1u) || c[a] == 0) continue; /* the neighbour must lie in another parent */
        uint32_t q[3] = {c[0], c[1], c[2]};
        q[a] -= 1;
        if (h.lab[l][lin(q, n)] == label) op = OP_NX + a;
      }
      if (op < 0 && (op_mask >> OP_LAST & 1) && out->n_pal >= 1 && out->pal[out->n_pal - 1] == label) op = OP_LAST;
      if (op < 0 && (op_mask >> OP_DELTA & 1)) {
        uint32_t reach = out->n_pal;
        if (short_delta && reach > SHORT_DELTA_MAX) reach = SHORT_DELTA_MAX;
        for (uint32_t d = 2; d <= reach; ++d)
          if (out->pal[out->n_pal - d] == label) { op = OP_DELTA; delta = d; break; }
      }
      if (op < 0) { op = OP_ADV; rc = push_pal(out, label); }
      if (!rc) rc = push_sym(out, (uint8_t)(op | (stop << 3)));
      if (!rc && op == OP_DELTA) {
        if (short_delta) {
          rc = push_sym(out, (uint8_t)(delta - 1u)); /* one entry: delta - 1 */
        } else {
          uint8_t e[11];
          int ne = oracle_delta_nibbles(delta, e);
          for (int i = 0; i < ne && !rc; ++i) rc = push_sym(out, e[i]);
        }
        out->n_delta++;
      }
    }
  }
  for (int l = 0; l <= L; ++l) free(expanded[l]);
  hier_free(&h);
  return rc;
}

/* ===================================================================================== */
/* Volume encoder                                                                          */
/* ===================================================================================== */

void oracle_free(void* p) { free(p); }

/* Encode a full volume V (x fastest, dims[0] * dims[1] * dims[2] labels).
 * Bricks: b = 2^log2b; brick (bx, by, bz) has id bx + nbx * (by + nby * bz); voxels beyond the
 * volume repeat the nearest edge voxel (clamp to edge). Output buffer: malloc'd, oracle_free. */
int oracle_encode_volume(const uint32_t* V, const uint32_t dims[3], uint32_t log2b, uint32_t op_mask,
                         uint32_t coder, uint32_t flags, uint8_t** out_bytes, size_t* out_size) {
  if (!V || !dims || !out_bytes || !out_size) return O_ERR_ARG;
  if (log2b < 1 || log2b > 6) return O_ERR_ARG;
  if (!(op_mask & (1u << OP_ADV)) || (op_mask & ~OP_ALL)) return O_ERR_ARG;
  if (coder > CODER_RANS || (flags & ~FLAGS_ALL)) return O_ERR_ARG;
  if (coder != CODER_RANS && (flags & FLAG_RUNS_MASK)) return O_ERR_ARG;
  for (int a = 0; a < 3; ++a) if (dims[a] == 0) return O_ERR_ARG;
  const uint32_t b = 1u << log2b;
  const int L = (int)log2b;
  uint32_t nb[3];
  for (int a = 0; a < 3; ++a) nb[a] = (dims[a] + b - 1) / b;
  const uint64_t n_bricks64 = (uint64_t)nb[0] * nb[1] * nb[2];
  if (n_bricks64 >= 0xFFFFFFFFull) return O_ERR_ARG;
  const uint32_t n_bricks = (uint32_t)n_bricks64;
  const size_t bv = (size_t)b * b * b;

  brick_stream* bs = (brick_stream*)calloc(n_bricks, sizeof(brick_stream));
  uint32_t* brick = (uint32_t*)malloc(bv * sizeof(uint32_t));
  if (!bs || !brick) { free(bs); free(brick); return O_ERR_OOM; }
  int rc = 0;
  uint64_t counts[16] = {0};
  for (uint32_t id = 0; id < n_bricks && !rc; ++id) {
    uint32_t bc[3] = {id % nb[0], (id / nb[0]) % nb[1], id / (nb[0] * nb[1])};
    for (uint32_t z = 0; z < b; ++z)
      for (uint32_t y = 0; y < b; ++y)
        for (uint32_t x = 0; x < b; ++x) {
          uint64_t g[3] = {(uint64_t)bc[0] * b + x, (uint64_t)bc[1] * b + y, (uint64_t)bc[2] * b + z};
          for (int a = 0; a < 3; ++a) if (g[a] >= dims[a]) g[a] = dims[a] - 1;
          brick[((size_t)z * b + y) * b + x] = V[(g[2] * dims[1] + g[1]) * dims[0] + g[0]];
        }
    rc = encode_brick(brick, L, op_mask, flags, &bs[id]);
    if (!rc) for (uint32_t i = 0; i < bs[id].n_sym; ++i) counts[bs[id].sym[i]]++;
  }
  free(brick);
  uint32_t freq[16] = {0};
  if (!rc && coder == CODER_RANS) rc = oracle_rans_quantize(counts, freq);

  /* records: header {n_pal, n_sym, coded_bytes, n_delta}, [rANS states and run starts],
   * palette, stream, zero padding to 16 bytes */
  const uint32_t K = runs_of(flags);
  uint8_t** rec = (uint8_t**)calloc(n_bricks, sizeof(uint8_t*));
  uint32_t* rec_words = (uint32_t*)calloc(n_bricks, sizeof(uint32_t));
  uint64_t total_words = 0;
  uint32_t max_pal = 0, max_sym = 0;
  if (!rec || !rec_words) rc = O_ERR_OOM;
  for (uint32_t id = 0; id < n_bricks && !rc; ++id) {
    brick_stream* s = &bs[id];
    uint32_t ns = (coder == CODER_RANS) ? rans_head_words(s->n_sym, K) : 0;
    uint32_t coded_bytes;
    uint16_t* words = NULL;
    uint32_t states[8 * RANS_LANES + 8];
    if (coder == CODER_RANS) {
      /* a 16-bit word per renormalisation; at most one per symbol */
      words = (uint16_t*)malloc(((size_t)s->n_sym + 1) * sizeof(uint16_t));
      if (!words) { rc = O_ERR_OOM; break; }
      long nw = rans_encode_runs(s->sym, s->n_sym, freq, K, states, words);
      if (nw < 0) { free(words); rc = O_ERR_ARG; break; }
      coded_bytes = (uint32_t)(2 * nw);
    } else {
      coded_bytes = (s->n_sym + 1) / 2;
    }
    size_t bytes = 16 + 4 * (size_t)ns + 4 * (size_t)s->n_pal + coded_bytes;
    size_t padded = (bytes + 15) & ~(size_t)15;
    uint8_t* r = (uint8_t*)calloc(padded, 1);
    if (!r) { free(words); rc = O_ERR_OOM; break; }
    wr32(r + 0, s->n_pal);
    wr32(r + 4, s->n_sym);
    wr32(r + 8, coded_bytes);
    wr32(r + 12, s->n_delta);
    uint8_t* p = r + 16;
    for (uint32_t l = 0; l < ns; ++l, p += 4) wr32(p, states[l]);
    for (uint32_t i = 0; i < s->n_pal; ++i, p += 4) wr32(p, s->pal[i]);
    if (coder == CODER_RANS) {
      for (uint32_t w = 0; w < coded_bytes / 2; ++w) { p[2 * w] = (uint8_t)words[w]; p[2 * w + 1] = (uint8_t)(words[w] >> 8); }
    } else {
      for (uint32_t i = 0; i < s->n_sym; ++i) p[i / 2] |= (uint8_t)((s->sym[i] & 15u) << (4 * (i & 1)));
    }
    free(words);
    rec[id] = r;
    rec_words[id] = (uint32_t)(padded / 4);
    total_words += padded / 4;
    if (s->n_pal > max_pal) max_pal = s->n_pal;
    if (s->n_sym > max_sym) max_sym = s->n_sym;
  }
  if (!rc && total_words >= 0xFFFFFFFFull) rc = O_ERR_ARG; /* 32-bit word offsets: 16 GiB */

  if (!rc) {
    size_t starts_bytes = 4 * ((size_t)n_bricks + 1);
    size_t rec_off = (O_HEADER_BYTES + starts_bytes + 15) & ~(size_t)15;
    size_t size = rec_off + 4 * (size_t)total_words;
    uint8_t* o = (uint8_t*)calloc(size, 1);
    if (!o) rc = O_ERR_OOM;
    else {
      wr32(o + 0, O_MAGIC);
      wr32(o + 4, O_VERSION);
      wr32(o + 8, dims[0]); wr32(o + 12, dims[1]); wr32(o + 16, dims[2]);
      wr32(o + 20, log2b);
      wr32(o + 24, op_mask);
      wr32(o + 28, coder);
      wr32(o + 32, flags);
      wr32(o + 36, n_bricks);
      wr32(o + 40, max_pal);
      wr32(o + 44, max_sym);
      for (int s = 0; s < 16; ++s) wr32(o + 48 + 4 * s, freq[s]);
      wr32(o + 112, (uint32_t)total_words);
      uint32_t acc = 0;
      for (uint32_t id = 0; id < n_bricks; ++id) {
        wr32(o + O_HEADER_BYTES + 4 * (size_t)id, acc);
        memcpy(o + rec_off + 4 * (size_t)acc, rec[id], 4 * (size_t)rec_words[id]);
        acc += rec_words[id];
      }
      wr32(o + O_HEADER_BYTES + 4 * (size_t)n_bricks, acc);
      *out_bytes = o;
      *out_size = size;
    }
  }
  for (uint32_t id = 0; id < n_bricks; ++id) {
    free(bs[id].sym); free(bs[id].pal);
    if (rec) free(rec[id]);
  }
  free(bs); free(rec); free(rec_words);
  return rc;
}

/* ===================================================================================== */
/* Decoder                                                                                 */
/* ===================================================================================== */

typedef struct {
  uint32_t dims[3], L, op_mask, coder, flags, n_bricks, max_pal, max_sym, records_words;
  uint32_t freq[16];
  const uint8_t* starts;
  const uint8_t* records;
} vol_view;

static int parse_volume(const uint8_t* v, size_t size, vol_view* o) {
  if (!v || size < O_HEADER_BYTES) return O_ERR_FORMAT;
  if (rd32(v) != O_MAGIC || rd32(v + 4) != O_VERSION) return O_ERR_FORMAT;
  for (int a = 0; a < 3; ++a) o->dims[a] = rd32(v + 8 + 4 * a);
  o->L = rd32(v + 20);
  o->op_mask = rd32(v + 24);
  o->coder = rd32(v + 28);
  o->flags = rd32(v + 32);
  o->n_bricks = rd32(v + 36);
  o->max_pal = rd32(v + 40);
  o->max_sym = rd32(v + 44);
  for (int s = 0; s < 16; ++s) o->freq[s] = rd32(v + 48 + 4 * s);
  o->records_words = rd32(v + 112);
  if (o->L < 1 || o->L > 6) return O_ERR_FORMAT;
  if (!(o->op_mask & (1u << OP_ADV)) || (o->op_mask & ~OP_ALL)) return O_ERR_FORMAT;
  if (o->coder > CODER_RANS || (o->flags & ~FLAGS_ALL)) return O_ERR_FORMAT;
  if (o->coder != CODER_RANS && (o->flags & FLAG_RUNS_MASK)) return O_ERR_FORMAT;
  uint32_t b = 1u << o->L;
  uint64_t nb = 1;
  for (int a = 0; a < 3; ++a) {
    if (o->dims[a] == 0) return O_ERR_FORMAT;
    nb *= (o->dims[a] + b - 1) / b;
  }
  if (nb != o->n_bricks) return O_ERR_FORMAT;
  if (o->coder == CODER_RANS) {
    uint32_t sum = 0;
    for (int s = 0; s < 16; ++s) sum += o->freq[s];
    if (sum != RANS_M) return O_ERR_FORMAT;
  }
  size_t starts_bytes = 4 * ((size_t)o->n_bricks + 1);
  size_t rec_off = (O_HEADER_BYTES + starts_bytes + 15) & ~(size_t)15;
  if (size < rec_off + 4 * (size_t)o->records_words) return O_ERR_FORMAT;
  o->starts = v + O_HEADER_BYTES;
  o->records = v + rec_off;
  return 0;
}

/* Locate and check one record; returns its symbols (malloc'd) and palette view. */
static int brick_symbols(const vol_view* V, uint32_t id, uint8_t** sym_out, uint32_t* S_out,
                         const uint8_t** pal_out, uint32_t* n_pal_out, uint32_t* n_delta_out) {
  if (id >= V->n_bricks) return O_ERR_ARG;
  uint32_t a = rd32(V->starts + 4 * (size_t)id), e = rd32(V->starts + 4 * ((size_t)id + 1));
  if (a > e || e > V->records_words || (a & 3u) || (e & 3u) || e - a < 4) return O_ERR_FORMAT;
  const uint8_t* r = V->records + 4 * (size_t)a;
  size_t avail = 4 * (size_t)(e - a);
  uint32_t n_pal = rd32(r), S = rd32(r + 4), cb = rd32(r + 8), n_delta = rd32(r + 12);
  uint32_t ns = (V->coder == CODER_RANS) ? rans_head_words(S, runs_of(V->flags)) : 0;
  size_t need = 16 + 4 * (size_t)ns + 4 * (size_t)n_pal + cb;
  if (((need + 15) & ~(size_t)15) != avail) return O_ERR_FORMAT;
  if (V->coder == CODER_PLAIN && cb != (S + 1) / 2) return O_ERR_FORMAT;
  if (V->coder == CODER_RANS && (cb & 1u)) return O_ERR_FORMAT;
  if (S == 0) return O_ERR_CORRUPT;
  uint8_t* sym = (uint8_t*)malloc(S);
  if (!sym) return O_ERR_OOM;
  const uint8_t* states = r + 16;
  const uint8_t* pal = states + 4 * (size_t)ns;
  const uint8_t* coded = pal + 4 * (size_t)n_pal;
  if (V->coder == CODER_PLAIN) {
    for (uint32_t i = 0; i < S; ++i) sym[i] = (uint8_t)((coded[i / 2] >> (4 * (i & 1))) & 15u);
  } else {
    int rc = rans_decode_runs(states, S, runs_of(V->flags), coded, cb / 2, V->freq, sym);
    if (rc) { free(sym); return rc; }
  }
  *sym_out = sym; *S_out = S; *pal_out = pal; *n_pal_out = n_pal; *n_delta_out = n_delta;
  return 0;
}

/* One decoded node, for inspection by tests. */
typedef struct {
  int32_t level;
  uint32_t morton;
  int32_t op;
  int32_t stop;
  uint32_t delta;
  uint32_t label;
  uint32_t k; /* palette entries read so far (before this node) */
} oracle_node;

/* Replay the operation stream of one brick. Writes the labels of level L - lod in x-fastest
 * order to out (may be NULL) and, if nodes != NULL, one row per emitted node (up to max_nodes).
 * The whole stream is always replayed and checked, whatever lod is requested. */
static int replay(const vol_view* V, uint32_t id, uint32_t lod, uint32_t* out, oracle_node* nodes,
                  uint32_t max_nodes, uint32_t* n_nodes_out) {
  uint8_t* sym = NULL;
  uint32_t S = 0, n_pal = 0, n_delta = 0;
  const uint8_t* pal = NULL;
  int rc = brick_symbols(V, id, &sym, &S, &pal, &n_pal, &n_delta);
  if (rc) return rc;
  const int L = (int)V->L;
  if (lod > (uint32_t)L) { free(sym); return O_ERR_ARG; }
  uint32_t* lab[7];
  uint8_t* expanded[7];
  for (int l = 0; l <= L; ++l) { lab[l] = NULL; expanded[l] = NULL; }
  for (int l = 0; l <= L && !rc; ++l) {
    size_t n = (size_t)1 << (3 * l);
    lab[l] = (uint32_t*)malloc(n * sizeof(uint32_t));
    expanded[l] = (uint8_t*)calloc(n, 1);
    if (!lab[l] || !expanded[l]) rc = O_ERR_OOM;
  }
  uint32_t i = 0, k = 0, deltas = 0, emitted = 0;
  for (int l = 0; l <= L && !rc; ++l) {
    uint32_t n = 1u << l;
    uint32_t cnt = 1u << (3 * l);
    for (uint32_t m = 0; m < cnt && !rc; ++m) {
      uint32_t c[3];
      demorton3(m, l, c);
      uint32_t pc[3] = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
      size_t ci = lin(c, n);
      if (l > 0 && !expanded[l - 1][lin(pc, n >> 1)]) { /* inherited from a stopped ancestor */
        lab[l][ci] = lab[l - 1][lin(pc, n >> 1)];
        continue;
      }
      if (i >= S) { rc = O_ERR_CORRUPT; break; }
      uint32_t s = sym[i++];
      int op = (int)(s & 7u), stop = (int)(s >> 3);
      uint32_t delta = 0, k_before = k, label = 0;
      if (op == 7 || !((V->op_mask >> op) & 1u)) { rc = O_ERR_CORRUPT; break; }
      if (stop && (l == L || (V->flags & FLAG_NO_STOP))) { rc = O_ERR_CORRUPT; break; }
      switch (op) {
        case OP_PARENT:
          if (l == 0) { rc = O_ERR_CORRUPT; break; }
          label = lab[l - 1][lin(pc, n >> 1)];
          break;
        case OP_NX: case OP_NY: case OP_NZ: {
          int a = op - OP_NX;
          if ((c[a] & 1u) || c[a] == 0) { rc = O_ERR_CORRUPT; break; }
          uint32_t q[3] = {c[0], c[1], c[2]};
          q[a] -= 1;
          label = lab[l][lin(q, n)];
          break;
        }
        case OP_ADV:
          if (k >= n_pal) { rc = O_ERR_CORRUPT; break; }
          label = rd32(pal + 4 * (size_t)k);
          ++k;
          break;
        case OP_LAST:
          if (k < 1) { rc = O_ERR_CORRUPT; break; }
          label = rd32(pal + 4 * (size_t)(k - 1));
          break;
        case OP_DELTA: {
          if (V->flags & FLAG_SHORT_DELTA) { /* one entry holding delta - 1; 2 <= delta <= 16 */
            if (i >= S) { rc = O_ERR_CORRUPT; break; }
            delta = (uint32_t)sym[i++] + 1u;
            if (delta < SHORT_DELTA_MIN) { rc = O_ERR_CORRUPT; break; }
          } else {
            int entries = 0;
            for (;;) {
              if (i >= S || entries == MAX_DELTA_ENTRIES) { rc = O_ERR_CORRUPT; break; }
              uint32_t e = sym[i++];
              ++entries;
              delta = (delta << 3) | (e & 7u);
              if (!(e & 8u)) break;
            }
          }
          if (rc) break;
          ++deltas;
          if (delta < 1 || delta > k) { rc = O_ERR_CORRUPT; break; }
          label = rd32(pal + 4 * (size_t)(k - delta));
          break;
        }
      }
      if (rc) break;
      lab[l][ci] = label;
      expanded[l][ci] = (uint8_t)(l < L && !stop);
      if (nodes && emitted < max_nodes) {
        oracle_node* nd = &nodes[emitted];
        nd->level = l; nd->morton = m; nd->op = op; nd->stop = stop; nd->delta = delta; nd->label = label; nd->k = k_before;
      }
      ++emitted;
    }
  }
  if (!rc && (i != S || k != n_pal || deltas != n_delta)) rc = O_ERR_CORRUPT;
  if (!rc && out) {
    int lo = L - (int)lod;
    uint32_t n = 1u << lo;
    memcpy(out, lab[lo], (size_t)n * n * n * sizeof(uint32_t));
  }
  if (n_nodes_out) *n_nodes_out = emitted;
  for (int l = 0; l <= L; ++l) { free(lab[l]); free(expanded[l]); }
  free(sym);
  return rc;
}

/* Decode brick `id` at level-of-detail `lod` (0 = finest): (b >> lod)^3 labels, x fastest. */
int oracle_decode_brick(const uint8_t* vol, size_t size, uint32_t id, uint32_t lod, uint32_t* out) {
  vol_view V;
  int rc = parse_volume(vol, size, &V);
  if (rc) return rc;
  return replay(&V, id, lod, out, NULL, 0, NULL);
}

/* Emitted nodes of one brick in stream order (tests inspect stop bits, deltas, palette use). */
int oracle_brick_nodes(const uint8_t* vol, size_t size, uint32_t id, oracle_node* nodes, uint32_t max_nodes,
                       uint32_t* n_nodes) {
  vol_view V;
  int rc = parse_volume(vol, size, &V);
  if (rc) return rc;
  return replay(&V, id, 0, NULL, nodes, max_nodes, n_nodes);
}

/* The symbols (4-bit values, one per byte) of one brick after entropy decoding. */
int oracle_brick_symbols(const uint8_t* vol, size_t size, uint32_t id, uint8_t* out, uint32_t cap, uint32_t* S_out) {
  vol_view V;
  int rc = parse_volume(vol, size, &V);
  if (rc) return rc;
  uint8_t* sym = NULL;
  uint32_t S = 0, n_pal = 0, n_delta = 0;
  const uint8_t* pal = NULL;
  rc = brick_symbols(&V, id, &sym, &S, &pal, &n_pal, &n_delta);
  if (rc) return rc;
  *S_out = S;
  if (out) memcpy(out, sym, S < cap ? S : cap);
  free(sym);
  return 0;
}

/* Decode the whole volume at finest resolution, cropping the padding (x fastest). */
int oracle_decode_volume(const uint8_t* vol, size_t size, uint32_t* out) {
  vol_view V;
  int rc = parse_volume(vol, size, &V);
  if (rc) return rc;
  const uint32_t b = 1u << V.L;
  uint32_t nb[3];
  for (int a = 0; a < 3; ++a) nb[a] = (V.dims[a] + b - 1) / b;
  uint32_t* brick = (uint32_t*)malloc((size_t)b * b * b * sizeof(uint32_t));
  if (!brick) return O_ERR_OOM;
  for (uint32_t id = 0; id < V.n_bricks && !rc; ++id) {
    rc = replay(&V, id, 0, brick, NULL, 0, NULL);
    if (rc) break;
    uint32_t bc[3] = {id % nb[0], (id / nb[0]) % nb[1], id / (nb[0] * nb[1])};
    for (uint32_t z = 0; z < b; ++z)
      for (uint32_t y = 0; y < b; ++y)
        for (uint32_t x = 0; x < b; ++x) {
          uint64_t g[3] = {(uint64_t)bc[0] * b + x, (uint64_t)bc[1] * b + y, (uint64_t)bc[2] * b + z};
          if (g[0] >= V.dims[0] || g[1] >= V.dims[1] || g[2] >= V.dims[2]) continue;
          out[(g[2] * V.dims[1] + g[1]) * V.dims[0] + g[0]] = brick[((size_t)z * b + y) * b + x];
        }
  }
  free(brick);
  return rc;
}

/* Assemble a one-brick volume from a caller-made symbol stream and palette (tests build
 * arbitrary legal and illegal streams this way). */
int oracle_pack_single_brick(uint32_t log2b, uint32_t op_mask, uint32_t coder, uint32_t flags, const uint8_t* sym,
                             uint32_t S, const uint32_t* pal, uint32_t n_pal, uint32_t n_delta, uint8_t** out_bytes,
                             size_t* out_size) {
  if (log2b < 1 || log2b > 6 || S == 0) return O_ERR_ARG;
  uint64_t counts[16] = {0};
  for (uint32_t i = 0; i < S; ++i) { if (sym[i] > 15) return O_ERR_ARG; counts[sym[i]]++; }
  uint32_t freq[16] = {0};
  uint32_t ns = 0, cb;
  uint32_t states[8 * RANS_LANES + 8];
  uint16_t* words = NULL;
  if (coder != CODER_RANS && (flags & FLAG_RUNS_MASK)) return O_ERR_ARG;
  if (coder == CODER_RANS) {
    oracle_rans_quantize(counts, freq);
    words = (uint16_t*)malloc(((size_t)S + 1) * sizeof(uint16_t));
    if (!words) return O_ERR_OOM;
    long nw = rans_encode_runs(sym, S, freq, runs_of(flags), states, words);
    if (nw < 0) { free(words); return O_ERR_ARG; }
    cb = (uint32_t)(2 * nw);
    ns = rans_head_words(S, runs_of(flags));
  } else {
    cb = (S + 1) / 2;
  }
  size_t bytes = 16 + 4 * (size_t)ns + 4 * (size_t)n_pal + cb;
  size_t padded = (bytes + 15) & ~(size_t)15;
  size_t rec_off = (O_HEADER_BYTES + 8 + 15) & ~(size_t)15;
  size_t size = rec_off + padded;
  uint8_t* o = (uint8_t*)calloc(size, 1);
  if (!o) { free(words); return O_ERR_OOM; }
  uint32_t b = 1u << log2b;
  wr32(o + 0, O_MAGIC); wr32(o + 4, O_VERSION);
  wr32(o + 8, b); wr32(o + 12, b); wr32(o + 16, b);
  wr32(o + 20, log2b); wr32(o + 24, op_mask); wr32(o + 28, coder); wr32(o + 32, flags);
  wr32(o + 36, 1); wr32(o + 40, n_pal); wr32(o + 44, S);
  for (int s = 0; s < 16; ++s) wr32(o + 48 + 4 * s, freq[s]);
  wr32(o + 112, (uint32_t)(padded / 4));
  wr32(o + O_HEADER_BYTES, 0);
  wr32(o + O_HEADER_BYTES + 4, (uint32_t)(padded / 4));
  uint8_t* r = o + rec_off;
  wr32(r, n_pal); wr32(r + 4, S); wr32(r + 8, cb); wr32(r + 12, n_delta);
  uint8_t* p = r + 16;
  for (uint32_t l = 0; l < ns; ++l, p += 4) wr32(p, states[l]);
  for (uint32_t i = 0; i < n_pal; ++i, p += 4) wr32(p, pal[i]);
  if (coder == CODER_RANS) {
    for (uint32_t w = 0; w < cb / 2; ++w) { p[2 * w] = (uint8_t)words[w]; p[2 * w + 1] = (uint8_t)(words[w] >> 8); }
  } else {
    for (uint32_t i = 0; i < S; ++i) p[i / 2] |= (uint8_t)((sym[i] & 15u) << (4 * (i & 1)));
  }
  free(words);
  *out_bytes = o;
  *out_size = size;
  return 0;
}

/* Assemble a volume of n bricks along x (dims b*n x b x b) from caller-made symbol streams and
 * palettes, concatenated: brick i has S_each[i] symbols, npal_each[i] palette entries and
 * nd_each[i] delta operations. The rANS table is quantised from all bricks' symbols. */
int oracle_pack_bricks(uint32_t log2b, uint32_t op_mask, uint32_t coder, uint32_t flags, uint32_t n,
                       const uint8_t* sym, const uint32_t* S_each, const uint32_t* pal, const uint32_t* npal_each,
                       const uint32_t* nd_each, uint8_t** out_bytes, size_t* out_size) {
  if (log2b < 1 || log2b > 6 || n == 0) return O_ERR_ARG;
  uint64_t counts[16] = {0};
  uint64_t total_sym = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (S_each[i] == 0) return O_ERR_ARG;
    for (uint32_t k = 0; k < S_each[i]; ++k) {
      if (sym[total_sym + k] > 15) return O_ERR_ARG;
      counts[sym[total_sym + k]]++;
    }
    total_sym += S_each[i];
  }
  uint32_t freq[16] = {0};
  if (coder == CODER_RANS) oracle_rans_quantize(counts, freq);
  uint8_t** rec = (uint8_t**)calloc(n, sizeof(uint8_t*));
  uint32_t* rw = (uint32_t*)calloc(n, sizeof(uint32_t));
  if (!rec || !rw) { free(rec); free(rw); return O_ERR_OOM; }
  int rc = 0;
  uint64_t so = 0, po = 0, words_total = 0;
  uint32_t max_pal = 0, max_sym = 0;
  for (uint32_t i = 0; i < n && !rc; ++i) {
    const uint8_t* s = sym + so;
    const uint32_t* p = pal + po;
    uint32_t S = S_each[i], np = npal_each[i];
    uint32_t ns = 0, cb;
    uint32_t states[8 * RANS_LANES + 8];
    uint16_t* words = NULL;
    if (coder != CODER_RANS && (flags & FLAG_RUNS_MASK)) { rc = O_ERR_ARG; break; }
    if (coder == CODER_RANS) {
      words = (uint16_t*)malloc(((size_t)S + 1) * sizeof(uint16_t));
      if (!words) { rc = O_ERR_OOM; break; }
      long nw = rans_encode_runs(s, S, freq, runs_of(flags), states, words);
      if (nw < 0) { free(words); rc = O_ERR_ARG; break; }
      cb = (uint32_t)(2 * nw);
      ns = rans_head_words(S, runs_of(flags));
    } else {
      cb = (S + 1) / 2;
    }
    size_t bytes = 16 + 4 * (size_t)ns + 4 * (size_t)np + cb;
    size_t padded = (bytes + 15) & ~(size_t)15;
    uint8_t* r = (uint8_t*)calloc(padded, 1);
    if (!r) { free(words); rc = O_ERR_OOM; break; }
    wr32(r, np); wr32(r + 4, S); wr32(r + 8, cb); wr32(r + 12, nd_each[i]);
    uint8_t* q = r + 16;
    for (uint32_t l = 0; l < ns; ++l, q += 4) wr32(q, states[l]);
    for (uint32_t k = 0; k < np; ++k, q += 4) wr32(q, p[k]);
    if (coder == CODER_RANS) {
      for (uint32_t w = 0; w < cb / 2; ++w) { q[2 * w] = (uint8_t)words[w]; q[2 * w + 1] = (uint8_t)(words[w] >> 8); }
    } else {
      for (uint32_t k = 0; k < S; ++k) q[k / 2] |= (uint8_t)((s[k] & 15u) << (4 * (k & 1)));
    }
    free(words);
    rec[i] = r;
    rw[i] = (uint32_t)(padded / 4);
    words_total += rw[i];
    if (np > max_pal) max_pal = np;
    if (S > max_sym) max_sym = S;
    so += S;
    po += np;
  }
  if (!rc) {
    size_t rec_off = (O_HEADER_BYTES + 4 * ((size_t)n + 1) + 15) & ~(size_t)15;
    size_t size = rec_off + 4 * (size_t)words_total;
    uint8_t* o = (uint8_t*)calloc(size, 1);
    if (!o) rc = O_ERR_OOM;
    else {
      uint32_t b = 1u << log2b;
      wr32(o + 0, O_MAGIC); wr32(o + 4, O_VERSION);
      wr32(o + 8, b * n); wr32(o + 12, b); wr32(o + 16, b);
      wr32(o + 20, log2b); wr32(o + 24, op_mask); wr32(o + 28, coder); wr32(o + 32, flags);
      wr32(o + 36, n); wr32(o + 40, max_pal); wr32(o + 44, max_sym);
      for (int s = 0; s < 16; ++s) wr32(o + 48 + 4 * s, freq[s]);
      wr32(o + 112, (uint32_t)words_total);
      uint32_t acc = 0;
      for (uint32_t i = 0; i < n; ++i) {
        wr32(o + O_HEADER_BYTES + 4 * (size_t)i, acc);
        memcpy(o + rec_off + 4 * (size_t)acc, rec[i], 4 * (size_t)rw[i]);
        acc += rw[i];
      }
      wr32(o + O_HEADER_BYTES + 4 * (size_t)n, acc);
      *out_bytes = o;
      *out_size = size;
    }
  }
  for (uint32_t i = 0; i < n; ++i) free(rec[i]);
  free(rec); free(rw);
  return rc;
}
