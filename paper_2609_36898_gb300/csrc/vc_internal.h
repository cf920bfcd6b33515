// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "vc.h"

namespace vc {

constexpr uint32_t kMagic = 0x315A4356u;  // "VCZ1"
constexpr uint32_t kVersion = 1u;
constexpr uint32_t kHeaderBytes = 128u;
constexpr uint32_t kRansLanes = 32u;
constexpr uint32_t kRansM = 4096u;
constexpr uint32_t kMaxIdx8 = 0xFCu;      // palette indices below this fit 8-bit grids (marks above)
constexpr uint32_t kMaxIdx16 = 0xFFF0u;   // same for 16-bit grids
constexpr uint32_t kFlagNoStop = 1u;
constexpr uint32_t kFlagShortDelta = 2u;  // a delta operation carries one 4-bit entry: delta - 1
// rANS runs (flags bits 2..3 = log2 K; rANS volumes only): a record's S symbols are cut into runs
// of Q = 32 ceil(S / 32K) symbols (the last may be shorter; small records have fewer runs), each
// coded on its own with 32 interleaved states, so that K warps can decode one brick side by side.
// Between the record's header and its palette: every run's final states (32 for every run but
// the last, min(last, 32) for it), then the first coded word of runs 1 .. n-1 (u32 each).
constexpr uint32_t kFlagRunsShift = 2u;
constexpr uint32_t kFlagRunsMask = 3u << kFlagRunsShift;
__host__ __device__ inline uint32_t runs_k(uint32_t flags) { return 1u << ((flags & kFlagRunsMask) >> kFlagRunsShift); }
// (K is a power of two: shifts, no division)
__host__ __device__ inline uint32_t run_q(uint32_t S, uint32_t K) {
  const uint32_t lk = K >= 8u ? 3u : K >= 4u ? 2u : K >= 2u ? 1u : 0u;
  const uint32_t per = (S + (32u << lk) - 1u) >> (5u + lk);
  return 32u * (per ? per : 1u);
}
__host__ __device__ inline uint32_t run_n(uint32_t S, uint32_t K) {
  const uint32_t q = run_q(S, K);
  uint32_t n = 1;
  for (uint32_t k = 1; k < K; ++k) n += S > k * q ? 1u : 0u;
  return n;
}
// Words between a rANS record's header and its palette (states, then run starts).
__host__ __device__ inline uint32_t head_words(uint32_t S, uint32_t K) {
  if (K == 1u) return S < 32u ? S : 32u;
  const uint32_t n = run_n(S, K), last = S - (n - 1u) * run_q(S, K);
  return 33u * (n - 1u) + (last < 32u ? last : 32u);
}
constexpr uint32_t kHandleVolume = 0x564F4C31u;  // "VOL1"
constexpr uint32_t kHandleServer = 0x53525631u;  // "SRV1"
constexpr uint32_t kHandleCache = 0x43484331u;   // "CHC1"
constexpr uint32_t kRansWarps = 16u;      // bricks (warps) per block of the rANS symbol kernel
constexpr uint32_t kRing = 3u;            // pipelined schedule: workspace slots (chunks in flight)
// From this level of detail on, the rANS symbol kernel decodes only a record's prefix up to the
// level needed (levels 0 .. L - lod) and the reconstruction parses that prefix (level 0 needs the
// whole stream). At level 1 the prefix is still about a quarter of a whole record and the gain is
// a few percent (32^3 bricks of the 512^3 workload: 0.258 -> 0.246 ms for 4096 bricks). The coarse
// records of a detail split hold levels 0 .. L - 1 only: level 1 needs them whole, so their
// prefix decode starts at level 2.
constexpr uint32_t kPrefixMinLod = 1;
// SmemLayout::big_sm: large regions of a b = 64 layout placed in shared memory
constexpr uint32_t kBigNodes = 1u, kBigDelta = 2u, kBigMasks = 4u, kBigFg = 8u, kBigQueues = 16u;
constexpr uint32_t kPrefixMinLodSplit = 2;

// Byte offsets of the reconstruction kernel's shared-memory regions (one brick per block).
struct SmemLayout {
  uint32_t misc_off;     // error flag, items, counters, mbarriers, warp totals, scan scratch
  uint32_t stage_off;    // staged record (plain) or record head + decoded symbols (rANS)
  uint32_t stage_alias;  // 1: the (single) stage lies over the masks .. rank lists span, which a
                         // brick fills only after its parse and no longer reads once its finest
                         // level is decoded (the next brick's copy then lands there)
  uint32_t stage_bytes;  // per buffer; 0 = read from global memory
  uint32_t nstage;       // 1 or 2 buffers (2 = prefetch the next brick in the batched kernel)
  uint32_t nodes_off;    // node-indexed operation symbols, 8 per u32 (delta bricks only)
  uint32_t nodes_words;
  uint32_t mask_off;     // adv_mask, del_mask (nwords u32 each), adv_pre, del_pre (nwords u16 each; u32 for b = 64)
  uint32_t nwords;
  uint32_t dlist_off;    // delta values of the brick's delta operations
  uint32_t dlist_cap;
  uint32_t g_off;        // palette index per cell of levels 0..L-1 (gt_bytes each)
  uint32_t ns_off;       // per level, one byte per parent cell: which children have stop bit 0
                         // (each level's bytes start 4-byte aligned, so that the level's open
                         // cells read as a bit array of u32 words in Morton order)
  uint32_t rank_off;     // u16 per 32 cells of level L-1: rank of the first open cell among them
  uint32_t pq_off;       // label output, 8-bit grids: ranks of the open cells whose children read the
  uint32_t pq_cap;       // palette (u16 each, over the rank list of level L-2; pq_cap entries)
  uint32_t mq_off;       // label output: one 224-byte queue of neighbour marks per warp (over the
                         // node operations .. cursor masks span, dead by then, or its own region)
  uint32_t fg_off;       // finest level: palette index per voxel (gt_bytes each; one z half for b = 32),
                         // or (label output) the 8 children of each open level-(L-1) cell by rank
  uint32_t plane_off;    // b = 32: the last z plane of the first half (for -z neighbours of the second)
  uint32_t fg_bytes;     // bytes of the finest grid region
  uint32_t wst_off;      // the parse's per-word automaton masks (the finest grid's region)
  uint32_t wst_bytes;
  uint32_t list_off;     // stop-0 cells by rank (u16), two buffers: even / odd levels
  uint32_t list0_cap;    // entries of the even-level buffer
  uint32_t list1_cap;    // entries of the odd-level buffer
  uint32_t pal_off;      // private copy of the brick's palette
  uint32_t pal_cap;      // entries it can hold (0 = palettes are read from the stage); byte grids: a
                         // power of two >= max_pal, zero padded (indices are masked with pal_cap - 1)
  uint32_t gt_bytes;     // 1 (max_pal < 252) or 2
  uint32_t total;
  uint32_t gscratch;     // 0: the regions are in shared memory; else b = 64: they are in a global
                         // scratch slice of this many bytes per thread block (no shared memory)
  uint32_t big_sm;       // b = 64 with a scratch slice: the large regions in shared memory instead
                         // (kBig* bits; the others are in the slice)
  // rANS symbol kernel
  uint32_t ws_stride;    // bytes of decoded symbols per request item (workspace)
  uint32_t a_buf;        // per-warp coded-word buffer bytes
  uint32_t a_smem;       // dynamic shared memory per block
};

// Device-side description of a loaded volume, passed by value to the kernels.
struct DevVolume {
  const uint32_t* records;   // record area (32-bit words)
  const uint32_t* starts;    // n_bricks + 1 word offsets
  const uint32_t* rans_tab;  // 4096 entries: freq | (slot - cum) << 13 | symbol << 25
  uint32_t n_bricks;
  uint32_t L;
  uint32_t op_mask;
  uint32_t coder;
  uint32_t flags;
  uint32_t prefix_lod;  // first level of detail decoded from a record prefix (kPrefixMinLod[Split])
  SmemLayout sm;
};

struct Volume {
  uint32_t kind;  // kHandleVolume
  int device;
  uint32_t dims[3];
  uint32_t L, op_mask, coder, flags, n_bricks, nb[3];
  uint32_t sms;          // multiprocessors of the device
  uint32_t max_pal, max_sym, max_delta, max_rec_words, max_stage;
  uint32_t max_nodes;    // max over bricks of S - n_delta (every delta operation has an entry): bounds nodes
  uint64_t encoded_bytes, device_bytes;
  vc_schedule sched;     // threads per block, staging depth, persistent blocks per SM, chunk
  cudaStream_t aux[2];   // pipelined schedule: symbol and reconstruction streams
  cudaEvent_t ev_fork, ev_join[2], ev_a[kRing], ev_f[kRing];
  uint8_t* d_file;       // device copy of the whole file (+ slack)
  uint8_t* d_tables;     // rANS table
  uint8_t* d_flags;      // per brick: bit 0 = palette holds label 0, bit 1 = holds another label
  DevVolume dv;          // dv.sm: the layout for label output
  SmemLayout sm_pal;     // the layout for packed palette indices (differs for b = 64)
  // staging for vc_decode_bricks_host
  uint32_t* d_host_ids;
  uint32_t* d_host_slots;
  uint32_t* d_host_cache;
  int32_t* d_host_status;
  uint32_t* h_rec_words;  // host copy: record size of each brick in 32-bit words (work ordering)
  // detail split (vc_load_compressed_split): the device copy holds the coarse levels only; the
  // whole encoding lives in pinned host memory mapped into the device's address space, read by
  // finest-level decodes
  bool split;
  uint8_t* h_full;
  const uint32_t* full_records;  // device addresses of the mapped host copy
  const uint32_t* full_starts;
  uint64_t host_bytes;
  size_t host_cap_items, host_cap_words;
  // kernel accounting: launches are always counted; with prof set, each grid / batched decode call
  // records three timing events (before the symbol kernel, between, after the reconstruction)
  uint64_t launches;
  bool prof;
  cudaEvent_t* prof_ev;    // kProfCalls x 3
  uint32_t prof_used;      // calls recorded since the last reset
  uint32_t prof_dropped;   // calls not recorded (ring full)
};

constexpr uint32_t kProfCalls = 4096;

// server.cpp: releases a vc_server (false if the handle is not one)
bool release_server(void* handle);
// cache.cpp: releases a vc_brick_cache (false if the handle is not one)
bool release_cache(void* handle);
// frame.cu: releases a vc_frame_cache (false if the handle is not one)
bool release_frame(void* handle);

// request.cu: a pinhole camera's frame (forward, right, up), pixel scales and level-of-detail
// scale, computed in double precision and rounded to float once (shared by the request stage and
// the renderer): the ray of pixel (px, py) is o + t (f + sx r + sy u), sx = ((px + 1/2) inv_w2 - 1)
// sxs, sy = (1 - (py + 1/2) inv_h2) sys
struct CamDev {
  float o[3], f[3], r[3], u[3];
  float sxs, sys, inv_w2, inv_h2, lod_s2;
  uint32_t W, H;
};
void camera_frame(const vc_camera& c, CamDev* d);
// Stratified subsets of vc_render / vc_postprocess: is pixel (px, py) rendered in frame f when one
// pixel of each s x s block is? (the block's pixel of frame f: (f + h(block)) mod s^2, h a fixed
// integer hash)
__host__ __device__ inline bool subset_pixel(uint32_t px, uint32_t py, uint32_t s, uint32_t f) {
  if (s <= 1u) return true;
  uint32_t h = (px / s) * 0x8DA6B343u ^ (py / s) * 0xD8163841u;
  h ^= h >> 13;
  h *= 0x85EBCA6Bu;
  h ^= h >> 16;
  return (px % s) + s * (py % s) == (f + h) % (s * s);
}

// request.cu: the camera request stage (rays -> visible bricks and their levels of detail)
size_t camera_scratch_bytes(const Volume& v, uint32_t ncams);
constexpr size_t kCamDevBytes = 76;  // per camera, pinned host staging
vc_status launch_camera_requests(const Volume& v, const vc_camera* cams, uint32_t ncams, uint32_t max_lod,
                                 uint32_t cap, uint8_t* d_scratch, void* h_cams_pinned, uint32_t* d_counts,
                                 uint32_t* d_ids, uint32_t* d_lods, cudaStream_t stream);

// request.cu: the brick rays of ncams cameras (any number; launched in groups) mark the visible
// bricks they pass in one shared bitmask (device, one bit per brick; bits are only set)
vc_status launch_shared_marks(const Volume& v, const vc_camera* cams, uint32_t ncams, uint32_t* marks,
                              cudaStream_t stream);

// vc_api.cu: the host-side checks of a VCZ1 file (header, Brick Starts, every record's sizes) and
// the maxima the decoder's layouts are sized by
struct VolumeScan {
  uint32_t dims[3], nb[3], L, op_mask, coder, flags, n_bricks, freq[16], records_words;
  size_t rec_off;  // byte offset of the record area
  uint32_t max_pal, max_sym, max_delta, max_words, max_stage, max_nodes;
  std::vector<uint8_t> bflags;  // per brick: bit 0 = palette holds label 0, bit 1 = another label
};
vc_status scan_volume(const uint8_t* p, size_t nbytes, VolumeScan* out);

// encode.cpp: 32-way interleaved rANS of S symbols with the volume's table (states of the first
// min(S, 32) lanes, words in the decoder's read order)
void rans_encode(const uint8_t* sym, uint32_t S, const uint32_t f[16], const uint32_t cum[17],
                 std::vector<uint16_t>& words, uint32_t states[32], uint32_t* n_states);

// decode.cu
// cache paletting: bits per palette index (ceil(log2 max_pal), >= 1) and indices per u32 word
void palette_packing(uint32_t max_pal, uint32_t* bits, uint32_t* per_word);
bool schedule_supported(uint32_t L, uint32_t threads);
// paletted: the layout for packed palette indices (b = 64: the finest level needs the voxel index
// grid, so the large regions stay in a global scratch slice); else for labels.
vc_status compute_layout(const Volume& v, int device, uint32_t threads, uint32_t nstage, SmemLayout* out,
                         bool paletted = false);
// presorted: the items are already in the order they should run (else requests of 1024 items or
// more in the grid / batched schedules run longest record first)
vc_status launch_decode(Volume& v, const uint32_t* ids, uint32_t n, const uint32_t* slots, uint32_t* cache,
                        uint32_t lod, uint32_t mode, int32_t* status, cudaStream_t stream, bool presorted = false);
// The coarsest level of detail (first palette entry) of n bricks, one launch on stream.
vc_status launch_coarsest(Volume& v, const uint32_t* ids, uint32_t n, uint32_t* out, int32_t* status,
                          cudaStream_t stream);
// Workspace bytes a decode of n items may use (rANS symbols, then b = 64 scratch slices); 0 if none.
size_t decode_ws_bytes(const Volume& v, uint32_t n);
// Same as launch_decode, with the workspace supplied by the caller (ws_ext, ws_cap bytes, 256-byte
// aligned) instead of allocated: VC_ERR_ARG if the rANS symbols of n items (plus one scratch slice
// for b = 64) need more than ws_cap or mode is pipelined. For b = 64 the persistent grid shrinks to
// the scratch slices that fit.
vc_status launch_decode_ws(Volume& v, const uint32_t* ids, uint32_t n, const uint32_t* slots, uint32_t* cache,
                           uint32_t lod, uint32_t mode, int32_t* status, cudaStream_t stream, uint8_t* ws_ext,
                           size_t ws_cap, bool presorted = false);

// Persistent decode of min(cap, *n_dev) items, the count read on the device (n_dev: device
// memory written earlier on the stream); ws: decode_ws_bytes(v, cap) bytes, 256-byte aligned.
// Labels only (no paletting); VC_ERR_UNSUPPORTED for the finest level of a split volume.
vc_status launch_decode_devcount(Volume& v, const uint32_t* ids, uint32_t cap, const uint32_t* n_dev,
                                 const uint32_t* slots, uint32_t* cache, uint32_t lod, int32_t* status,
                                 cudaStream_t stream, uint8_t* ws, size_t ws_cap);

// A one-thread kernel waits (bounded, budget_us) on an mbarrier nothing arrives at and reports
// VC_ERR_TIMEOUT to status[0], the elapsed nanoseconds to status[2..3].
vc_status launch_wait_selftest(uint32_t budget_us, int32_t* status, cudaStream_t stream);

}  // namespace vc
