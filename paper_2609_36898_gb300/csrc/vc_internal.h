// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "vc.h"

namespace vc {

constexpr uint32_t kMagic = 0x315A4356u;  // "VCZ1"
constexpr uint32_t kVersion = 1u;
constexpr uint32_t kHeaderBytes = 128u;
constexpr uint32_t kRansLanes = 32u;
constexpr uint32_t kRansM = 4096u;
constexpr uint32_t kThreads = 256u;       // threads per decoder thread block
constexpr uint32_t kMaxIdx16 = 0xFFF0u;   // palette indices live in 16-bit grids; above: pending marks
constexpr uint32_t kFlagNoStop = 1u;
constexpr uint32_t kHandleVolume = 0x564F4C31u;  // "VOL1"

// Byte offsets of the decoder's shared-memory regions (one brick in flight per thread block).
struct SmemLayout {
  uint32_t stage_off;    // staged record, two buffers of stage_bytes (prefetch in batched mode)
  uint32_t stage_bytes;  // 0 = records are read from global memory
  uint32_t nib_off;      // rANS: decoded symbols, two per byte (low nibble first)
  uint32_t op_off;       // delta bricks: one operation symbol per node (bytes)
  uint32_t mask_off;     // adv_mask, del_mask, adv_pre, del_pre: 4 x nwords u32
  uint32_t nwords;
  uint32_t dlist_off;    // delta values of the brick's delta operations
  uint32_t grid_off;     // G (u16 palette index) then R (u16 rank) for levels 0..L-1
  uint32_t ncells;
  uint32_t chunk_off;    // per-32-cell masks and prefixes of the level being built
  uint32_t nchunks;
  uint32_t parse_off;    // per-thread summaries of the delta-entry parse
  uint32_t rans_off;     // slot -> symbol table (4096 B) + freq[16] + cum[17]
  uint32_t misc_off;     // scalars: error flag, item numbers, counters, mbarriers
  uint32_t total;
};

// Device-side description of a loaded volume, passed by value to the kernels.
struct DevVolume {
  const uint32_t* records;  // record area (32-bit words)
  const uint32_t* starts;   // n_bricks + 1 word offsets
  const uint8_t* rans_sym;  // 4096 slot -> symbol
  const uint32_t* rans_fc;  // freq[16], cum[17]
  uint32_t n_bricks;
  uint32_t L;
  uint32_t op_mask;
  uint32_t coder;
  uint32_t flags;
  SmemLayout sm;
};

struct Volume {
  uint32_t kind;  // kHandleVolume
  int device;
  uint32_t dims[3];
  uint32_t L, op_mask, coder, flags, n_bricks, nb[3];
  uint32_t max_pal, max_sym, max_delta, max_rec_words;
  uint64_t encoded_bytes, device_bytes;
  uint8_t* d_file;       // device copy of the whole file
  uint8_t* d_tables;     // rANS tables
  DevVolume dv;
  // staging for vc_decode_bricks_host
  uint32_t* d_host_ids;
  uint32_t* d_host_slots;
  uint32_t* d_host_cache;
  int32_t* d_host_status;
  size_t host_cap_items, host_cap_words;
};

// decode.cu
vc_status compute_layout(uint32_t L, uint32_t coder, uint32_t max_sym, uint32_t max_pal, uint32_t max_delta,
                         uint32_t max_rec_words, int device, SmemLayout* out);
vc_status launch_decode(const Volume& v, const uint32_t* ids, uint32_t n, const uint32_t* slots, uint32_t* cache,
                        uint32_t lod, uint32_t mode, int32_t* status, cudaStream_t stream);

}  // namespace vc
