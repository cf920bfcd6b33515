/*
 * vc.h — C ABI of the GB300 brick decoder for CSGV compressed segmentation volumes.
 *
 * The library decodes bricks of a compressed segmentation volume V: N^3 -> N (uint32 labels)
 * that is resident in GPU memory into uint32 label bricks in a caller-owned device cache, in the
 * form Volcanite defines (Methods, "Compressed segmentation volumes"; Results, "CSGV results";
 * Fig. "CSGV" caption; Supplementary Fig. "CSGV ablation" caption): every brick of b^3 voxels is a
 * multi-resolution grid of 2^3 blocks described by a stream of 4-bit operations (copy the parent,
 * copy the x/y/z neighbour that has a different parent, advance / re-read / delta-index the brick's
 * label palette, stop bits for constant subtrees), optionally range-ANS coded.
 *
 * Conventions
 *   - Every call returns a vc_status (0 = VC_OK, negative = error) and never exits or throws.
 *   - Pointers documented as "device" are CUDA device addresses on the volume's device (for
 *     example torch.Tensor.data_ptr()); "host" pointers are ordinary CPU memory.
 *   - Streams are cudaStream_t passed as void*; NULL means the legacy default stream. Calls that
 *     take a stream are asynchronous on it unless documented otherwise.
 *   - The library owns what it allocates (a volume's device copy of the encoding); the caller owns
 *     every buffer it passes in and must keep it alive until the work on the stream completes.
 *   - Decode errors found on the device are reported through a caller-owned status buffer
 *     (VC_STATUS_WORDS int32 words): word 0 = first error code (0 if none; the first writer wins),
 *     word 1 = index of the request item that raised it, words 2..3 = library scratch (the work
 *     counter of the batched decoder, reset by each call). The kernels never trap, and a corrupt
 *     record (any byte of its operation stream, symbol words or states) is reported, never read
 *     or written past the regions its decode uses; its output slot then holds unspecified labels.
 *
 * ------------------------------------------------------------------------------------------
 * Byte format ("VCZ1", all integers little endian). The paper fixes the operations, the
 * unlimited-delta entries and the 32-bit Brick Starts in 32-bit words; the rest is this library's
 * concrete reading of the parts the paper leaves open.
 *
 *   header (128 bytes):
 *     u32 magic = 0x315A4356 ("VCZ1")   u32 version = 1
 *     u32 dims[3] (voxels x, y, z)      u32 log2b (L, 1..6; brick edge b = 2^L)
 *     u32 op_mask (bit o = operation o enabled; bit 4, palette advance, always set)
 *     u32 coder (0 = plain 4-bit, 1 = rANS)   u32 flags (bit 0 = no stop bits were written;
 *                                                        bit 1 = limited delta, see DELTA;
 *                                                        bits 2..3 = log2 K, rANS runs, see rANS)
 *     u32 n_bricks = prod ceil(dims[a] / b)   u32 max_pal   u32 max_sym  (maxima over bricks)
 *     u32 freq[16] (rANS symbol frequencies, sum 4096; zero for plain)
 *     u32 records_words (size of the record area in 32-bit words), 12 reserved bytes
 *   u32 brick_starts[n_bricks + 1]: record offsets in 32-bit words from the record area start;
 *     multiples of 4 (16-byte aligned); brick_starts[n_bricks] = records_words ("Brick Starts",
 *     Methods, "Encoding buffer optimizations": 32-bit word offsets, at most 16 GiB)
 *   zero padding to 16 bytes, then the record area.
 *   Brick (bx, by, bz) has id bx + nbx * (by + nby * bz); voxels beyond the volume repeat the
 *   nearest edge voxel, and callers crop them.
 *
 *   record of one brick (16-byte aligned, zero padded to 16 bytes):
 *     u32 n_pal, u32 n_sym (S), u32 coded_bytes, u32 n_delta (number of delta operations)
 *     [rANS only: u32 state[...] of every run, then u32 run_start[runs - 1] (see rANS)]
 *     u32 palette[n_pal]
 *     u8  coded[coded_bytes]: plain = symbol i in byte i/2, low nibble first;
 *                             rANS  = 16-bit words, see below
 *
 *   symbol stream: levels l = 0 .. L (level l is a (2^l)^3 grid, level L the voxels); inside a
 *   level, the emitted nodes in increasing Morton order of their level coordinates (bit 3i = bit i
 *   of x, 3i+1 of y, 3i+2 of z). The root is emitted; a node of level l+1 is emitted iff its
 *   parent was emitted with stop bit 0. Each emitted node has one symbol op | stop << 3:
 *     0 PARENT   label of the parent (not at level 0)
 *     1/2/3 NX/NY/NZ  label of the same-level cell c - e_axis; legal only when c_axis is even
 *                and > 0, i.e. when that neighbour lies in another parent ("the neighbour that has a
 *                different parent"); a cell that was not emitted holds its nearest emitted
 *                ancestor's label
 *     4 ADV      palette[k], then k += 1 (k = palette entries advanced so far in this brick)
 *     5 LAST     palette[k - 1]
 *     6 DELTA    followed by entries e (1..7 of them): delta = (delta << 3) | (e & 7) while e & 8;
 *                label palette[k - delta], 1 <= delta <= k. With flags bit 1 (limited delta, the
 *                original back reference that stores 1 < delta <= 16 in one 4-bit entry: Results,
 *                "CSGV segmentation volume compression"): exactly one entry, delta = e + 1 with
 *                e >= 1 (so 2 <= delta <= 16; e = 0 is corrupt; a label further back is appended
 *                again)
 *     7          invalid
 *   The stop bit is 0 at level L (and everywhere when flags bit 0 is set). A record is valid iff
 *   every symbol is legal, the stream ends exactly after the last node of level L, k ends at
 *   n_pal and the number of delta operations equals n_delta.
 *
 *   rANS (coder 1): M = 4096, state x in [2^16, 2^32), 32 interleaved states, symbol i uses state
 *   i mod 32. Decoding step t (symbols 32t .. 32t+31): each lane with a symbol takes
 *   slot = x & 4095, s with cum[s] <= slot < cum[s+1], x = freq[s] * (x >> 12) + slot - cum[s];
 *   then, in lane order, every such lane with x < 2^16 shifts in the next 16-bit word. A valid
 *   record reads all words and leaves every used state at 2^16.
 *   Runs (flags bits 2..3 = log2 K, K = 1, 2, 4 or 8; not in the paper, which leaves its coder's
 *   layout to the encoder): the S symbols are cut into runs of Q = 32 ceil(S / 32K) symbols (the
 *   last may be shorter; small records have fewer than K runs), each coded on its own as above
 *   with its own states, so that K warps decode one brick side by side. The record holds the
 *   runs' final states one run after the other (min(run length, 32) each), then the first coded
 *   word of every run but the first; the coded words are the runs' words one run after the other.
 *   Each run must read exactly its words. K = 1 is the record described above. For 64^3 bricks
 *   the symbol chain is ~2,250 rANS steps per brick, and 4 runs cut it to a quarter (about 2 %
 *   more bytes).
 * ------------------------------------------------------------------------------------------
 */
#ifndef VC_H_
#define VC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t vc_status;
#define VC_OK 0
#define VC_ERR_ARG (-1)         /* bad argument (NULL pointer, id out of range, bad mode) */
#define VC_ERR_FORMAT (-2)      /* bytes are not a valid VCZ1 volume (header, offsets) */
#define VC_ERR_OOM (-3)         /* device or host allocation failed */
#define VC_ERR_CUDA (-4)        /* a CUDA call failed */
#define VC_ERR_CORRUPT (-5)     /* a brick's operation stream is invalid (device-side check) */
#define VC_ERR_TIMEOUT (-6)     /* a bounded device wait gave up */
#define VC_ERR_BUSY (-7)        /* resource exhausted for now (serving admission) */
#define VC_ERR_UNSUPPORTED (-8) /* valid volume outside this build's limits */

#define VC_STATUS_WORDS 4

/* Encoding flags (header word 8) */
#define VC_FLAG_NO_STOP 1u
#define VC_FLAG_SHORT_DELTA 2u
#define VC_FLAG_RUNS(k) ((k) >= 8 ? 12u : (k) >= 4 ? 8u : (k) >= 2 ? 4u : 0u) /* k rANS runs per record */

/* decode schedules */
#define VC_MODE_PLAIN 0   /* one kernel launch per brick (the baseline the paper's frame loop replaces) */
#define VC_MODE_GRID 1    /* one launch, one thread block per brick */
#define VC_MODE_BATCHED 2 /* one persistent launch: thread blocks pull bricks from a work counter and
                             prefetch the next brick's record with a bulk copy while decoding */
#define VC_MODE_PIPELINED 3 /* chunks of bricks (vc_schedule.chunk) flow through the rANS symbol kernel
                               and the reconstruction kernel on two library streams, so that one
                               chunk's symbols decode while the previous chunk is reconstructed;
                               the caller's stream waits for both (plain volumes: one launch) */

#define VC_MODE_PALETTED 0x100 /* OR'ed into a mode: cache paletting (Methods, "Cache paletting"): each
                                  slot holds packed palette indices instead of u32 labels, see
                                  vc_volume_slot_words; not with VC_MODE_PIPELINED */

typedef struct vc_volume vc_volume;

typedef struct vc_volume_info {
  uint32_t dims[3];
  uint32_t brick_size;     /* b */
  uint32_t log2b;          /* L */
  uint32_t n_bricks;
  uint32_t bricks_per_axis[3];
  uint32_t op_mask, coder, flags;
  uint32_t max_pal, max_sym, max_delta;
  uint64_t encoded_bytes;  /* bytes passed to vc_load_compressed */
  uint64_t device_bytes;   /* device memory owned by the volume */
  uint32_t smem_bytes;     /* dynamic shared memory per thread block of the decoder (b = 64: the
                              small regions; 0 when all of a brick's regions are in global scratch) */
  uint32_t device;
  uint32_t split;          /* 1: loaded by vc_load_compressed_split */
  uint64_t host_bytes;     /* split volumes: pinned host memory owned by the volume (whole encoding) */
} vc_volume_info;

/* Parses and validates `nbytes` host bytes of a VCZ1 volume (header, Brick Starts, every record's
 * sizes), copies the encoding to device memory that the volume owns (cudaMalloc on `device`) and
 * builds the decoder's per-volume tables (rANS slot table). The copy is enqueued on `cuda_stream`;
 * the call synchronises that stream before returning, so the caller may free `host_bytes` at once.
 * Errors: VC_ERR_ARG (NULL pointer), VC_ERR_FORMAT (invalid bytes), VC_ERR_UNSUPPORTED (a brick
 * of b <= 32 needs more shared memory than a thread block has, or a palette of 65520 entries or
 * more), VC_ERR_OOM, VC_ERR_CUDA. Bricks of b = 64 are decoded with the large parts of their
 * working set (node operations, cursor masks, the 64^3 index grid) in global scratch memory (a
 * few hundred KB per persistent thread block, allocated per decode call) and the rest in shared
 * memory. On error *out is
 * NULL and nothing is leaked. (Paper: the compressed volume is uploaded to GPU memory once and
 * decoded on demand, Methods "Volcanite rendering".) */
vc_status vc_load_compressed(const void* host_bytes, size_t nbytes, int device, void* cuda_stream,
                             vc_volume** out);

/* Detail split (Methods, "Encoding buffer optimizations": the finest level of detail can be kept
 * out of GPU memory and brought in only for bricks needed at full resolution). Same input and
 * errors as vc_load_compressed (VC_ERR_FORMAT also for a record whose symbols do not decode). The
 * device copy holds, per brick, a record of the coarse levels 0 .. L-1 alone (its palette prefix,
 * symbol and delta counts; same coder), so decodes at lod >= 1 read device memory only. The whole
 * encoding is copied to pinned host memory that the volume owns and that is mapped into the
 * device's address space: decodes at lod = 0 read those records over the host link (NVLink-C2C
 * on GB300) with plain loads, with no copy in between (the batched schedule runs as the grid
 * schedule there). device_bytes counts the device copy, host_bytes the pinned host copy. Every
 * other call treats the volume like any other. */
vc_status vc_load_compressed_split(const void* host_bytes, size_t nbytes, int device, void* cuda_stream,
                                   vc_volume** out);

/* Host-only view of the split of one brick (no CUDA calls): out[0] = its symbols S, out[1] = the
 * symbols of levels 0 .. L-1, out[2] = the palette advances and out[3] = the delta operations
 * among those. VC_ERR_ARG / VC_ERR_FORMAT as for loading; VC_ERR_CORRUPT if the stream ends inside
 * the coarse levels or its coded words do not decode. */
vc_status vc_split_counts(const void* host_bytes, size_t nbytes, uint32_t brick_id, uint32_t out[4]);

/* Fills *info. Host only, no CUDA calls. */
vc_status vc_volume_info_get(const vc_volume* vol, vc_volume_info* info);

/* How a volume's bricks are mapped onto the GPU (the autotuner's knobs). Paper: decoding runs in
 * parallel over all requested bricks (Results, "GPU-based rendering pipeline"); the schedule is
 * this library's choice. */
typedef struct vc_schedule {
  uint32_t threads;       /* threads per brick-decoding block: 256, 512 or 1024 (512/1024 for b >= 16) */
  uint32_t stage_depth;   /* 1 = stage the current brick's record only, 2 = prefetch the next one */
  uint32_t blocks_per_sm; /* batched schedule: persistent blocks per SM, 0 = as many as fit */
  uint32_t chunk;         /* pipelined schedule: bricks per chunk, 0 = 512 */
} vc_schedule;

/* Sets the schedule used by later decode calls on this volume (host only; not while a decode of
 * this volume is being enqueued from another thread). VC_ERR_UNSUPPORTED if the combination
 * is not built or its shared memory does not fit; the previous schedule then stays. The default
 * after loading is {256, 1, 0, 512} ({1024, 1, 0, 512} for b = 64). For b = 64 every schedule runs
 * one persistent kernel (blocks_per_sm, 0 = 2, blocks per SM, each with its own global scratch
 * slice); stage_depth and chunk have no effect there. */
vc_status vc_volume_set_schedule(vc_volume* vol, const vc_schedule* sched);
vc_status vc_volume_get_schedule(const vc_volume* vol, vc_schedule* sched);

/* Autotuner: times every schedule this build supports for the volume (threads per brick 256 /
 * 512 / 1024, staging depth 1 / 2, persistent blocks per SM all / 1 / 2, grid and batched) by
 * decoding the given sample (same arguments as vc_decode_bricks; the cache is overwritten) once
 * untimed and `reps` times timed (0 = 3) with CUDA events on `cuda_stream`, then keeps the fastest
 * schedule on the volume. *best and *best_mode receive it, *best_ms (may be NULL) its mean time.
 * Synchronises the stream. Status words accumulate errors of all runs. */
vc_status vc_volume_autotune(vc_volume* vol, const uint32_t* brick_ids, uint32_t n, const uint32_t* cache_slots,
                             uint32_t* cache, uint32_t lod, int32_t* status_dev, void* cuda_stream, uint32_t reps,
                             vc_schedule* best, uint32_t* best_mode, float* best_ms);

/* Size of one cache slot at level of detail lod: *words u32 words. Labels: (b >> lod)^3 words
 * (*bits = 32, *per_word = 1). Paletted (paletted != 0): I = ceil(log2 max_pal) bits per voxel
 * (at least 1), E = floor(32 / I) indices per word, none straddling a word; voxel v (x fastest)
 * is bits [I (v mod E), I (v mod E) + I) of word v / E; its label is the brick's palette entry
 * at that index (the palette stays in the encoding). Host only. */
vc_status vc_volume_slot_words(const vc_volume* vol, uint32_t lod, uint32_t paletted, uint32_t* words,
                               uint32_t* bits, uint32_t* per_word);

/* Decodes n bricks on `cuda_stream` (the Decompress stage: all requested bricks in parallel,
 * Results "GPU-based rendering pipeline"; Methods "GPU rendering pipeline").
 *   brick_ids   device, n x u32: brick ids (< n_bricks); duplicates allowed
 *   cache_slots device, n x u32: destination slot of each brick
 *   cache       device, u32 words; brick i is written to cache + cache_slots[i] * W as W words, W =
 *               (b >> lod)^3 labels x fastest, or with VC_MODE_PALETTED the packed indices of
 *               vc_volume_slot_words; must be 16-byte aligned; caller-owned
 *   lod         level of detail: 0 = finest (b^3 labels), k = level L - k of the brick's hierarchy
 *               (each node the mode of its 2^3 children); 0 <= lod <= L
 *   mode        VC_MODE_PLAIN, VC_MODE_GRID, VC_MODE_BATCHED or VC_MODE_PIPELINED (same output,
 *               optionally | VC_MODE_PALETTED except with the pipelined schedule;
 *               different schedule); the pipelined schedule uses the volume's own streams, so calls
 *               on one volume must not be enqueued from several host threads at once; for b = 64
 *               grid and pipelined run the batched schedule
 *   status_dev  device, VC_STATUS_WORDS int32 (see Conventions); the caller zeroes words 0..1 before
 *               the first call and reads them after synchronising; errors accumulate across calls
 * Returns VC_ERR_ARG for bad host-side arguments and VC_ERR_CUDA if a launch fails; stream-side
 * errors (an id >= n_bricks: VC_ERR_ARG; an invalid record: VC_ERR_CORRUPT) land in status_dev.
 * At lod > 0 only the levels needed are decoded, so corruption in finer levels may go unreported.
 * Requests of 1024 or more items in the grid and batched schedules run longest record first (one
 * small sorting kernel; the result does not depend on the order). n = 0 is a no-op. Calls that
 * overlap on the GPU must not share a status buffer. */
vc_status vc_decode_bricks(vc_volume* vol, const uint32_t* brick_ids, uint32_t n, const uint32_t* cache_slots,
                           uint32_t* cache, uint32_t lod, uint32_t mode, int32_t* status_dev, void* cuda_stream);

/* Same as vc_decode_bricks with host arrays: copies brick_ids (host, n x u32) to the device,
 * decodes brick i into slot i of the volume's own device staging cache and copies the labels back
 * to labels_out (host, n * (b >> lod)^3 u32, brick i at offset i * (b >> lod)^3). Synchronous.
 * *status_out receives the device status word 0. If labels_out is pinned host memory that CUDA
 * maps into the device's address space (cudaHostAlloc, or cudaHostRegister with mapping; 16-byte
 * aligned), the decode kernels write the labels into it directly over the host link (NVLink-C2C
 * on GB300) and no device staging buffer or copy is used; otherwise the labels go through a
 * device staging buffer and one device-to-host copy. The staging buffers are allocated on first
 * use and grow as needed (owned by the volume). */
vc_status vc_decode_bricks_host(vc_volume* vol, const uint32_t* brick_ids, uint32_t n, uint32_t lod,
                                uint32_t mode, uint32_t* labels_out, int32_t* status_out, void* cuda_stream);

/* The coarsest level of detail read straight from the encoding, without decoding (Methods,
 * "Memory management": bricks that do not fit into the cache are accessed in their coarsest level
 * of detail directly from the encoding; "Brick request limitation": an undecoded brick is seen as
 * its most frequent label). The root node of every brick is a palette advance, so the root's
 * label, the top of the brick's mode hierarchy, is its first palette entry: out_labels[i] equals
 * the single label vc_decode_bricks writes for brick_ids[i] at lod = L.
 *   brick_ids   device, n x u32
 *   out_labels  device, n x u32, caller-owned
 *   status_dev  as in vc_decode_bricks: an id >= n_bricks gives VC_ERR_ARG (and label 0) for that
 *               item, an empty palette VC_ERR_CORRUPT; the stream itself is not read or checked
 * One kernel launch on cuda_stream (one thread per item); n = 0 is a no-op. */
vc_status vc_coarsest_labels(vc_volume* vol, const uint32_t* brick_ids, uint32_t n, uint32_t* out_labels,
                             int32_t* status_dev, void* cuda_stream);

/* ---- serving: device brick cache, admission, continuous batching ----
 * Paper (Methods, "GPU rendering pipeline"; Results, "GPU-based rendering pipeline"): bricks are
 * requested, cache space is freed from bricks no longer needed and assigned to new bricks, and
 * all new bricks are decoded in parallel, every frame. A vc_server runs that loop for many
 * clients at once on one device: it owns one device cache buffer, admits requests in arrival
 * order when their missing bricks fit into free plus evictable (unpinned, least recently used
 * first) cache memory, and decodes the missing bricks of all admitted requests in shared batches
 * (one batched-schedule launch per volume and level of detail), up to max_inflight batches on the
 * GPU at a time. Requests that arrive while batches run join the next batch.
 *
 * Cache layout: an 8-ary buddy allocator over the buffer. A block of class c is 4 * 8^c bytes, a
 * (2^c)^3 brick of u32 labels; a brick of edge e = b >> lod takes a block of class
 * max(log2 e, min_class) and its labels (x fastest) start at the block's byte offset, which is a
 * multiple of the block size. A request's bricks stay pinned (never evicted or moved) from its
 * admission until vc_request_release. All calls are thread-safe. */

#define VC_REQ_WAITING 0   /* submitted, not yet admitted (not enough cache memory yet) */
#define VC_REQ_ADMITTED 1  /* cache space assigned, decode pending or running */
#define VC_REQ_DONE 2      /* every brick resident; offsets valid until vc_request_release */
#define VC_REQ_FAILED 3    /* a decode error (status holds its code) or a fatal CUDA error */

typedef struct vc_server vc_server;

#define VC_SERVER_GRAPHS 1u  /* launch each batch as one CUDA graph (captured once per batch slot and
                                shape, then updated in place with the next batch's parameters) */

typedef struct vc_server_config {
  uint64_t cache_bytes;      /* device cache size (rounded down to whole top-class blocks) */
  int32_t device;            /* CUDA device of the server and of every volume added to it */
  uint32_t max_batch_items;  /* bricks per decode batch (0 = 65536) */
  uint32_t max_inflight;     /* batches on the GPU at once, 1..8 (0 = 2) */
  uint32_t min_class;        /* smallest block class (0 = 2, i.e. 256 bytes) */
  uint32_t max_class;        /* largest block class = log2 of the largest brick edge (0 = 6) */
  uint32_t flags;            /* VC_SERVER_GRAPHS */
  uint32_t reserved[2];
} vc_server_config;

typedef struct vc_request_info {
  int32_t state, status;
  uint32_t volume_index, n_bricks, hits; /* hits: bricks already cached or being decoded */
  uint32_t reserved;
  uint64_t bytes;                        /* cache bytes the request pins */
  uint64_t t_submit_ns, t_admit_ns, t_done_ns;  /* host steady clock */
} vc_request_info;

typedef struct vc_server_stats {
  uint64_t cache_bytes, cache_free_bytes, cache_evictable_bytes, cache_entries, evictions;
  uint64_t requests_submitted, requests_admitted, requests_done, requests_failed, requests_waiting;
  uint64_t bricks_hit, bricks_missed, bricks_decoded, batches, batches_inflight, batch_errors;
  uint64_t voxels_decoded;  /* sum of (b >> lod)^3 over decoded bricks */
  uint64_t graph_launches, graph_instantiations;  /* VC_SERVER_GRAPHS: batches launched as graphs,
                                                     graphs instantiated (the rest were updated) */
} vc_server_stats;

/* Creates a server (allocates the cache, batch buffers and streams; starts its thread).
 * VC_ERR_ARG for an invalid configuration, VC_ERR_OOM if the cache does not fit. */
vc_status vc_server_create(const vc_server_config* cfg, vc_server** out);
/* Makes a loaded volume servable under *volume_index. The server does not own the volume: keep
 * it loaded until the server is released. VC_ERR_ARG if it lives on another device,
 * VC_ERR_UNSUPPORTED if its bricks exceed max_class. */
vc_status vc_server_add_volume(vc_server* srv, vc_volume* vol, uint32_t* volume_index);
/* Enqueues a request for n bricks (host arrays: ids, and levels of detail or NULL for all 0);
 * returns at once with its id. VC_ERR_ARG for an id or lod out of range, VC_ERR_BUSY if the
 * request needs more bytes than the whole cache (it could never be admitted). */
vc_status vc_submit_bricks(vc_server* srv, uint32_t volume_index, const uint32_t* brick_ids, const uint32_t* lods,
                           uint32_t n, uint64_t* request_id);
/* Reads a request's state; once VC_REQ_DONE, offsets_out (host, n x u64, may be NULL) receives
 * each brick's byte offset in the cache buffer. Returns the request's error code if it failed. */
vc_status vc_poll(vc_server* srv, uint64_t request_id, int32_t* state, uint64_t* offsets_out);
/* Blocks until the request is done or failed, or timeout_ms passed (VC_ERR_TIMEOUT). */
vc_status vc_wait(vc_server* srv, uint64_t request_id, uint32_t timeout_ms, int32_t* state);
/* The coarsest level of detail of a request's bricks, read straight from the encoding without cache
 * space (Methods, "Memory management": bricks that cannot be held in the cache are accessed in their
 * coarsest level of detail directly from the encoding). For a request that waits for cache space
 * (vc_poll state VC_REQ_WAITING) or whose decode is in flight (VC_REQ_ADMITTED), a client can show
 * these labels until the request is done: labels_dev[i] (device, one u32 per brick of the request,
 * in submission order, caller-owned) receives the single label the brick has at lod = L, as
 * vc_coarsest_labels. status_dev: as in vc_decode_bricks. Any state but a released request;
 * asynchronous on cuda_stream (the brick list is copied before the call returns). */
vc_status vc_request_coarsest(vc_server* srv, uint64_t request_id, uint32_t* labels_dev, int32_t* status_dev,
                              void* cuda_stream);
vc_status vc_request_info_get(vc_server* srv, uint64_t request_id, vc_request_info* info);
/* Unpins a done or failed request's bricks (they become evictable) and forgets the request.
 * VC_ERR_BUSY while it is still waiting or admitted. */
vc_status vc_request_release(vc_server* srv, uint64_t request_id);
/* The cache buffer (device) and its size; read decoded bricks at the offsets vc_poll gives. */
vc_status vc_server_cache(vc_server* srv, void** cache_dev, uint64_t* cache_bytes);
vc_status vc_server_stats_get(vc_server* srv, vc_server_stats* out);

/* ---- camera request stage ----
 * Paper, Methods "GPU rendering pipeline" and Results "Ray marching": rays mark the bricks they
 * pass as visible, bricks with no visible label are skipped, and the level of detail of a brick
 * depends only on its centre, so that one of its voxels covers about one pixel. This library's
 * reading at brick granularity: pixel (px, py) of a W x H pinhole camera shoots the ray
 * pos + t (f + sx r + sy u), f = dir / |dir|, r = f x up / |f x up|, u = r x f,
 * sx = ((px + 1/2) 2/W - 1) tan(fov_y/2) W/H, sy = (1 - (py + 1/2) 2/H) tan(fov_y/2); it walks the
 * brick grid cell by cell (DDA with an integer brick index and a sub-brick position in [0, 1]);
 * every brick whose palette holds a label other than 0 is requested, and the ray ends after the
 * first brick whose palette has no label 0. Level of detail of a requested brick = the largest
 * k <= max_lod with 4^k <= |centre - pos|^2 (2 tan(fov_y/2) / H)^2. Coordinates are voxel units
 * (voxel (x, y, z) spans [x, x+1) x ...). The frame is computed in double precision and rounded to
 * float; every per-ray step is one correctly rounded float operation in a fixed order. */
typedef struct vc_camera {
  float pos[3], dir[3], up[3];
  float fov_y;             /* vertical field of view, radians */
  uint32_t width, height;  /* pixels (width * height < 2^32) */
} vc_camera;

/* Runs the request stage for ncams cameras on `cuda_stream` and waits for it: counts[i] (host)
 * receives the number of bricks camera i requests; brick_ids / lods (host, ncams x cap u32;
 * camera i at i * cap) receive the first min(counts[i], cap) of them in ascending id order with
 * their levels of detail. Device scratch comes from the stream-ordered allocator. */
vc_status vc_camera_bricks(vc_volume* vol, const vc_camera* cams, uint32_t ncams, uint32_t max_lod, uint32_t cap,
                           uint32_t* counts, uint32_t* brick_ids, uint32_t* lods, void* cuda_stream);

/* ---- frame cache: the per-frame cache stages on the device (Methods, "GPU rendering pipeline";
 * Results, "GPU-based rendering pipeline": no GPU to CPU synchronisation within a frame; Methods,
 * "Memory management", "Cache defragmentation") ----
 * A device-resident brick cache of one volume, driven once per frame:
 *   1. marks: the bricks seen this frame set their bit in the cache's visibility marks, by
 *      vc_frame_mark_cameras (the request stage's brick rays) and/or by vc_render with
 *      params->marks = the view's marks (the rays of the renderer, as in the paper);
 *   2. vc_frame_update runs Request (one thread per brick: a cached brick that is not marked, or is
 *      marked at another level of detail, frees its region onto its level's free stack; a marked
 *      brick not cached at its level is pushed onto its level's request stack; the marks are
 *      cleared), Provision (per level, finest first: requests take regions from the free stack,
 *      then from the top of the buffer), Assign (brick -> region, offset, level) and Decode (the
 *      persistent decoder over the assigned bricks of each level), all enqueued on the stream;
 *   3. vc_render reads the view's offsets / lods / cache (an undecoded brick shows its coarsest
 *      label, Methods "Brick request limitation").
 * Level of detail of a marked brick: the request stage's rule for each camera given to the update,
 * the finest over them. A region of level k holds (b / 2^k)^3 labels, starts at a multiple of its
 * size and keeps its level while free. A free stack holds free_stack_entries regions; a region
 * freed onto a full stack stays dead. At most max_bricks_per_frame bricks are assigned per update
 * (the rest stay undecoded and are requested again while they are marked). When the top of the
 * buffer runs out and the space held by free regions of other levels, dead regions and the rest of
 * the buffer would hold what is missing, the next update first empties the cache (defragmentation;
 * never two updates in a row). Calls on one frame cache must not overlap; every call enqueues on
 * the caller's stream and only vc_frame_stats_get waits. */
typedef struct vc_frame_cache vc_frame_cache;
typedef struct vc_frame_cache_view {
  uint64_t* offsets;    /* device, n_bricks: label offset of the brick's region, ~0 = not cached */
  uint8_t* lods;        /* device, n_bricks: its level of detail, 255 = not cached */
  uint32_t* cache;      /* device, cache_words labels */
  uint32_t* marks;      /* device, ceil(n_bricks / 32) words of visibility bits */
  uint64_t cache_words;
  uint32_t n_bricks, max_bricks_per_frame, free_stack_entries;
} vc_frame_cache_view;
typedef struct vc_frame_stats {
  uint64_t frames, bricks_requested, bricks_decoded, voxels_decoded, bricks_freed, bricks_unassigned;
  uint64_t resets, level_switches; /* defragmentations; bricks freed while marked (level changed) */
  uint64_t top_words, dead_words;  /* buffer in use from the bottom; labels in dead regions */
  uint32_t last_resident, last_requested, last_decoded, last_unassigned, last_freed, reset_pending;
  uint32_t free_entries[8];        /* per level of detail */
} vc_frame_stats;
/* Allocates the cache on the volume's device: cache_bytes of labels (>= 4), max_bricks_per_frame
 * (0: min(n_bricks, 262144)) and free_stack_entries per level (0: 1,048,576, the paper's). The
 * decode workspace is sized for max_bricks_per_frame bricks. Released by vc_release. */
vc_status vc_frame_cache_create(vc_volume* vol, uint64_t cache_bytes, uint32_t max_bricks_per_frame,
                                uint32_t free_stack_entries, vc_frame_cache** out);
vc_status vc_frame_cache_view_get(vc_frame_cache* fc, vc_frame_cache_view* out);
/* The request stage's brick rays of ncams cameras set their bricks' marks (any ncams). */
vc_status vc_frame_mark_cameras(vc_frame_cache* fc, const vc_camera* cams, uint32_t ncams, void* cuda_stream);
/* One frame's Request, Provision, Assign and Decode for the marks set since the last update, with
 * levels of detail from cams (1..256 cameras) up to max_lod (clamped to L). status_dev: as in
 * vc_decode_bricks (words 0..1 zeroed by the caller; decode errors land there). */
vc_status vc_frame_update(vc_frame_cache* fc, const vc_camera* cams, uint32_t ncams, uint32_t max_lod,
                          int32_t* status_dev, void* cuda_stream);
/* Waits for the stream and reads the counters. */
vc_status vc_frame_stats_get(vc_frame_cache* fc, vc_frame_stats* out, void* cuda_stream);

/* ---- rendering from decoded bricks (Methods, "Volcanite rendering": "Shading Modes",
 * "Transparency", "Ray marching", "Random number generation"; headless: device buffers) ----
 *
 * One thread per pixel ray of a pinhole camera (the request stage's camera model) marches the
 * voxels of the volume front to back. Voxel positions are an integer voxel index plus a sub-voxel
 * position in [0, 1) per axis (the paper's numerically stable DDA); in a brick decoded at level of
 * detail k the ray steps through the brick's cells of edge 2^k (the paper's LOD DDA: the position
 * is taken to the coarse cell, stepped once, and taken back); a brick whose palette holds no label
 * other than 0 is crossed in one step of edge b; a brick not decoded is seen as one cell holding
 * its coarsest label (its first palette entry, read from the encoding).
 *   Labels map to materials: label 0 is background (empty); label l != 0 has material
 *   materials[hash(l) % n_materials] (rgb albedo in [0, 1], opacity in [0, 1]; opacity 0 = not
 *   shown). Entering a semi-transparent material (0 < opacity < 1) adds its Lambertian local
 *   shading times opacity times the throughput and multiplies the throughput by 1 - opacity; an
 *   opaque material is the surface hit, shaded by the mode:
 *     VC_SHADE_LOCAL   ambient + (1 - ambient) max(0, n . l) (n the entered face's normal)
 *     VC_SHADE_SHADOW  the same with the direct term 0 if a ray towards the light hits an opaque
 *                      voxel before leaving the volume
 *     VC_SHADE_AO      albedo x sky x (0 if a ray in a random cosine-weighted direction around n
 *                      hits an opaque voxel within ao_radius voxels, else 1)
 *     VC_SHADE_PATH    path tracing: Lambertian bounces in random cosine-weighted directions,
 *                      throughput x albedo per bounce, sky radiance when a path leaves the
 *                      volume, Russian roulette from the fourth bounce on, at most max_bounces
 *   Random numbers: PCG2D (Jarzynski and Olano's 2D integer hash) of the pixel and of the frame
 *   index and bounce; random directions by rejection in the unit ball (bounded tries). With
 *   jitter set, the primary ray of frame f goes through a sub-pixel offset drawn from a bell-shaped
 *   approximation of a Blackman-Harris window (temporal anti-aliasing). Every per-ray float step is
 *   one correctly rounded operation in a fixed order, so results are a pure function of the inputs.
 * Inputs (device unless noted): brick_offsets (n_bricks u64: word offset in `cache` of the brick's
 * labels at its level of detail, x fastest, edge b >> brick_lods[i]; UINT64_MAX = not decoded),
 * brick_lods (n_bricks u8), cache (u32 labels), cam and params (host). Outputs (device, W x H, row
 * py at py * W, any may be NULL): labels (first opaque label hit, 0 = none), depth (ray distance
 * in voxels to the entered face of that voxel, +inf = none), face (entered face: 1..6 = -x, +x,
 * -y, +y, -z, +z side of the voxel, 0 = none or the camera inside it), rgb (3 floats per pixel).
 * VC_ERR_ARG for bad sizes or parameters; asynchronous on cuda_stream. */
#define VC_SHADE_LOCAL 0u
#define VC_SHADE_SHADOW 1u
#define VC_SHADE_AO 2u
#define VC_SHADE_PATH 3u
typedef struct vc_material {
  float rgb[3];
  float opacity;
} vc_material;
typedef struct vc_render_params {
  uint32_t mode;         /* VC_SHADE_* */
  uint32_t frame;        /* sample index */
  uint32_t jitter;       /* 1 = temporal anti-aliasing jitter of the primary rays */
  uint32_t max_bounces;  /* path tracing, 1..32 */
  float light_dir[3];    /* towards the light, any length > 0 */
  float ambient;         /* local shading's ambient term, [0, 1] */
  float ao_radius;       /* ambient occlusion reach in voxels, > 0 */
  float sky;             /* environment radiance */
  uint32_t n_materials;  /* 1..256 */
  const vc_material* materials; /* host */
  uint32_t subsample;    /* 0 or 1: every pixel; 2, 4 or 8: one pixel of each s x s block per frame
                            (VC_SUBSET_PIXEL), the others are not written */
  uint32_t* marks;       /* device, ceil(n_bricks / 32) u32, or NULL: visibility marks (Methods, "GPU
                            rendering pipeline": the rays mark the bricks they access). Bit id % 32
                            of word id / 32 is set (atomic OR; never cleared here) for every brick
                            holding a label other than 0 that a ray of path depth <= request_depth
                            enters, decoded or not. The primary ray has depth 0; shadow and ambient
                            occlusion rays and the first path-tracing bounce depth 1; bounce k depth
                            k (Methods, "Brick request limitation": a ray depth limit for requests,
                            1 by default). A vc_frame_cache's marks take them. */
  uint32_t request_depth;
} vc_render_params;
/* Stratified subsets (Methods, "Upsampling": one pixel of each 2^2, 4^2 or 8^2 block is rendered
 * per frame, every pixel of a block within s^2 frames; the blocks' sequences are displaced
 * against each other): pixel (px, py) is rendered in frame f iff
 * (px mod s) + s (py mod s) == (f + h(px / s, py / s)) mod s^2, h a fixed integer hash of the
 * block (white noise standing in for the paper's blue-noise displacement). */
vc_status vc_render(vc_volume* vol, const uint64_t* brick_offsets, const uint8_t* brick_lods, const uint32_t* cache,
                    const vc_camera* cam, const vc_render_params* params, uint32_t* labels_out, float* depth_out,
                    uint8_t* face_out, float* rgb_out, void* cuda_stream);

/* ---- post-processing: accumulation, G-buffer, edge-avoiding À-trous denoising, upsampling
 * (Methods, "Post-processing": "G-Buffer", "Denoising", "Upsampling") ----
 *
 * One call per frame after vc_render, on the pixels that frame rendered (params->subsample and
 * frame as given to vc_render). `state` (device, vc_post_state_bytes(W, H) bytes, caller-owned)
 * keeps, per pixel, the accumulated colour and sample count and the G-buffer of the most recent
 * frame that rendered it: 48 bits, the surface normal (3 bits: axis | (1 if the normal points to
 * -axis) << 2; 3 = no surface hit, 7 = not rendered yet), the depth (13 bits: the hit distance
 * normalised to the dataset's bounding sphere as seen from the camera, 0 .. 8191) and the label
 * (32 bits). reset = 1 clears it (the accumulation restarts, e.g. when the camera moves).
 *   Then `iterations` passes i = 0, 1, ... each combine 3 x 3 pixels q at distance 2^i around p:
 *   c_{i+1}(p) = sum h(q) w(q, p) c_i(q) / sum h(q) w(q, p), h = (1, 2, 1) x (1, 2, 1), w = 0 if
 *   p's and q's normal codes differ, else 1 / (1 + |phi_rho (hsv(albedo_p) - hsv(albedo_q))|^2)
 *   exp(-phi_d |depth_p - depth_q|) with depths in voxels (albedo: the label's material).
 *   A pixel not rendered yet takes no part in the filter; instead the passes find its nearest
 *   rendered pixel (the jump-flood rule o_p <- shortest of o_p and o_q + (q - p)) and it gets
 *   that pixel's filtered colour. The result is tone mapped (x (2.51 x + 0.03) / (x (2.43 x +
 *   0.59) + 0.14), Narkowicz's ACES fit, after scaling by `exposure`), gamma corrected and written
 *   as RGBA8 (x = byte 0 .. alpha = 255 in byte 3) to rgba_out (device, W x H u32).
 * Inputs (device, W x H, as written by vc_render for this frame): labels, depth, face, rgb.
 * params->materials: host, as for vc_render. VC_ERR_ARG for bad sizes or parameters;
 * asynchronous on cuda_stream. */
typedef struct vc_post_params {
  uint32_t width, height;
  uint32_t iterations;          /* 0..10 */
  uint32_t subsample, frame;    /* as given to vc_render for this frame */
  uint32_t reset;               /* 1 = clear the state first */
  float cam_pos[3];             /* the camera position (depth normalisation) */
  float phi_rho, phi_d;         /* edge-stopping weights: albedo (the paper: 8) and depth per voxel */
  float exposure, gamma;        /* tone mapping */
  uint32_t n_materials;
  const vc_material* materials; /* host */
} vc_post_params;
size_t vc_post_state_bytes(uint32_t width, uint32_t height);
vc_status vc_postprocess(vc_volume* vol, const vc_post_params* params, const uint32_t* labels, const float* depth,
                         const uint8_t* face, const float* rgb, void* state, uint32_t* rgba_out, void* cuda_stream);

/* Serving form of the same: runs the request stage for ncams cameras (on the server's own
 * stream; concurrent callers take turns), then submits one request per camera with its bricks
 * and levels of detail, exactly as vc_submit_bricks would; request_ids_out (host, ncams) receives
 * their ids. Returns once the requests are queued (not decoded). */
vc_status vc_request_bricks(vc_server* srv, uint32_t volume_index, const vc_camera* cams, uint32_t ncams,
                            uint32_t max_lod, uint64_t* request_ids_out);

/* Host-only view of the server's cache bookkeeping (no device memory, no CUDA calls): the same
 * buddy allocator, LRU eviction and all-or-nothing admission that a vc_server runs, over an
 * abstract buffer of `bytes` bytes. Keys are opaque 64-bit values; classes as above. */
typedef struct vc_brick_cache vc_brick_cache;
typedef struct vc_brick_cache_stats {
  uint64_t capacity_bytes, free_bytes, evictable_bytes, entries, evictions, hits, misses;
} vc_brick_cache_stats;
/* VC_ERR_ARG unless min_class <= max_class <= 9, bytes holds one max_class block and the number of
 * min_class blocks is at most 2^31. */
vc_status vc_brick_cache_create(uint64_t bytes, uint32_t min_class, uint32_t max_class, vc_brick_cache** out);
/* Pins an entry per key (allocating, evicting least recently used unpinned entries as needed);
 * all or nothing: VC_ERR_BUSY and no pin taken if the keys do not fit. hits_out[i] = 1 if the key
 * was present. Each pin is dropped by one vc_brick_cache_unpin of its entry. */
vc_status vc_brick_cache_acquire(vc_brick_cache* c, const uint64_t* keys, const uint32_t* classes, uint32_t n,
                                 uint32_t* entries_out, uint64_t* offsets_out, uint8_t* hits_out);
vc_status vc_brick_cache_unpin(vc_brick_cache* c, const uint32_t* entries, uint32_t n);
/* Marks an entry invalid (a failed decode): never a hit again, freed with its last pin. */
vc_status vc_brick_cache_invalidate(vc_brick_cache* c, uint32_t entry);
vc_status vc_brick_cache_stats_get(vc_brick_cache* c, vc_brick_cache_stats* out);

/* ---- decode without allocation (the paper has no counterpart) ----
 * For callers that must not allocate device memory while decoding: real-time loops that cannot
 * wait for the allocator (an allocation may block on other streams' frees), processes whose device
 * memory is reserved up front by another allocator and may be exhausted on purpose.
 * vc_decode_bricks allocates the rANS symbol workspace per call
 * (stream-ordered); this entry point uses one statically reserved device array of
 * VC_NOALLOC_WS_BYTES per device instead and allocates nothing (no cudaMalloc, no cudaMallocAsync,
 * no library that allocates).
 *   Same arguments, output and status reporting as vc_decode_bricks, with mode VC_MODE_GRID or
 *   VC_MODE_BATCHED only (VC_ERR_ARG otherwise).
 *   Size limit: for rANS volumes, n x (16 * ceil(ceil(max_sym / 2) / 16) + 16) bytes (rounded up
 *   to 256) must fit in VC_NOALLOC_WS_BYTES, else VC_ERR_ARG and nothing is enqueued; plain-coded
 *   volumes of b <= 32 need no symbol workspace and have no size limit. Requests of 1024 or more
 *   bricks also keep their size-aware order (4 n bytes) in the array when it fits after the
 *   symbols (else they run unordered, with the same result), plain-coded ones included, so they
 *   share the array too. For b = 64 the rest of the array must also hold at least one scratch
 *   slice of the decoder (VC_ERR_ARG otherwise); the persistent grid is cut to the slices that
 *   fit.
 *   Zeroing: the workspace needs none; as for vc_decode_bricks, the caller zeroes status words
 *   0..1 before the first call.
 *   Set-up: the first call on a device (with that device current) looks up the array's device
 *   address once (cudaGetSymbolAddress); make that first call before any stream capture.
 *   Concurrency: all calls on one device share the one workspace, so calls whose work may
 *   overlap on the GPU (other streams, other host threads) race on it and corrupt each other's
 *   output; order them on one stream or with events. */
#define VC_NOALLOC_WS_BYTES (32u << 20)
vc_status vc_decode_bricks_noalloc(vc_volume* vol, const uint32_t* brick_ids, uint32_t n, const uint32_t* cache_slots,
                                   uint32_t* cache, uint32_t lod, uint32_t mode, int32_t* status_dev,
                                   void* cuda_stream);

/* ---- kernel accounting (diagnostics; the paper has no counterpart) ---- */

typedef struct vc_kernel_stats {
  uint64_t launches;       /* kernels this library launched for the volume since the last reset */
  uint32_t timed_calls;    /* grid / batched decode calls timed while profiling was on */
  uint32_t dropped_calls;  /* calls made while profiling was on that found no free event set */
  double symbol_ms;        /* summed device time of the rANS symbol kernel of the timed calls */
  double reconstruct_ms;   /* summed device time of the reconstruction kernel of the timed calls
                              (for the batched schedule this includes the work-counter reset) */
} vc_kernel_stats;

/* enable != 0: later grid and batched decode calls on this volume record CUDA timing events on
 * their stream around the symbol kernel and the reconstruction kernel (up to 4096 calls between
 * resets; the events are the library's). Host only; allocates the events on first use. */
vc_status vc_volume_set_profiling(vc_volume* vol, int enable);

/* Fills *out. Synchronises on the recorded events, so call it after the timed work was enqueued.
 * reset != 0 zeroes the counters and frees the event sets for reuse afterwards. */
vc_status vc_volume_kernel_stats(vc_volume* vol, int reset, vc_kernel_stats* out);

/* Releases a handle returned by this library (a vc_volume, vc_server or vc_brick_cache); NULL is
 * a no-op.
 * A volume: synchronises the device before freeing device memory. A server: stops its thread,
 * waits for its batches on the GPU and frees its cache (pending requests are dropped). */
vc_status vc_release(void* handle);

/* ---- encoder (CPU, multi-threaded; the paper compresses on the CPU with OpenMP, Methods
 * "Compressed segmentation volumes") ---- */

/* Encodes a volume (host, dims[0] * dims[1] * dims[2] uint32 labels, x fastest) into VCZ1 bytes.
 * log2b in 1..6; op_mask as in the format (bit 4 required); coder 0 (plain) or 1 (rANS); flags bit 0
 * = write no stop bits, bit 1 = limited delta (one entry per delta operation, 2 <= delta <= 16),
 * bits 2..3 = log2 of the rANS runs per record (VC_FLAG_RUNS(k); rANS only). Uses `threads` worker
 * threads (0 = all cores). The operation of each node
 * is the first applicable enabled one in the order parent, x, y, z neighbour, last, delta
 * (smallest), advance; coarse nodes hold the mode of their 2^3 children (ties to the smallest
 * label). *out_bytes is allocated by the library; free it with vc_free_bytes. */
vc_status vc_encode_volume(const uint32_t* voxels, const uint32_t dims[3], uint32_t log2b, uint32_t op_mask,
                           uint32_t coder, uint32_t flags, uint32_t threads, uint8_t** out_bytes,
                           size_t* out_size);
/* The same with the rANS frequency table given (freq_in: 16 entries summing to 4096, nonzero for
 * every symbol the volume's streams use; NULL = quantised from the volume's own symbol counts,
 * as vc_encode_volume does). A volume too large to encode at once can so be encoded in z slabs of
 * whole bricks that share one table and whose records are concatenated (Brick Starts offset by
 * the records before each slab). VC_ERR_ARG if the table does not cover a symbol or does not sum
 * to 4096. */
vc_status vc_encode_volume_freq(const uint32_t* voxels, const uint32_t dims[3], uint32_t log2b, uint32_t op_mask,
                                uint32_t coder, uint32_t flags, uint32_t threads, const uint32_t* freq_in,
                                uint8_t** out_bytes, size_t* out_size);
/* Joins VCZ1 volumes stacked in z into one: parts[k] (sizes[k] bytes, host) must share the brick
 * size, operation mask, coder, flags, x / y extent and rANS table, and every part but the last must
 * cover whole bricks in z. The result's bricks are the parts' bricks in order (brick ids of part k
 * follow those of parts 0..k-1, which is the x-fastest id order of the stacked volume), its
 * records the parts' records with Brick Starts offset accordingly. *out_bytes is allocated by the
 * library (vc_free_bytes). VC_ERR_FORMAT for a malformed part, VC_ERR_ARG for parts that do not
 * match. Not in the paper; with vc_encode_volume_freq it encodes volumes too large for one pass,
 * the way the paper's encoder imports large volumes in chunks (Methods, "Compressed segmentation
 * volumes"). */
vc_status vc_concat_volumes_z(const uint8_t* const* parts, const size_t* sizes, uint32_t nparts, uint8_t** out_bytes,
                              size_t* out_size);
void vc_free_bytes(uint8_t* bytes);

/* Human-readable name of a status code (static string). */
const char* vc_status_string(vc_status s);

/* Self-test of the bounded device-side wait that the batched schedule uses for its bulk-copy
 * prefetch (every wait gives up after 1 s of wall-clock time and reports VC_ERR_TIMEOUT instead of
 * hanging): one thread waits, with a budget of budget_us microseconds (1 .. 10^7), on an mbarrier
 * that nothing arrives at and no copy is bound to, then returns. Enqueued on `cuda_stream`;
 * status_dev (device, VC_STATUS_WORDS int32, words 0..1 zeroed by the caller) receives
 * VC_ERR_TIMEOUT in word 0 and the time waited in nanoseconds in words 2 (low) and 3 (high). The
 * context stays usable. */
vc_status vc_selftest_bounded_wait(uint32_t budget_us, int32_t* status_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* VC_H_ */
