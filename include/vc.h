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
 *     counter of the batched decoder, reset by each call). The kernels never trap.
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
 *     u32 coder (0 = plain 4-bit, 1 = rANS)   u32 flags (bit 0 = no stop bits were written)
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
 *     [rANS only: u32 state[min(S, 32)]]
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
 *                label palette[k - delta], 1 <= delta <= k
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

/* decode schedules */
#define VC_MODE_PLAIN 0   /* one kernel launch per brick (the baseline the paper's frame loop replaces) */
#define VC_MODE_GRID 1    /* one launch, one thread block per brick */
#define VC_MODE_BATCHED 2 /* one persistent launch: thread blocks pull bricks from a work counter and
                             prefetch the next brick's record with a bulk copy while decoding */
#define VC_MODE_PIPELINED 3 /* chunks of bricks flow through three kernels on three library streams:
                               rANS symbols, reconstruction (finest index grids to a workspace), and
                               output expansion; the caller's stream waits for all of them */

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
  uint32_t smem_bytes;     /* dynamic shared memory per thread block of the decoder */
  uint32_t device;
} vc_volume_info;

/* Parses and validates `nbytes` host bytes of a VCZ1 volume (header, Brick Starts, every record's
 * sizes), copies the encoding to device memory that the volume owns (cudaMalloc on `device`) and
 * builds the decoder's per-volume tables (rANS slot table). The copy is enqueued on `cuda_stream`;
 * the call synchronises that stream before returning, so the caller may free `host_bytes` at once.
 * Errors: VC_ERR_ARG (NULL pointer), VC_ERR_FORMAT (invalid bytes), VC_ERR_UNSUPPORTED (a brick
 * needs more shared memory than a thread block has), VC_ERR_OOM, VC_ERR_CUDA. On error *out is
 * NULL and nothing is leaked. (Paper: the compressed volume is uploaded to GPU memory once and
 * decoded on demand, Methods "Volcanite rendering".) */
vc_status vc_load_compressed(const void* host_bytes, size_t nbytes, int device, void* cuda_stream,
                             vc_volume** out);

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
 * after loading is {256, 1, 0, 512}. */
vc_status vc_volume_set_schedule(vc_volume* vol, const vc_schedule* sched);
vc_status vc_volume_get_schedule(const vc_volume* vol, vc_schedule* sched);

/* Decodes n bricks on `cuda_stream` (the Decompress stage: all requested bricks in parallel,
 * Results "GPU-based rendering pipeline"; Methods "GPU rendering pipeline").
 *   brick_ids   device, n x u32: brick ids (< n_bricks); duplicates allowed
 *   cache_slots device, n x u32: destination slot of each brick
 *   cache       device, u32 labels; brick i is written to cache + cache_slots[i] * (b >> lod)^3 as
 *               (b >> lod)^3 labels, x fastest; must be 16-byte aligned; caller-owned
 *   lod         level of detail: 0 = finest (b^3 labels), k = level L - k of the brick's hierarchy
 *               (each node the mode of its 2^3 children); 0 <= lod <= L
 *   mode        VC_MODE_PLAIN, VC_MODE_GRID, VC_MODE_BATCHED or VC_MODE_PIPELINED (same output,
 *               different schedule); the pipelined schedule uses the volume's own streams, so calls
 *               on one volume must not be enqueued from several host threads at once
 *   status_dev  device, VC_STATUS_WORDS int32 (see Conventions); the caller zeroes words 0..1 before
 *               the first call and reads them after synchronising; errors accumulate across calls
 * Returns VC_ERR_ARG for bad host-side arguments and VC_ERR_CUDA if a launch fails; stream-side
 * errors (an id >= n_bricks: VC_ERR_ARG; an invalid record: VC_ERR_CORRUPT) land in status_dev.
 * At lod > 0 only the levels needed are decoded, so corruption in finer levels may go unreported.
 * n = 0 is a no-op. Calls that overlap on the GPU must not share a status buffer. */
vc_status vc_decode_bricks(vc_volume* vol, const uint32_t* brick_ids, uint32_t n, const uint32_t* cache_slots,
                           uint32_t* cache, uint32_t lod, uint32_t mode, int32_t* status_dev, void* cuda_stream);

/* Same as vc_decode_bricks with host arrays: copies brick_ids (host, n x u32) to the device,
 * decodes brick i into slot i of the volume's own device staging cache and copies the labels back
 * to labels_out (host, n * (b >> lod)^3 u32, brick i at offset i * (b >> lod)^3). Synchronous.
 * *status_out receives the device status word 0. Host buffers are best pinned. The staging
 * buffers are allocated on first use and grow as needed (owned by the volume). */
vc_status vc_decode_bricks_host(vc_volume* vol, const uint32_t* brick_ids, uint32_t n, uint32_t lod,
                                uint32_t mode, uint32_t* labels_out, int32_t* status_out, void* cuda_stream);

/* ---- decode without allocation (the paper has no counterpart) ----
 * For callers that must not allocate device memory while decoding: code that runs inside CUDA
 * stream capture, real-time loops that cannot wait for the allocator, processes whose device
 * memory is reserved up front. vc_decode_bricks allocates the rANS symbol workspace per call
 * (stream-ordered); this entry point uses one statically reserved device array of
 * VC_NOALLOC_WS_BYTES per device instead and allocates nothing (no cudaMalloc, no cudaMallocAsync,
 * no library that allocates).
 *   Same arguments, output and status reporting as vc_decode_bricks, with mode VC_MODE_GRID or
 *   VC_MODE_BATCHED only (VC_ERR_ARG otherwise).
 *   Size limit: for rANS volumes, n x (16 * ceil(ceil(max_sym / 2) / 16) + 16) bytes must fit in
 *   VC_NOALLOC_WS_BYTES, else VC_ERR_ARG and nothing is enqueued; plain-coded volumes use no
 *   workspace and have no limit.
 *   Zeroing: the workspace needs none; as for vc_decode_bricks, the caller zeroes status words
 *   0..1 before the first call.
 *   Set-up: the first call on a device (with that device current) looks up the array's device
 *   address once; make that first call outside any stream capture.
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
 * their stream around the symbol kernel and the reconstruction kernel (up to 256 calls between
 * resets; the events are the library's). Host only; allocates the events on first use. */
vc_status vc_volume_set_profiling(vc_volume* vol, int enable);

/* Fills *out. Synchronises on the recorded events, so call it after the timed work was enqueued.
 * reset != 0 zeroes the counters and frees the event sets for reuse afterwards. */
vc_status vc_volume_kernel_stats(vc_volume* vol, int reset, vc_kernel_stats* out);

/* Releases a handle returned by this library (a vc_volume); NULL is a no-op. Synchronises the
 * device before freeing device memory. */
vc_status vc_release(void* handle);

/* ---- encoder (CPU, multi-threaded; the paper compresses on the CPU with OpenMP, Methods
 * "Compressed segmentation volumes") ---- */

/* Encodes a volume (host, dims[0] * dims[1] * dims[2] uint32 labels, x fastest) into VCZ1 bytes.
 * log2b in 1..6; op_mask as in the format (bit 4 required); coder 0 (plain) or 1 (rANS); flags bit 0
 * = write no stop bits. Uses `threads` worker threads (0 = all cores). The operation of each node
 * is the first applicable enabled one in the order parent, x, y, z neighbour, last, delta
 * (smallest), advance; coarse nodes hold the mode of their 2^3 children (ties to the smallest
 * label). *out_bytes is allocated by the library; free it with vc_free_bytes. */
vc_status vc_encode_volume(const uint32_t* voxels, const uint32_t dims[3], uint32_t log2b, uint32_t op_mask,
                           uint32_t coder, uint32_t flags, uint32_t threads, uint8_t** out_bytes,
                           size_t* out_size);
void vc_free_bytes(uint8_t* bytes);

/* Human-readable name of a status code (static string). */
const char* vc_status_string(vc_status s);

#ifdef __cplusplus
}
#endif

#endif /* VC_H_ */
