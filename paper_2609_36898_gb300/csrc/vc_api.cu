// Host side of the C ABI: volume loading and validation, decode dispatch, release.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "vc_internal.h"

using namespace vc;

namespace {

inline uint32_t le32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
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

void destroy_pipeline(Volume* v) {
  for (int i = 0; i < 2; ++i) {
    if (v->aux[i]) cudaStreamDestroy(v->aux[i]);
    if (v->ev_join[i]) cudaEventDestroy(v->ev_join[i]);
  }
  if (v->ev_fork) cudaEventDestroy(v->ev_fork);
  for (uint32_t i = 0; i < kRing; ++i) {
    if (v->ev_a[i]) cudaEventDestroy(v->ev_a[i]);
    if (v->ev_f[i]) cudaEventDestroy(v->ev_f[i]);
  }
}

bool create_pipeline(Volume* v) {
  bool ok = true;
  for (int i = 0; i < 2; ++i) {
    ok = ok && cudaStreamCreateWithFlags(&v->aux[i], cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&v->ev_join[i], cudaEventDisableTiming) == cudaSuccess;
  }
  ok = ok && cudaEventCreateWithFlags(&v->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (uint32_t i = 0; i < kRing; ++i) {
    ok = ok && cudaEventCreateWithFlags(&v->ev_a[i], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&v->ev_f[i], cudaEventDisableTiming) == cudaSuccess;
  }
  return ok;
}


void free_volume(Volume* v) {
  if (!v) return;
  DeviceGuard g(v->device);
  cudaDeviceSynchronize();
  destroy_pipeline(v);
  if (v->prof_ev) {
    for (uint32_t i = 0; i < 3 * kProfCalls; ++i)
      if (v->prof_ev[i]) cudaEventDestroy(v->prof_ev[i]);
    delete[] v->prof_ev;
  }
  cudaFree(v->d_file);
  cudaFree(v->d_tables);
  cudaFree(v->d_flags);
  cudaFree(v->d_host_ids);
  cudaFree(v->d_host_slots);
  cudaFree(v->d_host_cache);
  cudaFree(v->d_host_status);
  if (v->h_full) cudaFreeHost(v->h_full);
  std::free(v->h_rec_words);
  v->kind = 0;
  delete v;
}

}  // namespace

extern "C" {

const char* vc_status_string(vc_status s) {
  switch (s) {
    case VC_OK: return "ok";
    case VC_ERR_ARG: return "invalid argument";
    case VC_ERR_FORMAT: return "invalid volume format";
    case VC_ERR_OOM: return "out of memory";
    case VC_ERR_CUDA: return "CUDA error";
    case VC_ERR_CORRUPT: return "corrupt brick record";
    case VC_ERR_TIMEOUT: return "device wait timed out";
    case VC_ERR_BUSY: return "busy";
    case VC_ERR_UNSUPPORTED: return "unsupported by this build";
    default: return "unknown status";
  }
}

vc_status vc_selftest_bounded_wait(uint32_t budget_us, int32_t* status_dev, void* cuda_stream) {
  if (!status_dev || budget_us == 0 || budget_us > 10000000u) return VC_ERR_ARG;
  return launch_wait_selftest(budget_us, status_dev, static_cast<cudaStream_t>(cuda_stream));
}

}  // extern "C"

namespace vc {

vc_status scan_volume(const uint8_t* p, size_t nbytes, VolumeScan* out) {
  VolumeScan& sc = *out;
  if (nbytes < kHeaderBytes) return VC_ERR_FORMAT;
  if (le32(p) != kMagic || le32(p + 4) != kVersion) return VC_ERR_FORMAT;
  uint32_t dims[3] = {le32(p + 8), le32(p + 12), le32(p + 16)};
  const uint32_t L = le32(p + 20), op_mask = le32(p + 24), coder = le32(p + 28), flags = le32(p + 32);
  const uint32_t n_bricks = le32(p + 36), hdr_max_pal = le32(p + 40), hdr_max_sym = le32(p + 44);
  uint32_t freq[16];
  for (int s = 0; s < 16; ++s) freq[s] = le32(p + 48 + 4 * s);
  const uint32_t records_words = le32(p + 112);
  if (L < 1 || L > 6) return VC_ERR_FORMAT;
  if (!(op_mask & (1u << 4)) || (op_mask & ~0x7Fu)) return VC_ERR_FORMAT;
  if (coder > 1 || (flags & ~(kFlagNoStop | kFlagShortDelta | kFlagRunsMask))) return VC_ERR_FORMAT;
  if (coder != 1 && (flags & kFlagRunsMask)) return VC_ERR_FORMAT;
  const uint32_t K = runs_k(flags);
  const uint32_t b = 1u << L;
  uint32_t nb[3];
  uint64_t nbt = 1;
  for (int a = 0; a < 3; ++a) {
    if (dims[a] == 0) return VC_ERR_FORMAT;
    nb[a] = (dims[a] + b - 1) / b;
    nbt *= nb[a];
  }
  if (nbt != n_bricks) return VC_ERR_FORMAT;
  if (coder == 1) {
    uint32_t sum = 0;
    for (int s = 0; s < 16; ++s) sum += freq[s];
    if (sum != kRansM) return VC_ERR_FORMAT;
  }
  const size_t starts_bytes = 4 * ((size_t)n_bricks + 1);
  const size_t rec_off = (kHeaderBytes + starts_bytes + 15) & ~(size_t)15;
  if (nbytes < rec_off + 4 * (size_t)records_words) return VC_ERR_FORMAT;
  // Brick Starts and every record's sizes
  const uint8_t* st = p + kHeaderBytes;
  const uint8_t* rec = p + rec_off;
  uint32_t max_pal = 0, max_sym = 0, max_delta = 0, max_words = 0, max_stage = 0, max_nodes = 0;
  std::vector<uint8_t> bflags(n_bricks, 0);
  uint32_t prev = le32(st);
  if (prev != 0) return VC_ERR_FORMAT;
  for (uint32_t i = 0; i < n_bricks; ++i) {
    const uint32_t a = le32(st + 4 * (size_t)i), e = le32(st + 4 * ((size_t)i + 1));
    if (e < a || e > records_words || (a & 3u) || (e & 3u) || e - a < 4) return VC_ERR_FORMAT;
    const uint8_t* r = rec + 4 * (size_t)a;
    const uint32_t n_pal = le32(r), S = le32(r + 4), cb = le32(r + 8), nd = le32(r + 12);
    if (S == 0) return VC_ERR_FORMAT;
    const uint64_t ns = coder == 1 ? head_words(S, K) : 0;  // rANS states and run starts
    const uint64_t need = 16 + 4 * ns + 4 * (uint64_t)n_pal + cb;
    if (((need + 15) & ~(uint64_t)15) != 4 * (uint64_t)(e - a)) return VC_ERR_FORMAT;
    if (coder == 0 && cb != (S + 1) / 2) return VC_ERR_FORMAT;
    if (coder == 1 && (cb & 1u)) return VC_ERR_FORMAT;
    if (coder == 1 && K > 1) {  // run starts: not decreasing, within the coded words
      const uint32_t nr = run_n(S, K);
      uint32_t prev_start = 0;
      for (uint32_t k = 1; k < nr; ++k) {
        const uint32_t w0 = le32(r + 16 + 4 * ((size_t)ns - (nr - 1u) + (k - 1u)));
        if (w0 < prev_start || w0 > cb / 2) return VC_ERR_FORMAT;
        prev_start = w0;
      }
    }
    if (nd > S) return VC_ERR_FORMAT;
    max_pal = std::max(max_pal, n_pal);
    max_sym = std::max(max_sym, S);
    max_delta = std::max(max_delta, nd);
    max_nodes = std::max(max_nodes, S - nd);
    max_words = std::max(max_words, e - a);
    // bytes the reconstruction kernel stages: the record (plain), or its head and decoded symbols (rANS)
    const uint32_t stage = coder == 0 ? 4 * (e - a)
                                      : (uint32_t)(((16 + 4 * ns + 4 * (uint64_t)n_pal) + 15) & ~15ull) +
                                            (((S + 1) / 2 + 15) & ~15u);
    max_stage = std::max(max_stage, stage);
    const uint8_t* pal = r + 16 + 4 * ns;
    for (uint32_t k = 0; k < n_pal; ++k) bflags[i] |= le32(pal + 4 * (size_t)k) == 0 ? 1u : 2u;
  }
  if (le32(st + 4 * (size_t)n_bricks) != records_words) return VC_ERR_FORMAT;
  if (max_pal > hdr_max_pal || max_sym > hdr_max_sym) return VC_ERR_FORMAT;
  if (max_pal >= kMaxIdx16) return VC_ERR_UNSUPPORTED;  // palette indices are kept in 16 bits

  for (int a = 0; a < 3; ++a) { sc.dims[a] = dims[a]; sc.nb[a] = nb[a]; }
  sc.L = L; sc.op_mask = op_mask; sc.coder = coder; sc.flags = flags; sc.n_bricks = n_bricks;
  for (int q = 0; q < 16; ++q) sc.freq[q] = freq[q];
  sc.records_words = records_words;
  sc.rec_off = rec_off;
  sc.max_pal = max_pal; sc.max_sym = max_sym; sc.max_delta = max_delta; sc.max_words = max_words;
  sc.max_stage = max_stage; sc.max_nodes = max_nodes;
  sc.bflags.swap(bflags);
  return VC_OK;
}

}  // namespace vc

extern "C" {

vc_status vc_load_compressed(const void* host_bytes, size_t nbytes, int device, void* cuda_stream, vc_volume** out) {
  if (!out) return VC_ERR_ARG;
  *out = nullptr;
  if (!host_bytes) return VC_ERR_ARG;
  const uint8_t* p = static_cast<const uint8_t*>(host_bytes);
  VolumeScan sc;
  {
    const vc_status rc0 = scan_volume(p, nbytes, &sc);
    if (rc0 != VC_OK) return rc0;
  }
  const uint32_t* dims = sc.dims;
  const uint32_t* nb = sc.nb;
  const uint32_t L = sc.L, op_mask = sc.op_mask, coder = sc.coder, flags = sc.flags, n_bricks = sc.n_bricks;
  const uint32_t* freq = sc.freq;
  const size_t rec_off = sc.rec_off;
  const uint32_t records_words = sc.records_words;
  const uint32_t max_pal = sc.max_pal, max_sym = sc.max_sym, max_delta = sc.max_delta, max_words = sc.max_words;
  const uint32_t max_stage = sc.max_stage, max_nodes = sc.max_nodes;
  const std::vector<uint8_t>& bflags = sc.bflags;
  const uint8_t* st = p + kHeaderBytes;

  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return VC_ERR_ARG;
  DeviceGuard g(device);
  Volume* v = new (std::nothrow) Volume();
  if (!v) return VC_ERR_OOM;
  v->kind = kHandleVolume;
  v->device = device;
  for (int a = 0; a < 3; ++a) { v->dims[a] = dims[a]; v->nb[a] = nb[a]; }
  v->L = L; v->op_mask = op_mask; v->coder = coder; v->flags = flags; v->n_bricks = n_bricks;
  v->max_pal = max_pal; v->max_sym = max_sym; v->max_delta = max_delta; v->max_rec_words = max_words;
  v->max_stage = max_stage;
  v->max_nodes = max_nodes;
  v->h_rec_words = static_cast<uint32_t*>(std::malloc(4 * (size_t)n_bricks + 4));
  if (!v->h_rec_words) { delete v; return VC_ERR_OOM; }
  for (uint32_t i = 0; i < n_bricks; ++i) v->h_rec_words[i] = le32(st + 4 * ((size_t)i + 1)) - le32(st + 4 * (size_t)i);
  v->encoded_bytes = nbytes;
  v->sched.threads = L >= 6 ? 1024 : 256;  // b = 64: more threads per (much larger) brick
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    std::free(v->h_rec_words);
    delete v;
    return VC_ERR_CUDA;
  }
  v->sms = (uint32_t)sms;
  v->sched.stage_depth = 1;
  v->sched.blocks_per_sm = 0;
  v->sched.chunk = 512;
  SmemLayout sl, sl_pal;
  vc_status rc = compute_layout(*v, device, v->sched.threads, v->sched.stage_depth, &sl);
  if (rc == VC_OK) rc = compute_layout(*v, device, v->sched.threads, v->sched.stage_depth, &sl_pal, true);
  if (rc != VC_OK) {
    std::free(v->h_rec_words);
    delete v;
    return rc;
  }
  if (!create_pipeline(v)) {
    cudaGetLastError();
    destroy_pipeline(v);
    std::free(v->h_rec_words);
    delete v;
    return VC_ERR_CUDA;
  }

  // the device copy carries 64 zero bytes of slack: 8-nibble windows may read past a record's end
  const size_t file_bytes = rec_off + 4 * (size_t)records_words;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaMalloc(&v->d_file, file_bytes + 64) != cudaSuccess) { cudaGetLastError(); free_volume(v); return VC_ERR_OOM; }
  if (cudaMalloc(&v->d_tables, 4 * kRansM) != cudaSuccess) {
    cudaGetLastError();
    free_volume(v);
    return VC_ERR_OOM;
  }
  if (cudaMalloc(&v->d_flags, n_bricks) != cudaSuccess) {
    cudaGetLastError();
    free_volume(v);
    return VC_ERR_OOM;
  }
  v->device_bytes = file_bytes + 64 + 4 * kRansM + n_bricks;
  // rANS table: per slot, freq[symbol] | (slot - cum[symbol]) << 13 | symbol << 25
  std::vector<uint32_t> tab(kRansM, 0);
  if (coder == 1) {
    uint32_t cum = 0;
    for (uint32_t s = 0; s < 16; ++s) {
      for (uint32_t k = 0; k < freq[s]; ++k) tab[cum + k] = freq[s] | (k << 13) | (s << 25);
      cum += freq[s];
    }
  }
  bool ok = cudaMemsetAsync(v->d_file + file_bytes, 0, 64, stream) == cudaSuccess &&
            cudaMemcpyAsync(v->d_file, p, file_bytes, cudaMemcpyHostToDevice, stream) == cudaSuccess &&
            cudaMemcpyAsync(v->d_tables, tab.data(), 4 * kRansM, cudaMemcpyHostToDevice, stream) == cudaSuccess &&
            cudaMemcpyAsync(v->d_flags, bflags.data(), n_bricks, cudaMemcpyHostToDevice, stream) == cudaSuccess &&
            cudaStreamSynchronize(stream) == cudaSuccess;
  if (!ok) { free_volume(v); return VC_ERR_CUDA; }
  v->dv.records = reinterpret_cast<const uint32_t*>(v->d_file + rec_off);
  v->dv.starts = reinterpret_cast<const uint32_t*>(v->d_file + kHeaderBytes);
  v->dv.rans_tab = reinterpret_cast<const uint32_t*>(v->d_tables);
  v->dv.n_bricks = n_bricks;
  v->dv.L = L;
  v->dv.op_mask = op_mask;
  v->dv.coder = coder;
  v->dv.flags = flags;
  v->dv.prefix_lod = kPrefixMinLod;
  v->dv.sm = sl;
  v->sm_pal = sl_pal;
  *out = reinterpret_cast<vc_volume*>(v);
  return VC_OK;
}

vc_status vc_volume_info_get(const vc_volume* vol, vc_volume_info* info) {
  const Volume* v = reinterpret_cast<const Volume*>(vol);
  if (!v || !info || v->kind != kHandleVolume) return VC_ERR_ARG;
  std::memset(info, 0, sizeof(*info));
  for (int a = 0; a < 3; ++a) { info->dims[a] = v->dims[a]; info->bricks_per_axis[a] = v->nb[a]; }
  info->brick_size = 1u << v->L;
  info->log2b = v->L;
  info->n_bricks = v->n_bricks;
  info->op_mask = v->op_mask;
  info->coder = v->coder;
  info->flags = v->flags;
  info->max_pal = v->max_pal;
  info->max_sym = v->max_sym;
  info->max_delta = v->max_delta;
  info->encoded_bytes = v->encoded_bytes;
  info->device_bytes = v->device_bytes;
  info->smem_bytes = v->dv.sm.total;
  info->split = v->split ? 1u : 0u;
  info->host_bytes = v->host_bytes;
  info->device = (uint32_t)v->device;
  return VC_OK;
}

vc_status vc_volume_set_schedule(vc_volume* vol, const vc_schedule* sched) {
  Volume* v = reinterpret_cast<Volume*>(vol);
  if (!v || !sched || v->kind != kHandleVolume) return VC_ERR_ARG;
  if (sched->stage_depth < 1 || sched->stage_depth > 2) return VC_ERR_ARG;
  if (!schedule_supported(v->L, sched->threads)) return VC_ERR_UNSUPPORTED;
  DeviceGuard g(v->device);
  SmemLayout sl, sl_pal;
  vc_status rc = compute_layout(*v, v->device, sched->threads, sched->stage_depth, &sl);
  if (rc == VC_OK) rc = compute_layout(*v, v->device, sched->threads, sched->stage_depth, &sl_pal, true);
  if (rc != VC_OK) return rc;
  v->sched = *sched;
  if (!v->sched.chunk) v->sched.chunk = 512;
  v->dv.sm = sl;
  v->sm_pal = sl_pal;
  return VC_OK;
}

vc_status vc_volume_get_schedule(const vc_volume* vol, vc_schedule* sched) {
  const Volume* v = reinterpret_cast<const Volume*>(vol);
  if (!v || !sched || v->kind != kHandleVolume) return VC_ERR_ARG;
  *sched = v->sched;
  return VC_OK;
}

vc_status vc_coarsest_labels(vc_volume* vol, const uint32_t* brick_ids, uint32_t n, uint32_t* out_labels,
                             int32_t* status_dev, void* cuda_stream) {
  Volume* v = reinterpret_cast<Volume*>(vol);
  if (!v || v->kind != kHandleVolume) return VC_ERR_ARG;
  if (n == 0) return VC_OK;
  if (!brick_ids || !out_labels || !status_dev) return VC_ERR_ARG;
  DeviceGuard g(v->device);
  return launch_coarsest(*v, brick_ids, n, out_labels, status_dev, static_cast<cudaStream_t>(cuda_stream));
}

vc_status vc_decode_bricks(vc_volume* vol, const uint32_t* brick_ids, uint32_t n, const uint32_t* cache_slots,
                           uint32_t* cache, uint32_t lod, uint32_t mode, int32_t* status_dev, void* cuda_stream) {
  Volume* v = reinterpret_cast<Volume*>(vol);
  if (!v || v->kind != kHandleVolume) return VC_ERR_ARG;
  if (n == 0) return VC_OK;
  if (!brick_ids || !cache_slots || !cache || !status_dev) return VC_ERR_ARG;
  if (lod > v->L || (mode & ~VC_MODE_PALETTED) > VC_MODE_PIPELINED) return VC_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(cache) & 15u) return VC_ERR_ARG;
  DeviceGuard g(v->device);
  return launch_decode(*v, brick_ids, n, cache_slots, cache, lod, mode, status_dev,
                       static_cast<cudaStream_t>(cuda_stream));
}

vc_status vc_decode_bricks_host(vc_volume* vol, const uint32_t* brick_ids, uint32_t n, uint32_t lod, uint32_t mode,
                                uint32_t* labels_out, int32_t* status_out, void* cuda_stream) {
  Volume* v = reinterpret_cast<Volume*>(vol);
  if (!v || v->kind != kHandleVolume || !status_out) return VC_ERR_ARG;
  *status_out = 0;
  if (n == 0) return VC_OK;
  if (!brick_ids || !labels_out || lod > v->L || mode > VC_MODE_PIPELINED) return VC_ERR_ARG;
  DeviceGuard g(v->device);
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  const uint32_t edge = (1u << v->L) >> lod;
  const size_t words = (size_t)n * edge * edge * edge;
  if (n > v->host_cap_items) {
    cudaFree(v->d_host_ids);
    cudaFree(v->d_host_slots);
    v->d_host_ids = v->d_host_slots = nullptr;
    v->host_cap_items = 0;
    if (cudaMalloc(&v->d_host_ids, 4 * (size_t)n) != cudaSuccess ||
        cudaMalloc(&v->d_host_slots, 4 * (size_t)n) != cudaSuccess) {
      cudaGetLastError();
      return VC_ERR_OOM;
    }
    std::vector<uint32_t> iota(n);
    for (uint32_t i = 0; i < n; ++i) iota[i] = i;
    if (cudaMemcpy(v->d_host_slots, iota.data(), 4 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess)
      return VC_ERR_CUDA;
    v->host_cap_items = n;
  }
  // pinned host memory that CUDA maps into the device's address space: the decode kernels write
  // the labels there directly (over NVLink-C2C on GB300), with no staging buffer and no copy
  uint32_t* direct = nullptr;
  {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, labels_out) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer && !(reinterpret_cast<uintptr_t>(pa.devicePointer) & 15u))
      direct = static_cast<uint32_t*>(pa.devicePointer);
    else
      cudaGetLastError();
  }
  if (!direct && words > v->host_cap_words) {
    cudaFree(v->d_host_cache);
    v->d_host_cache = nullptr;
    v->host_cap_words = 0;
    if (cudaMalloc(&v->d_host_cache, 4 * words) != cudaSuccess) { cudaGetLastError(); return VC_ERR_OOM; }
    v->host_cap_words = words;
  }
  if (!v->d_host_status) {
    if (cudaMalloc(&v->d_host_status, 4 * VC_STATUS_WORDS) != cudaSuccess) { cudaGetLastError(); return VC_ERR_OOM; }
  }
  if (cudaMemsetAsync(v->d_host_status, 0, 4 * VC_STATUS_WORDS, stream) != cudaSuccess) return VC_ERR_CUDA;
  if (cudaMemcpyAsync(v->d_host_ids, brick_ids, 4 * (size_t)n, cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return VC_ERR_CUDA;
  vc_status rc = launch_decode(*v, v->d_host_ids, n, v->d_host_slots, direct ? direct : v->d_host_cache, lod, mode,
                               v->d_host_status, stream);
  if (rc != VC_OK) return rc;
  if (!direct &&
      cudaMemcpyAsync(labels_out, v->d_host_cache, 4 * words, cudaMemcpyDeviceToHost, stream) != cudaSuccess)
    return VC_ERR_CUDA;
  int32_t st = 0;
  if (cudaMemcpyAsync(&st, v->d_host_status, 4, cudaMemcpyDeviceToHost, stream) != cudaSuccess) return VC_ERR_CUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return VC_ERR_CUDA;
  *status_out = st;
  return VC_OK;
}

vc_status vc_volume_slot_words(const vc_volume* vol, uint32_t lod, uint32_t paletted, uint32_t* words,
                               uint32_t* bits, uint32_t* per_word) {
  const Volume* v = reinterpret_cast<const Volume*>(vol);
  if (!v || v->kind != kHandleVolume || !words || lod > v->L) return VC_ERR_ARG;
  const uint32_t edge = (1u << v->L) >> lod;
  uint32_t I = 32, E = 1;
  if (paletted) palette_packing(v->max_pal, &I, &E);
  *words = (edge * edge * edge + E - 1u) / E;
  if (bits) *bits = I;
  if (per_word) *per_word = E;
  return VC_OK;
}

vc_status vc_volume_set_profiling(vc_volume* vol, int enable) {
  Volume* v = reinterpret_cast<Volume*>(vol);
  if (!v || v->kind != kHandleVolume) return VC_ERR_ARG;
  if (enable && !v->prof_ev) {
    DeviceGuard g(v->device);
    v->prof_ev = new (std::nothrow) cudaEvent_t[3 * kProfCalls]();
    if (!v->prof_ev) return VC_ERR_OOM;
    for (uint32_t i = 0; i < 3 * kProfCalls; ++i) {
      if (cudaEventCreate(&v->prof_ev[i]) != cudaSuccess) {
        cudaGetLastError();
        for (uint32_t j = 0; j < i; ++j) cudaEventDestroy(v->prof_ev[j]);
        delete[] v->prof_ev;
        v->prof_ev = nullptr;
        return VC_ERR_CUDA;
      }
    }
  }
  v->prof = enable != 0;
  return VC_OK;
}

vc_status vc_volume_kernel_stats(vc_volume* vol, int reset, vc_kernel_stats* out) {
  Volume* v = reinterpret_cast<Volume*>(vol);
  if (!v || v->kind != kHandleVolume || !out) return VC_ERR_ARG;
  DeviceGuard g(v->device);
  std::memset(out, 0, sizeof(*out));
  out->launches = v->launches;
  out->timed_calls = v->prof_used;
  out->dropped_calls = v->prof_dropped;
  for (uint32_t c = 0; c < v->prof_used; ++c) {
    cudaEvent_t* e = v->prof_ev + 3 * c;
    float a = 0.f, b = 0.f;
    if (cudaEventSynchronize(e[2]) != cudaSuccess || cudaEventElapsedTime(&a, e[0], e[1]) != cudaSuccess ||
        cudaEventElapsedTime(&b, e[1], e[2]) != cudaSuccess)
      return VC_ERR_CUDA;
    out->symbol_ms += a;
    out->reconstruct_ms += b;
  }
  if (reset) {
    v->launches = 0;
    v->prof_used = 0;
    v->prof_dropped = 0;
  }
  return VC_OK;
}

vc_status vc_release(void* handle) {
  if (!handle) return VC_OK;
  uint32_t kind = *static_cast<uint32_t*>(handle);
  if (kind == kHandleVolume) {
    free_volume(static_cast<Volume*>(handle));
    return VC_OK;
  }
  if (release_server(handle)) return VC_OK;
  if (release_cache(handle)) return VC_OK;
  if (release_frame(handle)) return VC_OK;
  return VC_ERR_ARG;
}

}  // extern "C"
