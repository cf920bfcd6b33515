// Schedule autotuner: times the decode schedules a volume supports on a sample of its bricks and
// keeps the fastest. The paper decodes all requested bricks in parallel (Results, "GPU-based
// rendering pipeline") and leaves the mapping onto the GPU open; the knobs here are this
// library's: threads per brick, staging depth, persistent blocks per SM, grid vs batched.
#include <cuda_runtime.h>

#include <vector>

#include "vc_internal.h"

using namespace vc;

extern "C" vc_status vc_volume_autotune(vc_volume* vol, const uint32_t* brick_ids, uint32_t n,
                                        const uint32_t* cache_slots, uint32_t* cache, uint32_t lod,
                                        int32_t* status_dev, void* cuda_stream, uint32_t reps, vc_schedule* best,
                                        uint32_t* best_mode, float* best_ms) {
  Volume* v = reinterpret_cast<Volume*>(vol);
  if (!v || v->kind != kHandleVolume || !best || !best_mode) return VC_ERR_ARG;
  if (n == 0 || !brick_ids || !cache_slots || !cache || !status_dev || lod > v->L) return VC_ERR_ARG;
  if (reps == 0) reps = 3;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != v->device) cudaSetDevice(v->device);
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  const vc_schedule start = v->sched;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  vc_status rc = VC_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = VC_ERR_CUDA;
  float best_t = 1e30f;
  vc_schedule best_s = start;
  uint32_t best_m = VC_MODE_BATCHED;
  const uint32_t threads[] = {256, 512, 1024};
  const uint32_t depths[] = {1, 2};
  const uint32_t per_sm[] = {0, 1, 2};
  for (uint32_t t : threads) {
    for (uint32_t d : depths) {
      for (uint32_t mode : {(uint32_t)VC_MODE_GRID, (uint32_t)VC_MODE_BATCHED}) {
        for (uint32_t bps : per_sm) {
          if (rc != VC_OK) break;
          if (mode == VC_MODE_GRID && (bps != 0 || d != 1)) continue;  // knobs of the batched schedule
          vc_schedule s{t, d, bps, start.chunk};
          if (vc_volume_set_schedule(vol, &s) != VC_OK) continue;  // not built or does not fit
          // one untimed run, then reps timed ones
          if (launch_decode(*v, brick_ids, n, cache_slots, cache, lod, mode, status_dev, stream) != VC_OK) continue;
          if (cudaEventRecord(e0, stream) != cudaSuccess) { rc = VC_ERR_CUDA; break; }
          bool ok = true;
          for (uint32_t r = 0; r < reps && ok; ++r)
            ok = launch_decode(*v, brick_ids, n, cache_slots, cache, lod, mode, status_dev, stream) == VC_OK;
          float ms = 0.f;
          if (!ok || cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = VC_ERR_CUDA;
            break;
          }
          ms /= (float)reps;
          if (ms < best_t) {
            best_t = ms;
            best_s = v->sched;
            best_m = mode;
          }
        }
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  const vc_schedule keep = rc == VC_OK && best_t < 1e30f ? best_s : start;
  vc_schedule k = keep;
  if (vc_volume_set_schedule(vol, &k) != VC_OK && rc == VC_OK) rc = VC_ERR_CUDA;
  if (rc == VC_OK) {
    *best = keep;
    *best_mode = best_m;
    if (best_ms) *best_ms = best_t;
  }
  if (prev >= 0 && prev != v->device) cudaSetDevice(prev);
  return rc;
}
