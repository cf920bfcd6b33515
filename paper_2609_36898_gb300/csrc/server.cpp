// Serving runtime: brick requests from many clients, a device brick cache with LRU eviction,
// admission by free cache memory, and continuous batching of the decode work.
//
// Paper (Methods, "GPU rendering pipeline"; Results, "GPU-based rendering pipeline"): each frame,
// the bricks that rays need are requested, cache space is provided by freeing bricks that are no
// longer used, free space is assigned to the new bricks, and all new bricks are decoded in
// parallel. Here the requests come from many concurrent clients instead of one frame loop: a
// server thread admits them in arrival order when their missing bricks fit in free plus evictable
// cache memory, gathers the missing bricks of every admitted request into decode batches (one
// batched-schedule launch per volume and level of detail), keeps up to `max_inflight` batches on
// the GPU, and retires them in order. Requests that arrive while batches run join the next batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <queue>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cache.h"
#include "vc_internal.h"

namespace vc {
namespace {

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
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

constexpr uint32_t kMaxGroups = 512;  // (volume, level of detail) pairs in one batch

inline uint64_t make_key(uint32_t vol, uint32_t lod, uint32_t brick) {
  return ((uint64_t)vol << 36) | ((uint64_t)lod << 32) | brick;
}

}  // namespace

struct Request {
  uint64_t id = 0;
  uint32_t vol = 0;
  std::vector<uint32_t> bricks, lods;
  std::vector<uint32_t> entries;
  std::vector<uint64_t> offsets;
  int32_t state = VC_REQ_WAITING;
  int32_t status = VC_OK;
  uint64_t dep = 0;  // decode positions up to dep (exclusive) must be retired
  uint32_t hits = 0;
  uint64_t bytes = 0;
  uint64_t t_submit = 0, t_admit = 0, t_done = 0;
};

struct BatchSlot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  uint32_t *h_ids = nullptr, *h_slots = nullptr, *d_ids = nullptr, *d_slots = nullptr;
  int32_t *h_status = nullptr, *d_status = nullptr;
  // CUDA-graph launches (VC_SERVER_GRAPHS): the rANS symbol workspace is the slot's own, so the
  // captured work allocates nothing and a later batch of the same shape updates the graph in place
  uint8_t* d_ws = nullptr;
  size_t ws_cap = 0;
  cudaGraphExec_t exec = nullptr;
};

struct Group {
  uint32_t vol, lod, first, count;
};

struct Batch {
  uint32_t slot;
  uint64_t pos_end;  // decode positions [.., pos_end) are in this or earlier batches
  std::vector<Group> groups;
  std::vector<uint32_t> entries;  // entry of each item
};

struct Pending {
  uint32_t vol, lod, brick, entry;
  uint64_t slot_index;
};

struct Server {
  uint32_t kind = kHandleServer;
  // camera request stage (callers of vc_request_bricks take req_mu, not mu)
  std::mutex req_mu;
  cudaStream_t req_stream = nullptr;
  void* h_cams = nullptr;
  uint32_t h_cams_cap = 0;
  vc_server_config cfg{};
  int device = 0;
  uint8_t* d_cache = nullptr;
  std::unique_ptr<BrickCache> cache;
  std::vector<Volume*> volumes;
  std::vector<BatchSlot> slots;
  std::vector<uint32_t> free_slots;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread thread;
  bool stop = false;
  uint64_t wake = 0;  // bumped by submissions and releases
  vc_status fatal = VC_OK;

  uint64_t next_id = 1;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> requests;
  std::deque<uint64_t> waiting;
  std::priority_queue<std::pair<uint64_t, uint64_t>, std::vector<std::pair<uint64_t, uint64_t>>,
                      std::greater<std::pair<uint64_t, uint64_t>>>
      by_dep;  // admitted requests by dep
  std::deque<Pending> pending;
  uint64_t pos_enqueued = 0, pos_launched = 0, pos_retired = 0;
  std::deque<Batch> inflight;
  std::vector<uint64_t> entry_pos;  // decode position of each cache entry's item

  vc_server_stats stats{};
};

namespace {

void free_server(Server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->thread.joinable()) s->thread.join();
  DeviceGuard g(s->device);
  for (BatchSlot& b : s->slots) {
    if (b.stream) cudaStreamSynchronize(b.stream);
    if (b.stream) cudaStreamDestroy(b.stream);
    if (b.done) cudaEventDestroy(b.done);
    if (b.exec) cudaGraphExecDestroy(b.exec);
    cudaFree(b.d_ws);
    cudaFreeHost(b.h_ids);
    cudaFreeHost(b.h_slots);
    cudaFreeHost(b.h_status);
    cudaFree(b.d_ids);
    cudaFree(b.d_slots);
    cudaFree(b.d_status);
  }
  cudaFree(s->d_cache);
  if (s->req_stream) cudaStreamDestroy(s->req_stream);
  cudaFreeHost(s->h_cams);
  s->kind = 0;
  delete s;
}

// --- everything below runs with s->mu held ---

void finish_request(Server* s, Request& r, int32_t state, int32_t status) {
  r.state = state;
  r.status = status;
  r.t_done = now_ns();
  if (state == VC_REQ_DONE) ++s->stats.requests_done;
  else ++s->stats.requests_failed;
}

// Admits waiting requests in arrival order while their missing bricks fit.
void admit(Server* s) {
  std::vector<uint64_t> keys;
  std::vector<uint32_t> cls;
  std::vector<BrickCache::Ref> refs;
  while (!s->waiting.empty()) {
    Request& r = *s->requests[s->waiting.front()];
    const Volume& v = *s->volumes[r.vol];
    const uint32_t n = (uint32_t)r.bricks.size();
    keys.resize(n);
    cls.resize(n);
    refs.resize(n);
    for (uint32_t i = 0; i < n; ++i) {
      keys[i] = make_key(r.vol, r.lods[i], r.bricks[i]);
      cls[i] = v.L - r.lods[i];
    }
    if (!s->cache->acquire(keys.data(), cls.data(), n, refs.data())) break;  // wait for space
    s->waiting.pop_front();
    r.entries.resize(n);
    r.offsets.resize(n);
    uint64_t dep = 0;
    for (uint32_t i = 0; i < n; ++i) {
      const uint32_t e = refs[i].entry;
      r.entries[i] = e;
      r.offsets[i] = refs[i].offset;
      if (e >= s->entry_pos.size()) s->entry_pos.resize(e + 1, 0);
      if (!refs[i].hit) {
        const uint32_t edge = (1u << v.L) >> r.lods[i];
        s->entry_pos[e] = s->pos_enqueued++;
        s->pending.push_back(Pending{r.vol, r.lods[i], r.bricks[i], e, refs[i].offset / (4ull * edge * edge * edge)});
      } else {
        ++r.hits;
      }
      dep = std::max(dep, s->entry_pos[e] + 1);
    }
    r.dep = dep;
    r.state = VC_REQ_ADMITTED;
    r.t_admit = now_ns();
    ++s->stats.requests_admitted;
    s->stats.bricks_hit += r.hits;
    s->stats.bricks_missed += n - r.hits;
    s->by_dep.push({r.dep, r.id});
  }
}

// Enqueues one batch of pending decode items on a free batch slot.
bool launch_batch(Server* s) {
  if (s->pending.empty() || s->free_slots.empty()) return false;
  const uint32_t si = s->free_slots.back();
  BatchSlot& B = s->slots[si];
  Batch batch;
  batch.slot = si;
  // take up to max_batch_items items, grouped by (volume, lod) in first-seen order
  const uint32_t cap = s->cfg.max_batch_items;
  std::map<std::pair<uint32_t, uint32_t>, std::vector<uint32_t>> by_group;
  std::vector<std::pair<uint32_t, uint32_t>> order;
  std::vector<Pending> taken;
  while (!s->pending.empty() && taken.size() < cap) {
    const Pending& p = s->pending.front();
    auto key = std::make_pair(p.vol, p.lod);
    auto it = by_group.find(key);
    if (it == by_group.end()) {
      if (order.size() == kMaxGroups) break;
      order.push_back(key);
      it = by_group.emplace(key, std::vector<uint32_t>()).first;
    }
    it->second.push_back((uint32_t)taken.size());
    taken.push_back(p);
    s->pending.pop_front();
  }
  uint32_t at = 0;
  for (const auto& key : order) {
    auto& idx = by_group[key];
    // longest records first: the persistent blocks take items in order, so the big bricks start
    // early and the short ones fill the tail
    const uint32_t* rw = s->volumes[key.first]->h_rec_words;
    std::stable_sort(idx.begin(), idx.end(),
                     [&](uint32_t a, uint32_t b) { return rw[taken[a].brick] > rw[taken[b].brick]; });
    batch.groups.push_back(Group{key.first, key.second, at, (uint32_t)idx.size()});
    const uint64_t edge = (1u << s->volumes[key.first]->L) >> key.second;
    s->stats.voxels_decoded += edge * edge * edge * idx.size();
    for (uint32_t k : idx) {
      B.h_ids[at] = taken[k].brick;
      B.h_slots[at] = (uint32_t)taken[k].slot_index;
      batch.entries.push_back(taken[k].entry);
      ++at;
    }
  }
  s->pos_launched += taken.size();
  batch.pos_end = s->pos_launched;
  const size_t ng = batch.groups.size();
  const bool graphs = (s->cfg.flags & VC_SERVER_GRAPHS) != 0;
  // workspace offsets of the groups (graph launches only)
  std::vector<size_t> ws_off(ng, 0);
  bool ok = true;
  if (graphs) {
    size_t need = 0;
    for (size_t g = 0; g < ng; ++g) {
      ws_off[g] = need;
      const Volume& v = *s->volumes[batch.groups[g].vol];
      need += (decode_ws_bytes(v, batch.groups[g].count) + 255) & ~size_t(255);
    }
    if (need > B.ws_cap) {  // grow outside any capture
      cudaStreamSynchronize(B.stream);
      cudaFree(B.d_ws);
      B.d_ws = nullptr;
      B.ws_cap = 0;
      if (cudaMalloc(reinterpret_cast<void**>(&B.d_ws), need) != cudaSuccess) {
        cudaGetLastError();
        ok = false;
      } else {
        B.ws_cap = need;
      }
    }
    ok = ok && cudaStreamBeginCapture(B.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  }
  ok = ok && cudaMemcpyAsync(B.d_ids, B.h_ids, 4ull * at, cudaMemcpyHostToDevice, B.stream) == cudaSuccess &&
       cudaMemcpyAsync(B.d_slots, B.h_slots, 4ull * at, cudaMemcpyHostToDevice, B.stream) == cudaSuccess &&
       cudaMemsetAsync(B.d_status, 0, 4ull * VC_STATUS_WORDS * ng, B.stream) == cudaSuccess;
  for (size_t g = 0; ok && g < ng; ++g) {
    const Group& G = batch.groups[g];
    Volume& v = *s->volumes[G.vol];
    if (graphs && decode_ws_bytes(v, G.count) != 0)  // rANS symbols or b = 64 scratch
      ok = launch_decode_ws(v, B.d_ids + G.first, G.count, B.d_slots + G.first, reinterpret_cast<uint32_t*>(s->d_cache),
                            G.lod, VC_MODE_BATCHED, B.d_status + VC_STATUS_WORDS * g, B.stream, B.d_ws + ws_off[g],
                            B.ws_cap - ws_off[g], /*presorted=*/true) == VC_OK;
    else
      ok = launch_decode(v, B.d_ids + G.first, G.count, B.d_slots + G.first, reinterpret_cast<uint32_t*>(s->d_cache),
                         G.lod, VC_MODE_BATCHED, B.d_status + VC_STATUS_WORDS * g, B.stream, /*presorted=*/true) == VC_OK;
  }
  ok = ok &&
       cudaMemcpyAsync(B.h_status, B.d_status, 4ull * VC_STATUS_WORDS * ng, cudaMemcpyDeviceToHost, B.stream) ==
           cudaSuccess;
  if (graphs) {
    cudaGraph_t graph = nullptr;
    const bool captured = cudaStreamEndCapture(B.stream, &graph) == cudaSuccess && graph;
    ok = ok && captured;
    if (ok) {
      cudaGraphExecUpdateResultInfo info;
      if (!B.exec || cudaGraphExecUpdate(B.exec, graph, &info) != cudaSuccess) {
        cudaGetLastError();
        if (B.exec) cudaGraphExecDestroy(B.exec);
        B.exec = nullptr;
        ok = cudaGraphInstantiate(&B.exec, graph, 0) == cudaSuccess;
        if (ok) ++s->stats.graph_instantiations;
      }
      ok = ok && cudaGraphLaunch(B.exec, B.stream) == cudaSuccess;
      if (ok) ++s->stats.graph_launches;
    }
    if (graph) cudaGraphDestroy(graph);
  }
  ok = ok && cudaEventRecord(B.done, B.stream) == cudaSuccess;
  if (!ok) {
    s->fatal = VC_ERR_CUDA;
    return false;
  }
  s->free_slots.pop_back();
  ++s->stats.batches;
  s->stats.bricks_decoded += at;
  s->inflight.push_back(std::move(batch));
  return true;
}

// Retires finished batches in launch order; completes requests whose bricks are all resident.
bool retire(Server* s) {
  bool any = false;
  while (!s->inflight.empty()) {
    Batch& b = s->inflight.front();
    BatchSlot& B = s->slots[b.slot];
    const cudaError_t q = cudaEventQuery(B.done);
    if (q == cudaErrorNotReady) break;
    if (q != cudaSuccess) {
      s->fatal = VC_ERR_CUDA;
      break;
    }
    bool failed = false;
    for (size_t g = 0; g < b.groups.size(); ++g) {
      const int32_t code = B.h_status[VC_STATUS_WORDS * g];
      if (code != 0) {
        failed = true;
        const Group& G = b.groups[g];
        for (uint32_t i = 0; i < G.count; ++i) s->cache->invalidate(b.entries[G.first + i]);
        ++s->stats.batch_errors;
      }
    }
    if (failed) {  // every admitted request holding a brick of a failed group fails with its code
      for (size_t g = 0; g < b.groups.size(); ++g) {
        const int32_t code = B.h_status[VC_STATUS_WORDS * g];
        if (code == 0) continue;
        const Group& G = b.groups[g];
        std::vector<uint32_t> bad(b.entries.begin() + G.first, b.entries.begin() + G.first + G.count);
        std::sort(bad.begin(), bad.end());
        for (auto& kv : s->requests) {
          Request& r = *kv.second;
          if (r.state != VC_REQ_ADMITTED) continue;
          for (uint32_t e : r.entries) {
            if (std::binary_search(bad.begin(), bad.end(), e)) {
              finish_request(s, r, VC_REQ_FAILED, code);
              break;
            }
          }
        }
      }
    }
    s->pos_retired = b.pos_end;
    s->free_slots.push_back(b.slot);
    s->inflight.pop_front();  // b is gone from here on
    any = true;
  }
  return any;
}

// Completes admitted requests whose decode positions are all retired.
bool complete(Server* s) {
  bool any = false;
  while (!s->by_dep.empty() && s->by_dep.top().first <= s->pos_retired) {
    const uint64_t id = s->by_dep.top().second;
    s->by_dep.pop();
    auto it = s->requests.find(id);
    if (it == s->requests.end() || it->second->state != VC_REQ_ADMITTED) continue;
    finish_request(s, *it->second, VC_REQ_DONE, VC_OK);
    any = true;
  }
  return any;
}

void server_loop(Server* s) {
  DeviceGuard g(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  uint64_t seen = s->wake;
  while (!s->stop) {
    bool progressed = retire(s);
    admit(s);
    while (s->fatal == VC_OK && launch_batch(s)) {
    }
    progressed |= complete(s);  // also requests admitted with every brick already resident
    if (progressed) s->cv_done.notify_all();
    if (s->fatal != VC_OK) {
      for (auto& kv : s->requests) {
        Request& r = *kv.second;
        if (r.state == VC_REQ_WAITING || r.state == VC_REQ_ADMITTED) finish_request(s, r, VC_REQ_FAILED, s->fatal);
      }
      s->waiting.clear();
      s->cv_done.notify_all();
      s->cv_work.wait(lock, [&] { return s->stop; });
      break;
    }
    if (!s->inflight.empty()) {  // poll the oldest batch's event
      lock.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(5));
      lock.lock();
    } else if (s->pending.empty() || s->free_slots.empty()) {  // idle until a submission or a release
      s->cv_work.wait(lock, [&] { return s->stop || s->wake != seen; });
      seen = s->wake;
    }
  }
}

}  // namespace
}  // namespace vc

using namespace vc;

extern "C" {

vc_status vc_server_create(const vc_server_config* cfg, vc_server** out) {
  if (!cfg || !out) return VC_ERR_ARG;
  *out = nullptr;
  vc_server_config c = *cfg;
  if (!c.max_batch_items) c.max_batch_items = 65536;
  if (!c.max_inflight) c.max_inflight = 2;
  if (!c.max_class) c.max_class = 6;
  if (!c.min_class) c.min_class = 2;
  if (c.min_class > c.max_class || c.max_class > 9 || c.max_inflight > 8 ||
      c.cache_bytes < BrickCache::block_bytes(c.max_class) || (c.flags & ~VC_SERVER_GRAPHS))
    return VC_ERR_ARG;
  Server* s = new (std::nothrow) Server();
  if (!s) return VC_ERR_OOM;
  s->cfg = c;
  s->device = c.device;
  DeviceGuard g(c.device);
  try {
    s->cache.reset(new BrickCache(c.cache_bytes, c.min_class, c.max_class));
  } catch (...) {
    delete s;
    return VC_ERR_OOM;
  }
  if (cudaMalloc(&s->d_cache, s->cache->capacity_bytes()) != cudaSuccess) {
    cudaGetLastError();
    s->cache.reset();
    delete s;
    return VC_ERR_OOM;
  }
  s->slots.resize(c.max_inflight);
  for (uint32_t i = 0; i < c.max_inflight; ++i) {
    BatchSlot& B = s->slots[i];
    const size_t nb = 4ull * c.max_batch_items, sb = 4ull * VC_STATUS_WORDS * kMaxGroups;
    if (cudaStreamCreateWithFlags(&B.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&B.h_ids), nb, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&B.h_slots), nb, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&B.h_status), sb, cudaHostAllocDefault) != cudaSuccess ||
        cudaMalloc(&B.d_ids, nb) != cudaSuccess || cudaMalloc(&B.d_slots, nb) != cudaSuccess ||
        cudaMalloc(&B.d_status, sb) != cudaSuccess) {
      cudaGetLastError();
      free_server(s);
      return VC_ERR_OOM;
    }
    s->free_slots.push_back(c.max_inflight - 1 - i);
  }
  if (cudaStreamCreateWithFlags(&s->req_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    free_server(s);
    return VC_ERR_CUDA;
  }
  s->stats.cache_bytes = s->cache->capacity_bytes();
  s->thread = std::thread(server_loop, s);
  *out = reinterpret_cast<vc_server*>(s);
  return VC_OK;
}

vc_status vc_server_add_volume(vc_server* srv, vc_volume* vol, uint32_t* volume_index) {
  Server* s = reinterpret_cast<Server*>(srv);
  Volume* v = reinterpret_cast<Volume*>(vol);
  if (!s || s->kind != kHandleServer || !v || v->kind != kHandleVolume || !volume_index) return VC_ERR_ARG;
  if (v->device != s->device) return VC_ERR_ARG;
  if (v->L > s->cfg.max_class) return VC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->volumes.size() >= (1u << 20)) return VC_ERR_UNSUPPORTED;
  *volume_index = (uint32_t)s->volumes.size();
  s->volumes.push_back(v);
  return VC_OK;
}

}  // extern "C"

namespace {

vc_status submit(Server* s, uint32_t volume_index, const uint32_t* brick_ids, const uint32_t* lods, uint32_t n,
                 uint64_t* request_id) {
  if (!request_id || (n && !brick_ids)) return VC_ERR_ARG;
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return VC_ERR_OOM;
  const Volume* v = nullptr;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (volume_index >= s->volumes.size()) return VC_ERR_ARG;
    v = s->volumes[volume_index];
  }
  r->vol = volume_index;
  r->bricks.assign(brick_ids, brick_ids + n);
  r->lods.assign(n, 0);
  if (lods) r->lods.assign(lods, lods + n);
  uint64_t bytes = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (r->bricks[i] >= v->n_bricks || r->lods[i] > v->L) return VC_ERR_ARG;
    const uint32_t c = std::max(v->L - r->lods[i], s->cfg.min_class);
    bytes += BrickCache::block_bytes(c);
  }
  if (bytes > s->cache->capacity_bytes()) return VC_ERR_BUSY;  // could never be admitted
  r->bytes = bytes;
  r->t_submit = now_ns();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->fatal != VC_OK) return s->fatal;
    r->id = s->next_id++;
    *request_id = r->id;
    ++s->stats.requests_submitted;
    if (n == 0) {
      r->state = VC_REQ_DONE;
      r->t_admit = r->t_done = r->t_submit;
      ++s->stats.requests_done;
    } else {
      s->waiting.push_back(r->id);
    }
    s->requests.emplace(r->id, std::move(r));
    ++s->wake;
  }
  s->cv_work.notify_one();
  return VC_OK;
}

}  // namespace

extern "C" {

vc_status vc_submit_bricks(vc_server* srv, uint32_t volume_index, const uint32_t* brick_ids, const uint32_t* lods,
                           uint32_t n, uint64_t* request_id) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || s->kind != kHandleServer) return VC_ERR_ARG;
  return submit(s, volume_index, brick_ids, lods, n, request_id);
}

vc_status vc_request_bricks(vc_server* srv, uint32_t volume_index, const vc_camera* cams, uint32_t ncams,
                            uint32_t max_lod, uint64_t* request_ids_out) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || s->kind != kHandleServer || !cams || !request_ids_out) return VC_ERR_ARG;
  if (ncams == 0) return VC_OK;
  Volume* v = nullptr;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (volume_index >= s->volumes.size()) return VC_ERR_ARG;
    v = s->volumes[volume_index];
  }
  for (uint32_t i = 0; i < ncams; ++i)
    if (cams[i].width == 0 || cams[i].height == 0 || (uint64_t)cams[i].width * cams[i].height > 0xFFFFFFFFull)
      return VC_ERR_ARG;
  std::lock_guard<std::mutex> rlock(s->req_mu);
  DeviceGuard g(s->device);
  cudaStream_t st = s->req_stream;
  if (s->h_cams_cap < ncams) {
    cudaFreeHost(s->h_cams);
    s->h_cams = nullptr;
    s->h_cams_cap = 0;
    if (cudaMallocHost(&s->h_cams, kCamDevBytes * ncams) != cudaSuccess) {
      cudaGetLastError();
      return VC_ERR_OOM;
    }
    s->h_cams_cap = ncams;
  }
  const uint32_t cap = v->n_bricks;
  const size_t sb = camera_scratch_bytes(*v, ncams), ob = 4ull * ncams * (1 + 2ull * cap);
  uint8_t *scratch = nullptr, *out = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&scratch), sb, st) != cudaSuccess ||
      cudaMallocAsync(reinterpret_cast<void**>(&out), ob, st) != cudaSuccess) {
    cudaGetLastError();
    if (scratch) cudaFreeAsync(scratch, st);
    return VC_ERR_OOM;
  }
  uint32_t* d_counts = reinterpret_cast<uint32_t*>(out);
  uint32_t* d_ids = d_counts + ncams;
  uint32_t* d_lods = d_ids + (size_t)ncams * cap;
  std::vector<uint32_t> counts(ncams);
  vc_status rc = launch_camera_requests(*v, cams, ncams, max_lod, cap, scratch, s->h_cams, d_counts, d_ids, d_lods, st);
  if (rc == VC_OK && (cudaMemcpyAsync(counts.data(), d_counts, 4ull * ncams, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                      cudaStreamSynchronize(st) != cudaSuccess))
    rc = VC_ERR_CUDA;
  std::vector<std::vector<uint32_t>> ids(ncams), lods(ncams);
  for (uint32_t i = 0; rc == VC_OK && i < ncams; ++i) {
    ids[i].resize(counts[i]);
    lods[i].resize(counts[i]);
    if (counts[i] &&
        (cudaMemcpyAsync(ids[i].data(), d_ids + (size_t)i * cap, 4ull * counts[i], cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaMemcpyAsync(lods[i].data(), d_lods + (size_t)i * cap, 4ull * counts[i], cudaMemcpyDeviceToHost, st) != cudaSuccess))
      rc = VC_ERR_CUDA;
  }
  if (rc == VC_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = VC_ERR_CUDA;
  cudaFreeAsync(scratch, st);
  cudaFreeAsync(out, st);
  for (uint32_t i = 0; rc == VC_OK && i < ncams; ++i)
    rc = submit(s, volume_index, ids[i].data(), lods[i].data(), counts[i], &request_ids_out[i]);
  return rc;
}

vc_status vc_poll(vc_server* srv, uint64_t request_id, int32_t* state, uint64_t* offsets_out) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || s->kind != kHandleServer || !state) return VC_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->requests.find(request_id);
  if (it == s->requests.end()) return VC_ERR_ARG;
  const Request& r = *it->second;
  *state = r.state;
  if (r.state == VC_REQ_FAILED) return r.status;
  if (offsets_out && r.state == VC_REQ_DONE) std::memcpy(offsets_out, r.offsets.data(), 8 * r.offsets.size());
  return VC_OK;
}

vc_status vc_wait(vc_server* srv, uint64_t request_id, uint32_t timeout_ms, int32_t* state) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || s->kind != kHandleServer || !state) return VC_ERR_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->requests.find(request_id);
  if (it == s->requests.end()) return VC_ERR_ARG;
  Request* r = it->second.get();
  const bool fin = s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), [&] {
    return r->state == VC_REQ_DONE || r->state == VC_REQ_FAILED;
  });
  *state = r->state;
  if (!fin) return VC_ERR_TIMEOUT;
  return r->state == VC_REQ_FAILED ? r->status : VC_OK;
}

vc_status vc_request_coarsest(vc_server* srv, uint64_t request_id, uint32_t* labels_dev, int32_t* status_dev,
                              void* cuda_stream) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || s->kind != kHandleServer || !labels_dev || !status_dev) return VC_ERR_ARG;
  std::vector<uint32_t> ids;
  Volume* v = nullptr;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->requests.find(request_id);
    if (it == s->requests.end()) return VC_ERR_ARG;
    ids = it->second->bricks;
    v = s->volumes[it->second->vol];
  }
  if (ids.empty()) return VC_OK;
  DeviceGuard g(s->device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  uint32_t* d_ids = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&d_ids), 4 * ids.size(), st) != cudaSuccess) {
    cudaGetLastError();
    return VC_ERR_OOM;
  }
  // the request's brick list is host memory owned here: copy it before this call returns
  vc_status rc = cudaMemcpyAsync(d_ids, ids.data(), 4 * ids.size(), cudaMemcpyHostToDevice, st) == cudaSuccess &&
                         cudaStreamSynchronize(st) == cudaSuccess
                     ? VC_OK
                     : VC_ERR_CUDA;
  if (rc == VC_OK) rc = launch_coarsest(*v, d_ids, (uint32_t)ids.size(), labels_dev, status_dev, st);
  cudaFreeAsync(d_ids, st);
  return rc;
}

vc_status vc_request_info_get(vc_server* srv, uint64_t request_id, vc_request_info* info) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || s->kind != kHandleServer || !info) return VC_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->requests.find(request_id);
  if (it == s->requests.end()) return VC_ERR_ARG;
  const Request& r = *it->second;
  std::memset(info, 0, sizeof(*info));
  info->state = r.state;
  info->status = r.status;
  info->volume_index = r.vol;
  info->n_bricks = (uint32_t)r.bricks.size();
  info->hits = r.hits;
  info->bytes = r.bytes;
  info->t_submit_ns = r.t_submit;
  info->t_admit_ns = r.t_admit;
  info->t_done_ns = r.t_done;
  return VC_OK;
}

vc_status vc_request_release(vc_server* srv, uint64_t request_id) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || s->kind != kHandleServer) return VC_ERR_ARG;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->requests.find(request_id);
    if (it == s->requests.end()) return VC_ERR_ARG;
    Request& r = *it->second;
    if (r.state == VC_REQ_ADMITTED || r.state == VC_REQ_WAITING) return VC_ERR_BUSY;
    for (uint32_t e : r.entries) s->cache->unpin(e);
    s->requests.erase(it);
    ++s->wake;
  }
  s->cv_work.notify_one();  // freed pins may let waiting requests in
  return VC_OK;
}

vc_status vc_server_cache(vc_server* srv, void** cache_dev, uint64_t* cache_bytes) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || s->kind != kHandleServer || !cache_dev || !cache_bytes) return VC_ERR_ARG;
  *cache_dev = s->d_cache;
  *cache_bytes = s->cache->capacity_bytes();
  return VC_OK;
}

vc_status vc_server_stats_get(vc_server* srv, vc_server_stats* out) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || s->kind != kHandleServer || !out) return VC_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->stats;
  out->cache_free_bytes = s->cache->free_bytes();
  out->cache_evictable_bytes = s->cache->evictable_bytes();
  out->cache_entries = s->cache->entries();
  out->evictions = s->cache->evictions();
  out->requests_waiting = s->waiting.size();
  out->batches_inflight = s->inflight.size();
  return VC_OK;
}

}  // extern "C"

namespace vc {
bool release_server(void* handle) {
  if (*static_cast<uint32_t*>(handle) != kHandleServer) return false;
  free_server(static_cast<Server*>(handle));
  return true;
}
}  // namespace vc
