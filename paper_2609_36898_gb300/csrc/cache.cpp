// Brick cache bookkeeping: 8-ary buddy allocator, LRU of unpinned entries, all-or-nothing admission.
#include "cache.h"

#include <algorithm>

namespace vc {

BrickCache::BrickCache(uint64_t bytes, uint32_t min_cls, uint32_t max_cls)
    : min_cls_(min_cls), max_cls_(max_cls) {
  const uint64_t top = block_bytes(max_cls);
  n_top_ = (uint32_t)std::min<uint64_t>(bytes / top, 0xFFFFFFFFull >> (3 * (max_cls - min_cls)));
  capacity_ = n_top_ * top;
  free_bytes_ = capacity_;
  levels_.resize(max_cls - min_cls + 1);
  for (uint32_t c = min_cls; c <= max_cls; ++c) {
    const uint64_t nb = (uint64_t)n_top_ << (3 * (max_cls - c));
    lv(c).state.assign(nb, kAbsent);
    lv(c).nfree.assign(c > min_cls ? nb : 0, 0);
  }
  Level& t = lv(max_cls);
  for (uint32_t i = 0; i < n_top_; ++i) t.state[i] = kFree;
  for (uint32_t i = n_top_; i-- > 0;) t.list.push_back(i);
  t.n_free = n_top_;
}

uint32_t BrickCache::alloc(uint32_t c) {
  Level& L = lv(c);
  while (!L.list.empty()) {
    const uint32_t idx = L.list.back();
    L.list.pop_back();
    if (L.state[idx] != kFree) continue;  // stale (merged or reallocated)
    L.state[idx] = kUsed;
    --L.n_free;
    if (c < max_cls_) --lv(c + 1).nfree[idx >> 3];
    return idx;
  }
  if (c == max_cls_) return kNone;
  const uint32_t p = alloc(c + 1);  // split a block of the next class
  if (p == kNone) return kNone;
  Level& U = lv(c + 1);
  U.state[p] = kSplit;
  U.nfree[p] = 7;
  const uint32_t first = 8u * p;
  for (uint32_t k = 8; k-- > 1;) {
    L.state[first + k] = kFree;
    L.list.push_back(first + k);
  }
  L.n_free += 7;
  L.state[first] = kUsed;
  return first;
}

void BrickCache::release_block(uint32_t c, uint32_t idx) {
  Level& L = lv(c);
  L.state[idx] = kFree;
  ++L.n_free;
  if (c < max_cls_) {
    const uint32_t p = idx >> 3;
    if (++lv(c + 1).nfree[p] == 8) {  // all 8 buddies free: merge into the parent block
      for (uint32_t k = 0; k < 8; ++k) L.state[8u * p + k] = kAbsent;
      L.n_free -= 8;
      lv(c + 1).nfree[p] = 0;
      release_block(c + 1, p);
      return;
    }
  }
  L.list.push_back(idx);
  if (L.list.size() > 2 * L.n_free + 4096) {  // drop stale indices now and then
    std::vector<uint32_t> keep;
    keep.reserve(L.n_free);
    for (uint32_t i : L.list)
      if (L.state[i] == kFree) keep.push_back(i);
    std::sort(keep.begin(), keep.end());
    keep.erase(std::unique(keep.begin(), keep.end()), keep.end());
    std::reverse(keep.begin(), keep.end());
    L.list.swap(keep);
  }
}

void BrickCache::lru_push_front(uint32_t e) {
  Entry& E = entries_[e];
  E.prev = -1;
  E.next = lru_head_;
  if (lru_head_ >= 0) entries_[lru_head_].prev = (int32_t)e;
  lru_head_ = (int32_t)e;
  if (lru_tail_ < 0) lru_tail_ = (int32_t)e;
  evictable_bytes_ += block_bytes(E.cls);
}

void BrickCache::lru_remove(uint32_t e) {
  Entry& E = entries_[e];
  if (E.prev >= 0) entries_[E.prev].next = E.next; else lru_head_ = E.next;
  if (E.next >= 0) entries_[E.next].prev = E.prev; else lru_tail_ = E.prev;
  E.prev = E.next = -1;
  evictable_bytes_ -= block_bytes(E.cls);
}

void BrickCache::remove_entry(uint32_t e) {
  Entry& E = entries_[e];
  if (map_.find(E.key) == e) map_.erase(E.key);
  release_block(E.cls, E.block);
  free_bytes_ += block_bytes(E.cls);
  E = Entry();
  free_entries_.push_back(e);
}

bool BrickCache::evict_one() {
  if (lru_tail_ < 0) return false;
  const uint32_t e = (uint32_t)lru_tail_;
  lru_remove(e);
  remove_entry(e);
  ++evictions_;
  return true;
}

bool BrickCache::acquire(const uint64_t* keys, const uint32_t* cls, uint32_t n, Ref* out) {
  // one lookup per key: the entries already present (hits) are remembered for the passes below
  found_.resize(n);
  if (++epoch_ == 0) {  // after 2^32 calls: old marks could match again
    std::fill(mark_.begin(), mark_.end(), 0u);
    epoch_ = 1;
  }
  if (mark_.size() < entries_.size()) mark_.resize(entries_.size(), 0);
  // admission: the missing keys' bytes must fit in free + evictable bytes, not counting the
  // evictable entries this call will pin as hits (each distinct key counted once)
  uint64_t need = 0, hit_evictable = 0;
  uint32_t n_hits = 0;
  bool seen_used = false;
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t c = std::max(cls[i], min_cls_);
    if (c > max_cls_) return false;
    const uint32_t e = map_.find(keys[i]);
    found_[i] = e;
    if (e != FlatMap::kMissing) {
      ++n_hits;
      if (mark_[e] != epoch_) {
        mark_[e] = epoch_;
        if (entries_[e].pins == 0) hit_evictable += block_bytes(entries_[e].cls);
      }
    } else {
      if (!seen_used) {
        seen_.clear();
        seen_used = true;
      }
      if (seen_.find(keys[i]) != FlatMap::kMissing) continue;
      seen_.put(keys[i], 0);
      need += block_bytes(c);
    }
  }
  if (need > free_bytes_ + evictable_bytes_ - hit_evictable) return false;

  // hits first, so that the evictions below cannot take them
  uint32_t done = 0;
  order_.resize(n);
  {
    uint32_t h = 0, m = n_hits;
    for (uint32_t i = 0; i < n; ++i) order_[found_[i] != FlatMap::kMissing ? h++ : m++] = i;
  }
  tmp_.resize(n);
  tmp_created_.assign(n, 0);
  auto undo = [&]() {
    for (uint32_t j = done; j-- > 0;) {
      const uint32_t e = tmp_[j].entry;
      Entry& E = entries_[e];
      if (--E.pins == 0) {
        if (tmp_created_[j] || !E.valid) remove_entry(e);
        else lru_push_front(e);
      }
    }
  };
  for (; done < n; ++done) {
    const uint32_t i = order_[done];
    const uint32_t c = std::max(cls[i], min_cls_);
    // a hit from the first pass, or a key created earlier in this pass (a duplicate miss)
    const uint32_t hit_e = done < n_hits ? found_[i] : map_.find(keys[i]);
    if (hit_e != FlatMap::kMissing) {
      const uint32_t e = hit_e;
      Entry& E = entries_[e];
      if (E.pins++ == 0) lru_remove(e);
      tmp_[done] = Ref{e, (uint64_t)E.block * block_bytes(E.cls), true};
      continue;
    }
    uint32_t blk;
    while ((blk = alloc(c)) == kNone) {
      if (!evict_one()) {
        undo();
        return false;
      }
    }
    free_bytes_ -= block_bytes(c);
    uint32_t e;
    if (!free_entries_.empty()) {
      e = free_entries_.back();
      free_entries_.pop_back();
    } else {
      e = (uint32_t)entries_.size();
      entries_.emplace_back();
    }
    Entry& E = entries_[e];
    E = Entry();
    E.key = keys[i];
    E.cls = c;
    E.block = blk;
    E.pins = 1;
    E.ready_seq = ~0ull;  // not decoded yet
    map_.put(keys[i], e);
    tmp_[done] = Ref{e, (uint64_t)blk * block_bytes(c), false};
    tmp_created_[done] = 1;
  }
  for (uint32_t j = 0; j < n; ++j) {
    out[order_[j]] = tmp_[j];
    if (tmp_[j].hit) ++hits_; else ++misses_;
  }
  return true;
}

void BrickCache::unpin(uint32_t e) {
  Entry& E = entries_[e];
  if (E.pins == 0) return;
  if (--E.pins == 0) {
    if (!E.valid) remove_entry(e);
    else lru_push_front(e);
  }
}

void BrickCache::invalidate(uint32_t e) {
  Entry& E = entries_[e];
  E.valid = false;
  if (map_.find(E.key) == e) map_.erase(E.key);
  if (E.pins == 0) {
    lru_remove(e);
    // removed from the map already: release the block and the entry
    release_block(E.cls, E.block);
    free_bytes_ += block_bytes(E.cls);
    E = Entry();
    free_entries_.push_back(e);
  }
}

}  // namespace vc

// ---- host-only C ABI over BrickCache (the server's bookkeeping, exposed for inspection) ----
#include <new>

#include "vc_internal.h"

namespace {
struct CacheHandle {
  uint32_t kind = vc::kHandleCache;
  vc::BrickCache cache;
  CacheHandle(uint64_t b, uint32_t lo, uint32_t hi) : cache(b, lo, hi) {}
};
CacheHandle* as_cache(vc_brick_cache* h) {
  CacheHandle* c = reinterpret_cast<CacheHandle*>(h);
  return c && c->kind == vc::kHandleCache ? c : nullptr;
}
}  // namespace

namespace vc {
bool release_cache(void* handle) {
  if (*static_cast<uint32_t*>(handle) != kHandleCache) return false;
  CacheHandle* c = static_cast<CacheHandle*>(handle);
  c->kind = 0;
  delete c;
  return true;
}
}  // namespace vc

extern "C" {

vc_status vc_brick_cache_create(uint64_t bytes, uint32_t min_class, uint32_t max_class, vc_brick_cache** out) {
  if (!out) return VC_ERR_ARG;
  *out = nullptr;
  if (min_class > max_class || max_class > 9 || bytes < vc::BrickCache::block_bytes(max_class)) return VC_ERR_ARG;
  if ((bytes / vc::BrickCache::block_bytes(max_class)) << (3 * (max_class - min_class)) > (1ull << 31))
    return VC_ERR_ARG;  // too many small blocks for the bookkeeping
  CacheHandle* c = nullptr;
  try {
    c = new CacheHandle(bytes, min_class, max_class);
  } catch (...) {
    return VC_ERR_OOM;
  }
  *out = reinterpret_cast<vc_brick_cache*>(c);
  return VC_OK;
}

vc_status vc_brick_cache_acquire(vc_brick_cache* h, const uint64_t* keys, const uint32_t* classes, uint32_t n,
                                 uint32_t* entries_out, uint64_t* offsets_out, uint8_t* hits_out) {
  CacheHandle* c = as_cache(h);
  if (!c || (n && (!keys || !classes || !entries_out || !offsets_out || !hits_out))) return VC_ERR_ARG;
  std::vector<vc::BrickCache::Ref> refs(n);
  if (!c->cache.acquire(keys, classes, n, refs.data())) return VC_ERR_BUSY;
  for (uint32_t i = 0; i < n; ++i) {
    entries_out[i] = refs[i].entry;
    offsets_out[i] = refs[i].offset;
    hits_out[i] = refs[i].hit ? 1 : 0;
  }
  return VC_OK;
}

vc_status vc_brick_cache_unpin(vc_brick_cache* h, const uint32_t* entries, uint32_t n) {
  CacheHandle* c = as_cache(h);
  if (!c || (n && !entries)) return VC_ERR_ARG;
  for (uint32_t i = 0; i < n; ++i) c->cache.unpin(entries[i]);
  return VC_OK;
}

vc_status vc_brick_cache_invalidate(vc_brick_cache* h, uint32_t entry) {
  CacheHandle* c = as_cache(h);
  if (!c) return VC_ERR_ARG;
  c->cache.invalidate(entry);
  return VC_OK;
}

vc_status vc_brick_cache_stats_get(vc_brick_cache* h, vc_brick_cache_stats* out) {
  CacheHandle* c = as_cache(h);
  if (!c || !out) return VC_ERR_ARG;
  out->capacity_bytes = c->cache.capacity_bytes();
  out->free_bytes = c->cache.free_bytes();
  out->evictable_bytes = c->cache.evictable_bytes();
  out->entries = c->cache.entries();
  out->evictions = c->cache.evictions();
  out->hits = c->cache.hits();
  out->misses = c->cache.misses();
  return VC_OK;
}

}  // extern "C"
