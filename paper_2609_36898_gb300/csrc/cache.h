// Device brick cache bookkeeping (host side): which (volume, level of detail, brick) sits where in
// one device buffer, LRU eviction of unpinned entries, and all-or-nothing admission of a set of
// bricks. Paper: decoded bricks live in a GPU cache that is kept between frames; bricks that are
// no longer requested are freed and their space reused, and new bricks are assigned free cache
// space before they are decoded (Methods, "GPU rendering pipeline": request, provision, assign,
// decompress stages).
//
// Space is handed out by an 8-ary buddy allocator: a block of class c holds 4 * 8^c bytes, i.e. a
// (2^c)^3 brick of uint32 labels, and splits into the 8 blocks of class c - 1, mirroring the 2^3
// hierarchy of the bricks' levels of detail. Every block starts at a multiple of its own size, so
// (block offset / block bytes) is the slot index a decode call needs.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

namespace vc {

// Open-addressing hash map from 64-bit keys (never ~0) to 32-bit values: linear probing,
// backward-shift deletion, power-of-two capacity kept at most half full.
class FlatMap {
 public:
  static constexpr uint64_t kEmpty = ~0ull;
  static constexpr uint32_t kMissing = 0xFFFFFFFFu;
  FlatMap() { rehash(64); }
  uint32_t find(uint64_t k) const {
    for (uint64_t i = home(k);; i = (i + 1) & mask_) {
      if (keys_[i] == k) return vals_[i];
      if (keys_[i] == kEmpty) return kMissing;
    }
  }
  void put(uint64_t k, uint32_t v) {
    if (2 * (size_ + 1) > keys_.size()) rehash(2 * keys_.size());
    uint64_t i = home(k);
    while (keys_[i] != kEmpty && keys_[i] != k) i = (i + 1) & mask_;
    if (keys_[i] == kEmpty) ++size_;
    keys_[i] = k;
    vals_[i] = v;
  }
  bool erase(uint64_t k) {
    uint64_t i = home(k);
    while (keys_[i] != k) {
      if (keys_[i] == kEmpty) return false;
      i = (i + 1) & mask_;
    }
    for (uint64_t j = i;;) {  // pull later members of the probe run back into the hole
      j = (j + 1) & mask_;
      if (keys_[j] == kEmpty) break;
      const uint64_t h = home(keys_[j]);
      const bool movable = i <= j ? (h <= i || h > j) : (h <= i && h > j);
      if (movable) {
        keys_[i] = keys_[j];
        vals_[i] = vals_[j];
        i = j;
      }
    }
    keys_[i] = kEmpty;
    --size_;
    return true;
  }
  void clear() {
    std::fill(keys_.begin(), keys_.end(), kEmpty);
    size_ = 0;
  }
  size_t size() const { return size_; }

 private:
  uint64_t home(uint64_t k) const { return (k * 0x9E3779B97F4A7C15ull) >> shift_; }
  void rehash(size_t cap) {
    std::vector<uint64_t> ok;
    std::vector<uint32_t> ov;
    ok.swap(keys_);
    ov.swap(vals_);
    keys_.assign(cap, kEmpty);
    vals_.assign(cap, 0);
    mask_ = cap - 1;
    shift_ = 64;
    for (size_t c = cap; c > 1; c >>= 1) --shift_;
    size_ = 0;
    for (size_t i = 0; i < ok.size(); ++i)
      if (ok[i] != kEmpty) put(ok[i], ov[i]);
  }
  std::vector<uint64_t> keys_;
  std::vector<uint32_t> vals_;
  uint64_t mask_ = 0;
  uint32_t shift_ = 64;
  size_t size_ = 0;
};

class BrickCache {
 public:
  static constexpr uint32_t kNone = 0xFFFFFFFFu;

  // bytes: usable bytes (rounded down to whole blocks of max_cls); min_cls <= max_cls <= 9.
  BrickCache(uint64_t bytes, uint32_t min_cls, uint32_t max_cls);

  struct Ref {
    uint32_t entry;   // entry index (pinned until unpin)
    uint64_t offset;  // byte offset of the block in the device buffer
    bool hit;         // already present (resident or being decoded by earlier work)
  };

  // Pins an entry for every key (class cls[i], raised to min_cls), allocating blocks for the keys
  // that are not present and evicting least recently used unpinned entries as needed. All or
  // nothing: if the keys cannot all be placed, every pin and allocation made by this call is
  // undone and false is returned (entries evicted on the way stay evicted). Duplicate keys pin
  // the same entry twice.
  bool acquire(const uint64_t* keys, const uint32_t* cls, uint32_t n, Ref* out);
  // Drops one pin; an entry with no pins becomes the most recently used evictable entry, or is
  // removed at once if it was marked invalid.
  void unpin(uint32_t entry);
  // Marks an entry invalid (its decode failed): it is removed when its last pin is dropped and is
  // never returned as a hit.
  void invalidate(uint32_t entry);

  // per-entry payload for the server: the work sequence number that makes the entry resident
  uint64_t& ready_seq(uint32_t entry) { return entries_[entry].ready_seq; }
  uint32_t entry_class(uint32_t entry) const { return entries_[entry].cls; }
  uint64_t entry_key(uint32_t entry) const { return entries_[entry].key; }

  uint64_t capacity_bytes() const { return capacity_; }
  uint64_t free_bytes() const { return free_bytes_; }
  uint64_t evictable_bytes() const { return evictable_bytes_; }
  uint64_t entries() const { return map_.size(); }
  uint64_t evictions() const { return evictions_; }
  uint64_t hits() const { return hits_; }
  uint64_t misses() const { return misses_; }
  uint32_t min_class() const { return min_cls_; }
  uint32_t max_class() const { return max_cls_; }
  static uint64_t block_bytes(uint32_t c) { return uint64_t(4) << (3 * c); }

 private:
  enum : uint8_t { kAbsent = 0, kFree = 1, kUsed = 2, kSplit = 3 };
  struct Level {
    std::vector<uint8_t> state;     // per block of this class
    std::vector<uint8_t> nfree;     // per block, while split: free children
    std::vector<uint32_t> list;     // free blocks (may hold stale indices; state decides)
    uint64_t n_free = 0;
  };
  struct Entry {
    uint64_t key = 0;
    uint64_t ready_seq = 0;
    uint32_t cls = 0, block = 0, pins = 0;
    int32_t prev = -1, next = -1;   // LRU links (only while pins == 0)
    bool valid = true;
  };

  uint32_t alloc(uint32_t c);
  void release_block(uint32_t c, uint32_t idx);
  void lru_push_front(uint32_t e);
  void lru_remove(uint32_t e);
  bool evict_one();
  void remove_entry(uint32_t e);
  Level& lv(uint32_t c) { return levels_[c - min_cls_]; }

  uint64_t capacity_ = 0, free_bytes_ = 0, evictable_bytes_ = 0;
  uint64_t evictions_ = 0, hits_ = 0, misses_ = 0;
  uint32_t min_cls_, max_cls_, n_top_ = 0;
  std::vector<Level> levels_;
  std::vector<Entry> entries_;
  std::vector<uint32_t> free_entries_;
  FlatMap map_;
  // scratch of acquire(): duplicate misses, per-key lookups, per-entry marks, pass order
  FlatMap seen_;
  std::vector<uint32_t> found_, mark_, order_;
  std::vector<Ref> tmp_;
  std::vector<uint8_t> tmp_created_;
  uint32_t epoch_ = 0;
  int32_t lru_head_ = -1, lru_tail_ = -1;
};

}  // namespace vc
