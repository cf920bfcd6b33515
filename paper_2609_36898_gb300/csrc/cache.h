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

#include <unordered_map>
#include <vector>

namespace vc {

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
  std::unordered_map<uint64_t, uint32_t> map_;
  int32_t lru_head_ = -1, lru_tail_ = -1;
};

}  // namespace vc
