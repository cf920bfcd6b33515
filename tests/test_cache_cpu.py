"""Host-side checks of the serving cache bookkeeping (buddy allocator, LRU, admission) through the
C ABI; no GPU is touched."""
import numpy as np
import pytest

import paper_2609_36898_gb300 as vc


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2609_36898_gb300 import build
    build.build()
    return vc._lib_handle()


def block(c):
    return 4 << (3 * c)


def live_blocks_disjoint(spans, capacity):
    spans = sorted(spans)
    for (a0, a1), (b0, _) in zip(spans, spans[1:]):
        assert a1 <= b0, "two live blocks overlap"
    assert all(0 <= a and b <= capacity for a, b in spans)


def test_blocks_are_aligned_disjoint_and_counted():
    c = vc.vc_brick_cache_create(8 * block(5), 2, 5)
    rng = np.random.default_rng(0)
    keys = np.arange(1, 60, dtype=np.uint64)
    cls = rng.integers(2, 6, size=keys.size).astype(np.uint32)
    live = {}
    for k, cl in zip(keys, cls):
        r = vc.vc_brick_cache_acquire(c, [k], [cl])
        if r is None:
            continue
        e, off, hit = r
        assert not hit[0]
        assert off[0] % block(cl) == 0
        live[int(k)] = (int(off[0]), int(off[0]) + block(cl))
    live_blocks_disjoint(list(live.values()), 8 * block(5))
    st = vc.vc_brick_cache_stats_get(c)
    used = sum(b - a for a, b in live.values())
    assert st.free_bytes == st.capacity_bytes - used
    assert st.entries == len(live) and st.evictable_bytes == 0  # all pinned
    vc.vc_release(c)


def test_admission_is_all_or_nothing_and_pins_block_eviction():
    c = vc.vc_brick_cache_create(4 * block(4), 2, 4)
    a = vc.vc_brick_cache_acquire(c, [1, 2, 3], [4, 4, 4])
    assert a is not None
    # two more top blocks do not fit while 1..3 are pinned: nothing changes
    before = vc.vc_brick_cache_stats_get(c)
    assert vc.vc_brick_cache_acquire(c, [10, 11], [4, 4]) is None
    after = vc.vc_brick_cache_stats_get(c)
    assert (before.free_bytes, before.entries, before.evictions) == (after.free_bytes, after.entries, after.evictions)
    # one fits
    b = vc.vc_brick_cache_acquire(c, [10], [4])
    assert b is not None
    # unpin 2: now it is evictable and the next request takes its block
    vc.vc_brick_cache_unpin(c, [a[0][1]])
    r = vc.vc_brick_cache_acquire(c, [11], [4])
    assert r is not None and r[1][0] == a[1][1]
    assert vc.vc_brick_cache_stats_get(c).evictions == 1
    vc.vc_release(c)


def test_lru_evicts_least_recently_unpinned_first():
    c = vc.vc_brick_cache_create(3 * block(3), 2, 3)
    ents = {}
    for k in (1, 2, 3):
        e, off, _ = vc.vc_brick_cache_acquire(c, [k], [3])
        ents[k] = (int(e[0]), int(off[0]))
    for k in (2, 1, 3):  # unpin order = recency order: 2 oldest
        vc.vc_brick_cache_unpin(c, [ents[k][0]])
    # a hit on 2 makes it most recent; 1 is now the oldest
    e2, _, hit = vc.vc_brick_cache_acquire(c, [2], [3])
    assert hit[0]
    vc.vc_brick_cache_unpin(c, e2)
    e4, off4, hit4 = vc.vc_brick_cache_acquire(c, [4], [3])
    assert not hit4[0] and off4[0] == ents[1][1]
    # 1 is gone, 2 and 3 remain
    assert vc.vc_brick_cache_acquire(c, [1], [3]) is not None  # evicts 3 (oldest unpinned)
    _, _, h2 = vc.vc_brick_cache_acquire(c, [2], [3]) or (None, None, [False])
    assert h2[0]
    vc.vc_release(c)


def test_duplicates_and_hits_share_one_entry():
    c = vc.vc_brick_cache_create(2 * block(3), 2, 3)
    e, off, hit = vc.vc_brick_cache_acquire(c, [5, 5, 6], [3, 3, 3])
    assert e[0] == e[1] and off[0] == off[1] and e[0] != e[2]
    assert list(hit) == [False, True, False]
    st = vc.vc_brick_cache_stats_get(c)
    assert st.entries == 2 and st.free_bytes == 0
    # 5 is pinned twice: one unpin leaves it pinned, so a new key cannot evict it
    vc.vc_brick_cache_unpin(c, [e[0], e[2]])
    r = vc.vc_brick_cache_acquire(c, [7], [3])
    assert r is not None and r[1][0] == off[2]
    assert vc.vc_brick_cache_acquire(c, [8], [3]) is None
    vc.vc_release(c)


def test_buddies_merge_back_into_large_blocks():
    c = vc.vc_brick_cache_create(block(5), 2, 5)
    keys = np.arange(1, 1 + 8 * 8 * 8, dtype=np.uint64)  # fill with the smallest class
    e, off, _ = vc.vc_brick_cache_acquire(c, keys, [2])
    assert sorted(off.tolist()) == [block(2) * i for i in range(512)]
    assert vc.vc_brick_cache_acquire(c, [9999], [5]) is None
    vc.vc_brick_cache_unpin(c, e)
    # all small entries are evictable: the big block needs every one of them evicted and merged
    r = vc.vc_brick_cache_acquire(c, [9999], [5])
    assert r is not None and r[1][0] == 0
    st = vc.vc_brick_cache_stats_get(c)
    assert st.evictions == 512 and st.entries == 1 and st.free_bytes == 0
    vc.vc_release(c)


def test_invalidated_entry_is_never_a_hit():
    c = vc.vc_brick_cache_create(4 * block(3), 2, 3)
    e, off, _ = vc.vc_brick_cache_acquire(c, [1], [3])
    vc.vc_brick_cache_invalidate(c, int(e[0]))
    e2, off2, hit2 = vc.vc_brick_cache_acquire(c, [1], [3])
    assert not hit2[0] and e2[0] != e[0]
    vc.vc_brick_cache_unpin(c, e)  # the invalid entry is freed with its last pin
    st = vc.vc_brick_cache_stats_get(c)
    assert st.entries == 1 and st.free_bytes == 3 * block(3)
    vc.vc_release(c)


def test_random_workload_keeps_invariants():
    """Against a plain model: live pinned sets never overlap, bytes add up, and a request that the
    model says fits (needed <= free + evictable) is admitted unless fragmentation blocks it."""
    rng = np.random.default_rng(3)
    cap = 16 * block(5)
    c = vc.vc_brick_cache_create(cap, 2, 5)
    held = []  # (entries, spans)
    pinned_bytes = {}
    for step in range(400):
        if held and (rng.random() < 0.45 or len(held) > 12):
            ents, _ = held.pop(int(rng.integers(len(held))))
            vc.vc_brick_cache_unpin(c, ents)
            continue
        n = int(rng.integers(1, 20))
        keys = rng.integers(1, 300, size=n).astype(np.uint64)
        cls = (keys % 4 + 2).astype(np.uint32)  # a key always has the same class
        r = vc.vc_brick_cache_acquire(c, keys, cls)
        if r is None:
            continue
        ents, offs, _ = r
        spans = [(int(o), int(o) + block(int(cl))) for o, cl in zip(offs, cls)]
        held.append((ents, spans))
        all_spans = {}
        for es, sp in held:
            for e_, s_ in zip(es, sp):
                all_spans[int(e_)] = s_
        live_blocks_disjoint(list(all_spans.values()), cap)
        st = vc.vc_brick_cache_stats_get(c)
        assert st.free_bytes + st.evictable_bytes + sum(b - a for a, b in all_spans.values()) == cap
    for ents, _ in held:
        vc.vc_brick_cache_unpin(c, ents)
    st = vc.vc_brick_cache_stats_get(c)
    assert st.free_bytes + st.evictable_bytes == cap
    vc.vc_release(c)
