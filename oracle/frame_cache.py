"""Frame cache oracle: one frame of the cache stages of the paper's GPU rendering pipeline, on
counts and per-brick states, in plain Python. TEST INFRASTRUCTURE ONLY (tests and the smoke check);
it shares no code with the GPU library.

Paper, Methods "GPU rendering pipeline":
  - Request: one thread per brick; newly visible bricks go onto the request stack of their level of
    detail, bricks in the cache that are no longer visible go onto a free stack;
  - Provision: if a level's free stack cannot serve all of that level's requests, new space is
    taken from the end of the cache buffer by moving its top;
  - Assign: newly visible bricks get free regions, from the free stacks or from the top; Decode
    then fills them.
Methods "Cache defragmentation": a region belongs to its level for good once allocated (freed
regions go onto that level's free stack); a free stack has a fixed capacity (1,048,576 entries in
the paper) and a region freed onto a full stack is left as dead space; the cache is reset once for
defragmentation when its capacity is exceeded. Methods "Memory management": a brick one level
coarser takes 8 times less memory.

Readings (the same in the library): a brick visible at another level than the one it is cached at
is freed from its old level and requested at the new one; levels are provisioned finest first; a
level's regions start at multiples of their size (the top is rounded up, the gap counted as dead);
at most `per_frame` bricks are assigned per frame (the rest stay requested-but-unassigned and are
requested again while visible); the reset happens at the start of the next frame, only if the space
held by other levels' free regions, dead regions and the rest of the buffer adds up to what was
missing, and never in two frames in a row.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

NONE = 255


def region(L: int, level: int) -> int:
    """Labels in a region of the given level of detail: (2^(L - level))^3."""
    return 8 ** (L - level)


@dataclass
class FrameState:
    """What a frame leaves for the next: each brick's cached level (NONE = not cached), the free
    stacks' entry counts per level, the top of the buffer, the dead labels, a pending reset."""
    lods: np.ndarray
    free_n: list = field(default_factory=list)
    top: int = 0
    dead: int = 0
    reset_pending: bool = False


def empty_state(n_bricks: int, L: int) -> FrameState:
    return FrameState(np.full(n_bricks, NONE, np.uint8), [0] * (L + 1), 0, 0, False)


def update(state: FrameState, want: np.ndarray, L: int, max_lod: int, cap: int, per_frame: int,
           free_cap: int) -> dict:
    """One frame. want[b] = the level brick b is visible at this frame (NONE = not visible).
    Returns the frame's sets and counts; 'assign_n' / 'requested_at' give, per level, how many of
    the requested bricks get a region (which ones is not fixed by the stages)."""
    nlev = min(max_lod, L) + 1
    lods = state.lods.copy()
    free_n = list(state.free_n)
    top, dead = state.top, state.dead
    in_reset = state.reset_pending
    if in_reset:  # defragmentation: every region is given up
        lods[:] = NONE
        free_n = [0] * (L + 1)
        top = dead = 0
    want = np.asarray(want, np.uint8)
    vis = want != NONE
    # Request
    freed = (lods != NONE) & (lods != want)
    requested = vis & (lods != want)
    resident = vis & (lods == want)
    for lev in range(L + 1):
        k = int(np.count_nonzero(freed & (lods == lev)))
        over = max(0, free_n[lev] + k - free_cap) - max(0, free_n[lev] - free_cap)
        dead += over * region(L, lev)
        free_n[lev] += k
    lods_after_free = np.where(freed, NONE, lods).astype(np.uint8)
    requested_at = [np.flatnonzero(requested & (want == lev)) for lev in range(L + 1)]
    # Provision
    left = per_frame
    assign_n, take_n = [0] * (L + 1), [0] * (L + 1)
    missing = 0
    overflow = False
    for lev in range(nlev):
        sz = region(L, lev)
        avail = min(free_n[lev], free_cap)
        w = min(len(requested_at[lev]), per_frame, left)
        take = min(w, avail)
        need = w - take
        at = -(-top // sz) * sz
        room = (cap - at) // sz if at < cap else 0
        from_top = min(need, room)
        if from_top < need:
            overflow = True
            missing += (need - from_top) * sz
        if from_top:
            dead += at - top
            top = at + from_top * sz
        free_n[lev] = avail - take
        take_n[lev] = take
        assign_n[lev] = take + from_top
        left -= take + from_top
    reset_pending = False
    if overflow and not in_reset:
        spare = dead + (cap - top) + sum(free_n[lev] * region(L, lev) for lev in range(nlev))
        reset_pending = spare >= missing
    return {
        "in_reset": in_reset, "freed": np.flatnonzero(freed), "resident": np.flatnonzero(resident),
        "requested": np.flatnonzero(requested), "requested_at": requested_at, "assign_n": assign_n,
        "take_n": take_n, "switches": int(np.count_nonzero(freed & vis)),
        "lods_after_free": lods_after_free, "free_n": free_n, "top": top, "dead": dead,
        "reset_pending": reset_pending,
    }


def next_state(result: dict, lods_after: np.ndarray) -> FrameState:
    """The state after a frame, given the bricks' levels after Assign (which requested bricks got
    regions is the implementation's choice; the counts are the oracle's)."""
    return FrameState(np.asarray(lods_after, np.uint8).copy(), list(result["free_n"]), result["top"],
                      result["dead"], result["reset_pending"])


def assign_first(result: dict) -> np.ndarray:
    """Levels after Assign when each level's first requests (ascending id) get the regions."""
    lods = result["lods_after_free"].copy()
    for lev, ids in enumerate(result["requested_at"]):
        lods[ids[:result["assign_n"][lev]]] = lev
    return lods
