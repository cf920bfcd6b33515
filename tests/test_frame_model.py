"""Pins of the frame cache oracle (oracle/frame_cache.py) on hand-worked frames of the cache stages
(Methods, "GPU rendering pipeline": request / provision / assign; "Cache defragmentation": regions
keep their level when free, a full free stack leaves a region dead, a reset when the capacity is
exceeded). Every expected number below is worked out from those rules by hand, in the comments."""
import numpy as np

from oracle import frame_cache as fm

N = fm.NONE


def _frame(state, want, **cfg):
    r = fm.update(state, np.asarray(want, np.uint8), **cfg)
    return r, fm.next_state(r, fm.assign_first(r))


def test_regions_scale_by_eight_per_level():
    assert [fm.region(5, k) for k in range(6)] == [32768, 4096, 512, 64, 8, 1]


def test_worked_frames_top_free_stack_switch_and_reset():
    cfg = dict(L=1, max_lod=1, cap=40, per_frame=100, free_cap=4)  # level 0: 8 labels, level 1: 1
    s = fm.empty_state(6, 1)
    # frame 1: bricks 0, 1, 2 at level 0 and 4 at level 1 are new: 3 regions of 8 from the top
    # (top 24), then one of 1 (top 25)
    r, s = _frame(s, [0, 0, 0, N, 1, N], **cfg)
    assert r["assign_n"][:2] == [3, 1] and r["take_n"][:2] == [0, 0]
    assert (r["top"], r["dead"], r["reset_pending"]) == (25, 0, False)
    assert list(s.lods) == [0, 0, 0, N, 1, N]
    # frame 2: brick 1 leaves (its region onto level 0's stack), brick 3 arrives at level 0, brick 4
    # switches 1 -> 0 (freed onto level 1's stack, requested at 0). Level 0: 2 requests, 1 from
    # the stack, 1 from the top rounded up from 25 to 32 (7 dead): top 40
    r, s = _frame(s, [0, N, 0, 0, 0, N], **cfg)
    assert list(r["freed"]) == [1, 4] and list(r["resident"]) == [0, 2] and r["switches"] == 1
    assert list(r["requested_at"][0]) == [3, 4]
    assert r["assign_n"][:2] == [2, 0] and r["take_n"][:2] == [1, 0]
    assert (r["top"], r["dead"], r["free_n"][:2]) == (40, 7, [0, 1])
    # frame 3: bricks 1 and 5 arrive at level 0; the stack is empty and the top is at capacity:
    # 16 labels are missing, and only 7 dead + 1 free at level 1 could be regained: no reset
    r3, s3 = _frame(s, [0] * 6, **cfg)
    assert r3["assign_n"][:2] == [0, 0] and len(r3["requested"]) == 2
    assert r3["reset_pending"] is False and (r3["top"], r3["dead"]) == (40, 7)
    # frame 3 instead: every brick at level 1. Bricks 0, 2, 3, 4 free their level-0 regions (the
    # stack takes all 4); 6 requests at level 1: 1 from its stack, 5 missing at the top. Spare =
    # 7 dead + 4 x 8 free at level 0 = 39 >= 5: the next frame resets
    r, s = _frame(s, [1] * 6, **cfg)
    assert r["assign_n"][:2] == [0, 1] and r["free_n"][:2] == [4, 0]
    assert r["reset_pending"] is True
    # frame 4: the reset empties everything; the 6 bricks get level-1 regions 0..5 from the top
    r, s = _frame(s, [1] * 6, **cfg)
    assert r["in_reset"] is True and r["assign_n"][:2] == [0, 6]
    assert (r["top"], r["dead"], r["free_n"][:2], r["reset_pending"]) == (6, 0, [0, 0], False)
    assert list(s.lods) == [1] * 6


def test_no_reset_in_two_frames_in_a_row():
    cfg = dict(L=1, max_lod=1, cap=16, per_frame=100, free_cap=8)
    s = fm.empty_state(4, 1)
    r, s = _frame(s, [0, 0, N, N], **cfg)            # top 16 = capacity
    r, s = _frame(s, [N, N, 0, 0], **cfg)            # 2 freed, 2 taken from the stack
    assert r["take_n"][0] == 2 and r["top"] == 16
    r, s = _frame(s, [1, 1, 1, 1], **cfg)            # 2 freed at 0; 4 at level 1 from a full top
    assert r["assign_n"][:2] == [0, 0] and r["reset_pending"] is True  # spare 2 x 8 >= 4
    r, s = _frame(s, [0, 0, 0, 0, ], **cfg)          # the reset frame: 2 of 4 fit (16 / 8)
    assert r["in_reset"] and r["assign_n"][0] == 2 and r["reset_pending"] is False  # not twice in a row


def test_full_free_stack_leaves_dead_regions():
    cfg = dict(L=1, max_lod=0, cap=64, per_frame=100, free_cap=1)
    s = fm.empty_state(4, 1)
    r, s = _frame(s, [0, 0, 0, N], **cfg)  # top 24
    r, s = _frame(s, [N, N, N, N], **cfg)  # 3 freed: 1 fits the stack, 2 regions (16 labels) are dead
    assert r["free_n"][0] == 1 and r["dead"] == 16 and len(r["freed"]) == 3
    r, s = _frame(s, [N, N, N, 0], **cfg)  # brick 3 takes the stacked region; the top stays
    assert r["take_n"][0] == 1 and r["top"] == 24 and r["free_n"][0] == 0


def test_per_frame_limit_spreads_decoding_over_frames():
    cfg = dict(L=2, max_lod=2, cap=10 ** 6, per_frame=2, free_cap=16)
    s = fm.empty_state(5, 2)
    counts = []
    for _ in range(4):
        r, s = _frame(s, [0, 1, 2, 0, 1], **cfg)
        counts.append((len(r["requested"]), sum(r["assign_n"])))
    # finest first: frame 1 assigns bricks 0 and 3 (level 0), frame 2 bricks 1 and 4, frame 3 brick 2
    assert counts == [(5, 2), (3, 2), (1, 1), (0, 0)]
    assert list(s.lods) == [0, 1, 2, 0, 1]


def test_levels_start_at_multiples_of_their_size():
    cfg = dict(L=2, max_lod=2, cap=10 ** 6, per_frame=100, free_cap=16)  # sizes 64, 8, 1
    s = fm.empty_state(3, 2)
    r, s = _frame(s, [N, N, 2], **cfg)  # one label: top 1
    r, s = _frame(s, [0, 1, 2], **cfg)  # level 0 at 64 (63 dead), level 1 at 128: top 136
    assert (r["top"], r["dead"]) == (136, 63)
