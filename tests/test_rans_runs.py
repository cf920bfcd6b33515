"""Pins of the rANS runs option (header flag bits 2..3 = log2 K; oracle/csgv_oracle.c): a record's
S symbols are cut into runs of Q = 32 ceil(S / 32K) symbols, each coded on its own with 32
interleaved states; the record holds every run's final states, then where runs 1.. start in the
coded words, then the palette and the runs' words. Pinned by the layout worked out by hand for
given S, by round trips to the volume for K = 2, 4, 8 at every brick size with the same symbols
and palette as the single-run coding, and by corrupt run starts."""
import numpy as np
import pytest

import oracle
import synth


def head_words(S, K):
    """The layout by hand: states of each run (min(run, 32)), then one start per run after the first."""
    Q = 32 * max(1, -(-S // (32 * K)))
    runs = [min(Q, S - k * Q) for k in range(max(1, -(-S // Q)))]
    return sum(min(r, 32) for r in runs) + len(runs) - 1, runs


@pytest.mark.parametrize("S,K,want", [(10, 1, 10), (10, 8, 10), (64, 2, 65), (65, 2, 34), (300, 8, 164),
                                      (1000, 1, 32), (1000, 2, 65), (1000, 4, 131), (1000, 8, 263), (33, 8, 34)])
def test_head_words_by_hand(S, K, want):
    lib = oracle._load()
    flags = oracle.runs_flag(K)
    assert lib.oracle_head_words(oracle.CODER_RANS, flags, S) == want
    assert head_words(S, K)[0] == want
    assert lib.oracle_head_words(oracle.CODER_PLAIN, 0, S) == 0


def _vol(b, seed):
    return synth.fill(synth.small(dims=(3 * b - 5, 2 * b + 3, b + 6), seed=seed, grid=max(4, b // 2),
                                  diameter=max(3.0, b / 2.5), bg=0.2))


@pytest.mark.parametrize("log2b,K", [(3, 2), (4, 2), (4, 4), (5, 2), (5, 8), (6, 4)])
def test_runs_round_trip_same_symbols_and_palette(log2b, K):
    V = _vol(1 << log2b, 30 + log2b + K)
    one = oracle.encode_volume(V, log2b, coder=oracle.CODER_RANS)
    enc = oracle.encode_volume(V, log2b, coder=oracle.CODER_RANS, flags=oracle.runs_flag(K))
    assert np.array_equal(oracle.decode_volume(enc), V)
    n = oracle.header(enc)["n_bricks"]
    multi = 0
    for b in range(n):
        r1, rk = oracle.brick_record(one, b), oracle.brick_record(enc, b)
        assert np.array_equal(oracle.brick_symbols(one, b), oracle.brick_symbols(enc, b))
        assert np.array_equal(r1["palette"], rk["palette"]) and r1["n_sym"] == rk["n_sym"]
        multi += len(head_words(rk["n_sym"], K)[1]) > 1
    assert multi > 0  # the volume has bricks of several runs


def test_runs_flag_only_with_rans():
    V = _vol(8, 5)
    with pytest.raises(oracle.OracleError):
        oracle.encode_volume(V, 3, coder=oracle.CODER_PLAIN, flags=oracle.runs_flag(2))


def test_corrupt_run_starts():
    V = _vol(16, 9)
    enc = oracle.encode_volume(V, 4, coder=oracle.CODER_RANS, flags=oracle.runs_flag(4))
    h = oracle.header(enc)
    rec_off = (128 + 4 * (h["n_bricks"] + 1) + 15) & ~15
    b = next(i for i in range(h["n_bricks"]) if len(head_words(oracle.brick_record(enc, i)["n_sym"], 4)[1]) >= 3)
    r = oracle.brick_record(enc, b)
    S = r["n_sym"]
    _, runs = head_words(S, 4)
    at = rec_off + 4 * r["offset_words"] + 16 + 4 * sum(min(x, 32) for x in runs)  # start of run 1
    starts = np.frombuffer(enc[at: at + 4 * (len(runs) - 1)].tobytes(), "<u4").copy()
    nw = r["coded_bytes"] // 2
    assert (np.diff(starts) >= 0).all() and 0 < starts[0] and starts[-1] <= nw
    for bad in ([starts[1] + 1] + list(starts[1:]),            # run 1 starts after run 2
                [starts[0] + 1] + list(starts[1:]),            # run 0 reads one word too many
                list(starts[:-1]) + [nw + 1]):                 # a start past the words
        e2 = enc.copy()
        e2[at: at + 4 * len(bad)] = np.asarray(bad, "<u4").view(np.uint8)
        assert oracle.decode_brick_status(e2, b) == oracle.ERR_CORRUPT
    assert oracle.decode_brick_status(enc, b) == 0
