"""Detail split, host side (no GPU): where each brick's finest level starts. vc_split_counts walks
the symbols level by level (level l + 1 = the 8 children of every node of level l emitted with
stop bit 0) and must agree with the oracle's own decode of the same brick: the symbols of levels
0 .. L-1 are their nodes plus the entries of their delta operations."""
import numpy as np
import pytest

import oracle
import synth
import paper_2609_36898_gb300 as vc


def _expected(enc, bid, log2b, short):
    nodes = oracle.brick_nodes(enc, bid)
    c = nodes[nodes["level"] < log2b]
    deltas = c["delta"][c["op"] == oracle.OP_DELTA]
    entries = len(deltas) if short else sum(len(oracle.delta_nibbles(int(d))) for d in deltas)
    return (oracle.brick_record(enc, bid)["n_sym"], len(c) + entries, int((c["op"] == oracle.OP_ADV).sum()),
            len(deltas))


@pytest.mark.parametrize("coder", [0, 1])
@pytest.mark.parametrize("flags", [0, 1, 2])
def test_split_counts_match_the_oracle(coder, flags):
    V = synth.fill(synth.small(dims=(72, 40, 36), seed=17, diameter=11.0, bg=0.2))
    for log2b in (1, 2, 3, 4, 5, 6):
        enc = vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=coder, flags=flags)
        n = oracle.header(enc)["n_bricks"]
        for bid in range(0, n, max(1, n // 48)):
            assert vc.vc_split_counts(enc, bid) == _expected(enc, bid, log2b, bool(flags & 2)), (log2b, bid)


@pytest.mark.parametrize("K", [2, 4, 8])
def test_split_counts_with_rans_runs(K):
    V = synth.fill(synth.small(dims=(72, 40, 36), seed=18, diameter=11.0, bg=0.2))
    for log2b in (3, 4, 5, 6):
        enc = vc.vc_encode_volume(V, log2b, op_mask=0x7F, coder=1, flags=oracle.runs_flag(K))
        n = oracle.header(enc)["n_bricks"]
        for bid in range(0, n, max(1, n // 24)):
            assert vc.vc_split_counts(enc, bid) == _expected(enc, bid, log2b, False), (log2b, bid)


def test_split_counts_uniform_and_corrupt():
    V = np.full((16, 16, 16), 5, dtype=np.uint32)
    enc = vc.vc_encode_volume(V, 4, coder=1)
    assert vc.vc_split_counts(enc, 0) == (1, 1, 1, 0)  # the root alone, stopped
    # a stream that ends inside the coarse levels
    g = oracle.pack_single_brick(2, [oracle.OP_ADV], [7], 0)
    with pytest.raises(vc.VCError) as ex:
        vc.vc_split_counts(g, 0)
    assert ex.value.code == vc.VC_ERR_CORRUPT
    with pytest.raises(vc.VCError):
        vc.vc_split_counts(enc, 1)  # no such brick


def test_split_load_rejects_undecodable_records_before_touching_a_device():
    """The split loader decodes every record on the host first: a record whose rANS words do not
    decode, or whose stream ends inside the coarse levels, fails with VC_ERR_FORMAT before any
    CUDA call."""
    V = synth.fill(synth.small(dims=(64, 64, 32), seed=5, diameter=10.0, bg=0.2))
    enc = vc.vc_encode_volume(V, 4, op_mask=0x7F, coder=1)
    h = oracle.header(enc)
    rec0 = (128 + 4 * (h["n_bricks"] + 1) + 15) & ~15
    rec = oracle.brick_record(enc, 3)
    # brick 3's coded word count: one word short of what its states consume
    off = rec0 + 4 * rec["offset_words"] + 8
    bad = enc.copy()
    bad[off:off + 4] = np.frombuffer(np.uint32(rec["coded_bytes"] - 2).tobytes(), np.uint8)
    with pytest.raises(vc.VCError) as ex:
        vc.vc_load_compressed_split(bad, 0, 0)
    assert ex.value.code in (vc.VC_ERR_FORMAT,)
    # a plain-coded brick whose stream stops after the root
    g = oracle.pack_single_brick(3, [oracle.OP_ADV], [7], 0)
    with pytest.raises(vc.VCError) as ex:
        vc.vc_load_compressed_split(g, 0, 0)
    assert ex.value.code == vc.VC_ERR_FORMAT
