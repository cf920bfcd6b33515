"""Host-side checks of libvc.so that need no GPU: it loads, exports every function include/vc.h
declares, and its multi-threaded CPU encoder writes the same bytes as the oracle's encoder."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth
import paper_2609_36898_gb300 as vc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(vc_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_36898_gb300 import build
    build.build()
    return vc._lib_handle()


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "vc_decode_bricks" in names and "vc_load_compressed" in names and "vc_release" in names
    for n in names:
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def test_status_strings(lib):
    for code in range(-8, 1):
        assert lib.vc_status_string(code)


def test_release_null_is_noop(lib):
    assert lib.vc_release(None) == 0


def test_load_rejects_bad_bytes_before_touching_a_device(lib):
    out = ctypes.c_void_p()
    junk = np.zeros(256, dtype=np.uint8)
    assert lib.vc_load_compressed(junk.ctypes.data, junk.size, 0, None, ctypes.byref(out)) == vc.VC_ERR_FORMAT
    assert lib.vc_load_compressed(None, 0, 0, None, ctypes.byref(out)) == vc.VC_ERR_ARG
    assert out.value is None


@pytest.mark.parametrize("log2b", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("coder", [0, 1])
def test_encoder_matches_oracle_bytes(lib, log2b, coder):
    V = synth.fill(synth.small(dims=(37, 21, 18), seed=4, diameter=9.0, bg=0.25))
    for mask in (0x7F, 0x7F & ~(1 << 5), 0x7F & ~(1 << 6), (1 << 4) | 1, 1 << 4):
        for flags in (0, 1, 2, 3):
            a = oracle.encode_volume(V, log2b, op_mask=mask, coder=coder, flags=flags)
            b = vc.vc_encode_volume(V, log2b, op_mask=mask, coder=coder, flags=flags, threads=3)
            assert a.size == b.size and np.array_equal(a, b), (mask, flags)


@pytest.mark.parametrize("log2b,K", [(3, 2), (4, 4), (5, 2), (5, 8), (6, 4)])
def test_encoder_matches_oracle_bytes_with_rans_runs(lib, log2b, K):
    V = synth.fill(synth.small(dims=(3 * (1 << log2b) - 3, 40, 21), seed=6, diameter=9.0, bg=0.25))
    for flags in (0, 1, 2):
        f = flags | oracle.runs_flag(K)
        a = oracle.encode_volume(V, log2b, coder=1, flags=f)
        b = vc.vc_encode_volume(V, log2b, coder=1, flags=f, threads=3)
        assert a.size == b.size and np.array_equal(a, b), (K, flags)
    with pytest.raises(vc.VCError):  # runs are a rANS option
        vc.vc_encode_volume(V, log2b, coder=0, flags=oracle.runs_flag(K))


def test_encoder_matches_oracle_on_workload_sample(lib):
    spec = synth.c1()
    V = synth.fill(spec)
    a = oracle.encode_volume(V, 5, coder=1)
    b = vc.vc_encode_volume(V, 5, coder=1)
    assert np.array_equal(a, b)
    assert np.array_equal(oracle.decode_volume(b), V)


def test_encoder_argument_checks(lib):
    V = np.zeros((4, 4, 4), dtype=np.uint32)
    with pytest.raises(vc.VCError):
        vc.vc_encode_volume(V, 0)
    with pytest.raises(vc.VCError):
        vc.vc_encode_volume(V, 3, op_mask=0x0F)  # palette advance disabled


def _full_table(freq) -> np.ndarray:
    """The table with every symbol at least 1 (taken from the largest), still summing to 4096."""
    f = np.asarray(freq, dtype=np.int64).copy()
    short = int((f == 0).sum())
    f[f == 0] = 1
    f[int(np.argmax(f))] -= short
    assert f.sum() == 4096 and (f >= 1).all()
    return f.astype(np.uint32)


@pytest.mark.parametrize("coder", [0, 1])
def test_slab_encoding_with_one_table_concatenates_to_a_valid_volume(lib, coder):
    """A volume encoded in z slabs of whole bricks with one shared rANS table, then joined with
    vc_concat_volumes_z, decodes (oracle) to the input everywhere; with the volume's own table the
    fixed-table encoder writes the same bytes as the plain one."""
    V = synth.fill(synth.small(dims=(48, 40, 70), seed=23, grid=8, diameter=9.0, bg=0.15))
    whole = vc.vc_encode_volume(V, 4, coder=coder)
    own = oracle.header(whole)["freq"]
    if coder == 1:
        again = vc.vc_encode_volume(V, 4, coder=coder, freq=own)
        assert np.array_equal(again, whole)
    table = _full_table(own) if coder == 1 else None
    parts = [vc.vc_encode_volume(V[z0:z0 + 32], 4, coder=coder, freq=table) for z0 in (0, 32, 64)]
    joined = vc.vc_concat_volumes_z(parts)
    h = oracle.header(joined)
    assert h["dims"] == oracle.header(whole)["dims"] and h["n_bricks"] == oracle.header(whole)["n_bricks"]
    assert np.array_equal(oracle.decode_volume(joined), V)
    # mismatched parts are refused
    other = vc.vc_encode_volume(V[:32], 3, coder=coder)
    with pytest.raises(vc.VCError):
        vc.vc_concat_volumes_z([parts[0], other])
    if coder == 1:
        bad = table.copy()
        bad[0] += 1
        with pytest.raises(vc.VCError):
            vc.vc_encode_volume(V[:32], 4, coder=coder, freq=bad)
