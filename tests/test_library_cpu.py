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
