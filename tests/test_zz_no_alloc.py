"""vc_decode_bricks_noalloc (statically reserved workspace) against vc_decode_bricks and the oracle,
through the C ABI.

Collected last on purpose: it must pass both alone and after every other GPU test has run in the
same process (other volumes loaded, the stream-ordered pool warm).

The entry point exists for callers that cannot allocate device memory while they decode (a
real-time loop that must not wait on the allocator, a process whose device memory is reserved up
front by another allocator). Its workspace is one fixed array per device, which three kinds of
call carve differently: the rANS symbols of every item, the 4-byte-per-item size-aware order of
requests of 1024 or more bricks, and (64^3 bricks) one scratch slice per persistent block. Each
kind is exercised here, next to the packed-index (cache paletting) output."""
import numpy as np
import pytest

import oracle
import synth
import paper_2609_36898_gb300 as vc

pytestmark = pytest.mark.gpu

VC_NOALLOC_WS_BYTES = 32 << 20


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _ws_stride(max_sym: int) -> int:
    return 16 * (((max_sym + 1) // 2 + 15) // 16) + 16


def _brick(V, b, bid):
    nbx, nby = V.shape[2] // b, V.shape[1] // b
    bx, by, bz = bid % nbx, (bid // nbx) % nby, bid // (nbx * nby)
    return V[bz * b:(bz + 1) * b, by * b:(by + 1) * b, bx * b:(bx + 1) * b]


def _unpack(words: np.ndarray, n: int, bits: int, per: int) -> np.ndarray:
    v = np.arange(n)
    w = words[v // per].astype(np.uint64)
    return ((w >> (bits * (v % per)).astype(np.uint64)) & ((1 << bits) - 1)).astype(np.int64)


def _both(torch, vol, ids, n, words, m, lod=0):
    """Decodes the same request with vc_decode_bricks and with the no-alloc entry point."""
    stream = torch.cuda.current_stream()
    slots = torch.arange(n, dtype=torch.int32, device="cuda")
    ref = torch.full((n * words,), -1, dtype=torch.int32, device="cuda")
    got = torch.full((n * words,), -1, dtype=torch.int32, device="cuda")
    st_ref = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
    st_got = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
    vc.vc_decode_bricks(vol.handle, ids.data_ptr(), n, slots.data_ptr(), ref.data_ptr(), lod, m,
                        st_ref.data_ptr(), stream.cuda_stream)
    vc.vc_decode_bricks_noalloc(vol.handle, ids.data_ptr(), n, slots.data_ptr(), got.data_ptr(), lod, m,
                                st_got.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    assert int(st_ref[0]) == 0 and int(st_got[0]) == 0, (st_ref.tolist(), st_got.tolist())
    return ref, got


@pytest.mark.parametrize("coder", [1, 0])
@pytest.mark.parametrize("mode", ["grid", "batched"])
def test_noalloc_matches_decode_bricks_twice_in_a_row(torch, coder, mode):
    V = synth.fill(synth.small(), (0, 0, 0), (128, 128, 128))
    enc = vc.vc_encode_volume(V, 5, op_mask=0x7F, coder=coder)
    vol = vc.Volume(enc)
    n = vol.n_bricks
    e3 = vol.b ** 3
    m = vc.MODES[mode]
    rng = np.random.default_rng(7 + coder)
    for call in range(2):  # two calls in a row: the shared workspace is reused
        ids_np = rng.permutation(n).astype(np.uint32)
        ids = torch.from_numpy(ids_np.view(np.int32)).cuda()
        ref, got = _both(torch, vol, ids, n, e3, m)
        assert torch.equal(ref, got), f"call {call}: noalloc output differs"
        # and both equal the input volume (lossless) and the oracle
        out = got.cpu().numpy().view(np.uint32).reshape(n, vol.b, vol.b, vol.b)
        for i in range(n):
            bid = int(ids_np[i])
            assert np.array_equal(out[i], _brick(V, vol.b, bid))
        for i in (0, n // 2, n - 1):
            assert np.array_equal(out[i], oracle.decode_brick(enc, int(ids_np[i])))
    vol.release()


@pytest.mark.parametrize("coder", [0, 1])
def test_noalloc_large_request_uses_the_order_array(torch, coder):
    """1024 or more bricks: the size-aware order's 4 bytes per item also come from the static
    array (after the symbols); 16^3 bricks keep the symbol workspace small enough for both."""
    V = synth.fill(synth.small(dims=(256, 128, 128), seed=11, diameter=8.0, bg=0.1))
    enc = vc.vc_encode_volume(V, 4, op_mask=0x7F, coder=coder)
    vol = vc.Volume(enc)
    n = vol.n_bricks
    assert n >= 1024
    info = vc.vc_volume_info_get(vol.handle)
    if coder == 1:
        assert n * _ws_stride(int(info.max_sym)) + 4 * n <= VC_NOALLOC_WS_BYTES
    e3 = vol.b ** 3
    rng = np.random.default_rng(21 + coder)
    for call in range(2):
        ids_np = rng.permutation(n).astype(np.uint32)
        ids = torch.from_numpy(ids_np.view(np.int32)).cuda()
        for mode in ("grid", "batched"):
            ref, got = _both(torch, vol, ids, n, e3, vc.MODES[mode])
            assert torch.equal(ref, got), (call, mode)
            out = got.cpu().numpy().view(np.uint32).reshape(n, vol.b, vol.b, vol.b)
            for i in range(n):
                assert np.array_equal(out[i], _brick(V, vol.b, int(ids_np[i]))), (call, mode, i)
            for i in rng.choice(n, size=6, replace=False):
                assert np.array_equal(out[i], oracle.decode_brick(enc, int(ids_np[i])))
    vol.release()


def test_noalloc_64cube_bricks_use_scratch_slices(torch):
    """64^3 bricks: one scratch slice per persistent block is carved out of the static array after
    the symbols (the grid shrinks to the slices that fit)."""
    V = synth.fill(synth.small(dims=(128, 128, 128), seed=5, diameter=16.0, bg=0.1))
    enc = vc.vc_encode_volume(V, 6, op_mask=0x7F, coder=1)
    vol = vc.Volume(enc)
    n = vol.n_bricks
    e3 = vol.b ** 3
    for call in range(2):
        ids_np = np.random.default_rng(31 + call).permutation(n).astype(np.uint32)
        ids = torch.from_numpy(ids_np.view(np.int32)).cuda()
        for lod in (0, 1):
            e = vol.b >> lod
            ref, got = _both(torch, vol, ids, n, e ** 3, vc.MODES["batched"], lod)
            assert torch.equal(ref, got), (call, lod)
            out = got.cpu().numpy().view(np.uint32).reshape(n, e, e, e)
            for i in range(n):
                want = _brick(V, vol.b, int(ids_np[i])) if lod == 0 else oracle.decode_brick(enc, int(ids_np[i]), lod)
                assert np.array_equal(out[i], want), (call, lod, i)
    assert e3 == 64 ** 3
    vol.release()


def test_noalloc_paletted_output(torch):
    """Cache paletting through the no-alloc entry point: packed indices equal vc_decode_bricks's and
    map through each brick's palette to the oracle's labels."""
    V = synth.fill(synth.small(dims=(128, 96, 64), seed=75, grid=16, diameter=14.0, bg=0.2))
    enc = vc.vc_encode_volume(V, 5, op_mask=0x7F, coder=1)
    vol = vc.Volume(enc)
    n = vol.n_bricks
    words, bits, per = vc.vc_volume_slot_words(vol.handle, 0, True)
    ids = torch.arange(n, dtype=torch.int32, device="cuda")
    for call in range(2):
        for mode in ("grid", "batched"):
            ref, got = _both(torch, vol, ids, n, words, vc.MODES[mode] | vc.VC_MODE_PALETTED)
            assert torch.equal(ref, got), (call, mode)
            out = got.cpu().numpy().view(np.uint32).reshape(n, words)
            for i in range(n):
                pal = oracle.brick_record(enc, i)["palette"]
                idx = _unpack(out[i], vol.b ** 3, bits, per)
                assert np.array_equal(pal[idx].reshape(vol.b, vol.b, vol.b), _brick(V, vol.b, i)), (call, mode, i)
    vol.release()


def test_noalloc_calls_leave_free_device_memory_unchanged(torch):
    """After a first call (which looks up the static array's address), further calls take no device
    memory: the device's free bytes stay the same across them."""
    V = synth.fill(synth.small(), (0, 0, 0), (128, 128, 64))
    enc = vc.vc_encode_volume(V, 5, op_mask=0x7F, coder=1)
    vol = vc.Volume(enc)
    n = vol.n_bricks
    e3 = vol.b ** 3
    stream = torch.cuda.current_stream()
    ids = torch.arange(n, dtype=torch.int32, device="cuda")
    cache = torch.zeros(n * e3, dtype=torch.int32, device="cuda")
    st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
    args = (vol.handle, ids.data_ptr(), n, ids.data_ptr(), cache.data_ptr(), 0, vc.VC_MODE_GRID, st.data_ptr(),
            stream.cuda_stream)
    vc.vc_decode_bricks_noalloc(*args)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        vc.vc_decode_bricks_noalloc(*args)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert int(st[0]) == 0 and free1 == free0
    out = cache.cpu().numpy().view(np.uint32).reshape(n, vol.b, vol.b, vol.b)
    for i in range(n):
        assert np.array_equal(out[i], _brick(V, vol.b, i))
    vol.release()


def test_noalloc_rejects_requests_beyond_its_workspace(torch):
    V = synth.fill(synth.small(), (0, 0, 0), (64, 64, 64))
    enc = vc.vc_encode_volume(V, 5, op_mask=0x7F, coder=1)
    vol = vc.Volume(enc)
    info = vc.vc_volume_info_get(vol.handle)
    stride = _ws_stride(int(info.max_sym))
    n_max = VC_NOALLOC_WS_BYTES // stride
    ids = torch.zeros(n_max + 1, dtype=torch.int32, device="cuda")
    cache = torch.zeros((n_max + 1) * vol.b ** 3, dtype=torch.int32, device="cuda")
    st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(vc.VCError) as ex:
        vc.vc_decode_bricks_noalloc(vol.handle, ids.data_ptr(), n_max + 1, ids.data_ptr(), cache.data_ptr(), 0,
                                    vc.VC_MODE_GRID, st.data_ptr(), s)
    assert ex.value.code == vc.VC_ERR_ARG
    # the largest accepted size decodes (every item is brick 0 into its own slot)
    slots = torch.arange(n_max, dtype=torch.int32, device="cuda")
    vc.vc_decode_bricks_noalloc(vol.handle, ids.data_ptr(), n_max, slots.data_ptr(), cache.data_ptr(), 0,
                                vc.VC_MODE_GRID, st.data_ptr(), s)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    first = cache[: vol.b ** 3]
    last = cache[(n_max - 1) * vol.b ** 3: n_max * vol.b ** 3]
    assert torch.equal(first, last)
    assert np.array_equal(first.cpu().numpy().view(np.uint32).reshape(vol.b, vol.b, vol.b),
                          oracle.decode_brick(enc, 0))
    # the pipelined schedule allocates, so it is refused here
    with pytest.raises(vc.VCError):
        vc.vc_decode_bricks_noalloc(vol.handle, ids.data_ptr(), 1, slots.data_ptr(), cache.data_ptr(), 0,
                                    vc.VC_MODE_PIPELINED, st.data_ptr(), s)
    vol.release()
