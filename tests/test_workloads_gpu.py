"""The benchmark's other workloads on the GPU, through the C ABI.

- 2048 x 2048 x 1024 power-diagram volume (~2M cells, log-normal radii, 30 % forced-uniform
  bricks) at full size: one subset of 100,000 random distinct bricks decoded in one batched launch
  with the autotuned schedule; sampled bricks checked bit-exactly against the generator's voxels
  (evaluated brick by brick, independently of the encoder) and against the oracle.
- The mixed serving workload (8 resident volumes of different brick sizes, cell diameters and
  background fractions) at reduced size: Poisson-arriving requests of log-uniform size from several
  clients under cache pressure; every request completes and sampled bricks match the oracle.
"""
import os
import threading
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_36898_gb300 as vc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vc._lib_handle()


def _host_ram_bytes() -> int:
    try:
        return os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        return 0


def test_uneven_power_diagram_volume_full_size_subset():
    if _host_ram_bytes() < (64 << 30):
        pytest.skip("the 17 GB raw volume needs a host with at least 64 GiB of memory")
    spec = synth.c3()
    V = synth.fill(spec)
    enc = vc.vc_encode_volume(V, 5, op_mask=0x7F, coder=1)
    del V
    vol = vc.Volume(enc)
    try:
        n_all = vol.n_bricks
        assert n_all == 64 * 64 * 32
        rng = np.random.default_rng(30)
        sub = rng.choice(n_all, size=100_000, replace=False).astype(np.uint32)
        ids = torch.from_numpy(sub.view(np.int32)).cuda()
        slots = torch.arange(sub.size, dtype=torch.int32, device="cuda")
        cache = torch.empty(sub.size * 32 ** 3, dtype=torch.int32, device="cuda")
        st = torch.zeros(vc.VC_STATUS_WORDS, dtype=torch.int32, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        # autotune on the first 10,000 items of the subset, then decode the whole subset
        _, mode, _ = vc.vc_volume_autotune(vol.handle, ids.data_ptr(), 10_000, slots.data_ptr(), cache.data_ptr(), 0,
                                           st.data_ptr(), s, reps=1)
        st.zero_()
        vol.decode(ids, slots, cache, 0, mode, st)
        torch.cuda.synchronize()
        assert int(st[0]) == 0, st.tolist()
        nbx, nby = 64, 64
        for i in rng.choice(sub.size, size=120, replace=False):
            bid = int(sub[i])
            bx, by, bz = bid % nbx, (bid // nbx) % nby, bid // (nbx * nby)
            want = synth.fill(spec, (32 * bx, 32 * by, 32 * bz), (32, 32, 32))
            got = cache[i * 32 ** 3:(i + 1) * 32 ** 3].cpu().numpy().view(np.uint32).reshape(32, 32, 32)
            assert np.array_equal(got, want), bid
        for i in rng.choice(sub.size, size=6, replace=False):
            got = cache[i * 32 ** 3:(i + 1) * 32 ** 3].cpu().numpy().view(np.uint32).reshape(32, 32, 32)
            assert np.array_equal(got, oracle.decode_brick(enc, int(sub[i]), 0))
        del cache
    finally:
        vol.release()


def test_mixed_volumes_poisson_serving():
    # the 8 volumes of the mixed workload at 128^3 (brick sizes 16, 32 and 64)
    specs = []
    for sp in synth.c5():
        b = sp.brick
        specs.append((synth.VolumeSpec(dims=(128, 128, 128), grid=sp.grid, seed=sp.seed, lam=sp.lam, bg=sp.bg, brick=b,
                                       name=sp.name + "_128"), b))
    vols, encs = [], []
    srv = vc.vc_server_create(48 << 20, 0, max_batch_items=4096)
    try:
        for sp, b in specs:
            enc = vc.vc_encode_volume(synth.fill(sp), b.bit_length() - 1, op_mask=0x7F, coder=1)
            encs.append((enc, b))
            h = vc.vc_load_compressed(enc, 0, 0)
            vols.append(h)
            vc.vc_server_add_volume(srv, h)
        ptr, nbytes = vc.vc_server_cache(srv)

        class _H:
            __cuda_array_interface__ = {"shape": (nbytes // 4,), "typestr": "<i4", "data": (ptr, False), "version": 3}
        cache = torch.as_tensor(_H(), device="cuda")
        errors, lat = [], []

        def client(tid):
            r = np.random.default_rng(500 + tid)
            try:
                for _ in range(10):
                    time.sleep(float(r.exponential(0.004)))
                    vi = int(r.integers(len(encs)))
                    enc, b = encs[vi]
                    nb = oracle.header(enc)["n_bricks"]
                    size = int(min(nb, max(1, round(float(np.exp(r.uniform(0, np.log(4096))))))))
                    bricks = r.choice(nb, size=size, replace=False).astype(np.uint32)
                    rid = vc.vc_submit_bricks(srv, vi, bricks)
                    if vc.vc_wait(srv, rid, 120000) != vc.VC_REQ_DONE:
                        errors.append(("not done", vi))
                        continue
                    _, offs = vc.vc_poll(srv, rid, size)
                    for k in r.choice(size, size=min(size, 2), replace=False):
                        w0 = int(offs[k]) // 4
                        got = cache[w0:w0 + b ** 3].cpu().numpy().view(np.uint32).reshape(b, b, b)
                        if not np.array_equal(got, oracle.decode_brick(enc, int(bricks[k]), 0)):
                            errors.append((vi, int(bricks[k])))
                    info = vc.vc_request_info_get(srv, rid)
                    lat.append((info.t_done_ns - info.t_submit_ns) / 1e6)
                    vc.vc_request_release(srv, rid)
            except Exception as e:
                errors.append(repr(e))

        threads = [threading.Thread(target=client, args=(t,)) for t in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join(300)
        assert not errors, errors[:5]
        assert len(lat) == 40
        st = vc.vc_server_stats_get(srv)
        assert st.requests_failed == 0 and st.requests_done == 40
    finally:
        vc.vc_release(srv)
        for h in vols:
            vc.vc_release(h)
