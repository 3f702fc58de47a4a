"""GPU parity of the prioritised restore: every allocation ends equal to the
image, and work the caller orders after snap_restore_ready(k) already sees
allocation k restored while later waves are still in flight."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2502_16631_b300 as snap
import workloads

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

MiB = 1 << 20
SIZES = [65536, 4096 * 3 + 16, 1, 0, 200000, 65536 * 2, 12345, 17, 65537, 3 * 65536 - 1, 5 * MiB + 48]


@pytest.fixture(scope="module", autouse=True)
def _oracle_threads():
    oracle.set_threads(min(16, len(os.sched_getaffinity(0))))
    yield
    oracle.set_threads(1)


def device_state(sizes, seed):
    ts, hs = [], []
    for k, n in enumerate(sizes):
        h = workloads.xorshift_bytes(n, seed, k)
        t = torch.empty(n, dtype=torch.uint8, device="cuda")
        if n:
            t.copy_(torch.from_numpy(h))
        ts.append(t)
        hs.append(h)
    torch.cuda.synchronize()
    return ts, hs


def make_set(ts, C=65536, **kw):
    s = snap.Set(chunk_bytes=C, **kw)
    for t in ts:
        s.register(t.data_ptr() if t.numel() else 0, t.numel())
    s.tensors = ts
    return s


def oracle_image(hs, C, gen=0):
    rc, exp = oracle.write_full(hs, C, generation=gen)
    assert rc == 0
    img = snap.HostBuffer(exp.size)
    img.array[:] = exp
    return img


def readback(ts):
    torch.cuda.synchronize()
    return [t.cpu().numpy().copy() if t.numel() else np.zeros(0, np.uint8) for t in ts]


@pytest.mark.parametrize("C,first", [(65536, [10, 4]), (4096, [2, 7, 0]), (65536, []),
                                     (1 << 20, list(range(len(SIZES))))])
def test_prioritised_restore_matches_image_and_orders_work(C, first):
    ts, hs = device_state(SIZES, seed=91)
    img = oracle_image(hs, C, gen=5)  # the image comes from the oracle
    for t in ts:
        t.zero_()
    s = make_set(ts, C)
    st = torch.cuda.Stream()
    s.restore_async(img, first)
    # the caller's work on the priority allocations, ordered after readiness
    copies = {}
    with torch.cuda.stream(st):
        for k in first:
            s.restore_ready(k, st)
            copies[k] = ts[k].clone()
        last = len(SIZES) - 1
        s.restore_ready(last, st)
        copies.setdefault(last, ts[last].clone())
    s.restore_wait()
    st.synchronize()
    for k, c in copies.items():
        assert np.array_equal(c.cpu().numpy(), hs[k]), k
    for a, b in zip(readback(ts), hs):
        assert np.array_equal(a, b)
    n = sum(oracle.n_chunks(x, C) for x in SIZES)
    got, gen = s.committed_hashes(n)
    assert gen == 5
    assert np.array_equal(got, np.concatenate([oracle.chunk_hashes(h, C) for h in hs]))
    stt = s.stats()
    assert stt["generation"] == 5 and 0 < stt["frozen_ms"] <= stt["total_ms"]
    # the restored base serves an incremental checkpoint with nothing dirty
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    used = s.checkpoint(patch, snap.INCREMENTAL)
    rc, exp, nd = oracle.write_patch(hs, C, [oracle.chunk_hashes(h, C) for h in hs], 6, 5)
    assert nd == 0 and np.array_equal(patch.view(used), exp)
    s.close()


def test_prioritised_restore_many_waves():
    """1,200 allocations of 256 KiB-1 MiB (about 700 MiB): the doubling waves
    cap at the maximum count; every allocation is checked after its own
    readiness point."""
    rng = np.random.default_rng(5)
    sizes = [int(x) for x in rng.integers(256 * 1024, 1 << 20, 1200)]
    ts = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
    for k, t in enumerate(ts):
        workloads.torch_random_bytes(t, 100 + k)
    hs = readback(ts)
    img = oracle_image(hs, 65536)
    s = make_set(ts, 65536)
    for t in ts:
        t.zero_()
    first = [1199, 3, 600]
    st = torch.cuda.Stream()
    s.restore_async(img, first)
    sums = []
    with torch.cuda.stream(st):
        for k in list(first) + list(range(0, 1200, 37)):
            s.restore_ready(k, st)
            sums.append((k, ts[k].to(torch.int64).sum()))
    s.restore_wait()
    st.synchronize()
    for k, v in sums:
        assert int(v.item()) == int(hs[k].astype(np.int64).sum()), k
    assert s.verify(img) == 0
    s.close()


def test_prioritised_restore_errors_and_busy():
    ts, hs = device_state(SIZES, seed=93)
    img = oracle_image(hs, 65536)
    s = make_set(ts, 65536)
    assert s.restore_wait_status(0) == snap.EINVAL  # nothing pending
    s.restore_ready(3)  # nothing pending: already in place
    with pytest.raises(snap.SnapError):
        s.restore_ready(len(SIZES))
    assert s.restore_async_status(img, [1, 1]) == snap.EINVAL
    assert s.restore_async_status(img, [len(SIZES)]) == snap.EINVAL
    pageable = img.view().copy()
    assert s.restore_async_status(pageable, []) == snap.EINVAL
    other = make_set(ts[:-1], 65536)
    assert other.restore_async_status(img, []) == snap.EMISMATCH
    bad = snap.HostBuffer(img.nbytes)
    bad.array[:] = img.array
    bad.array[0] ^= 1
    assert s.restore_async_status(bad, []) == snap.EFORMAT
    s.restore_async(img, [0])
    assert s.restore_status(img) == snap.EBUSY
    assert s.checkpoint_status(img, snap.FULL)[0] == snap.EBUSY
    assert s.restore_async_status(img, []) == snap.EBUSY
    s.restore_wait()
    assert s.restore_wait_status(0) == snap.EINVAL
    for a, b in zip(readback(ts), hs):
        assert np.array_equal(a, b)
    s.close()
    other.close()


def test_prioritised_restore_gpt2_state():
    """GPT-2 small state (593 allocations, 2.26 GB): restore with the fp32
    weights first; a copy of the weights ordered after their readiness is
    bit-exact, and the whole state equals the image."""
    spec = workloads.gpt2_state_spec()
    sizes = workloads.spec_bytes(spec)
    ts = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
    workloads.torch_fill_spec(ts, spec, seed=94)
    s = make_set(ts, 65536)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    used = s.checkpoint(img, snap.FULL)
    host = readback(ts)
    rc, exp = oracle.write_full(host, 65536, 0)
    assert np.array_equal(img.view(used), exp)
    del exp
    weights = [k for k, e in enumerate(spec) if e[0].startswith("w.")] or list(range(148))
    for t in ts:
        t.zero_()
    st = torch.cuda.Stream()
    s.restore_async(img, weights)
    with torch.cuda.stream(st):
        for k in weights:
            s.restore_ready(k, st)
        cw = [ts[k].clone() for k in weights]
    s.restore_wait()
    st.synchronize()
    for k, c in zip(weights, cw):
        assert np.array_equal(c.cpu().numpy(), host[k]), k
    for a, b in zip(readback(ts), host):
        assert np.array_equal(a, b)
    s.close()
