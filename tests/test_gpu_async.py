"""GPU parity of the asynchronous checkpoint: the image produced in the
background equals the oracle's image of the state at the cut, even though the
caller overwrites its buffers as soon as snap_checkpoint_async returns."""
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


def readback(ts):
    torch.cuda.synchronize()
    return [t.cpu().numpy().copy() if t.numel() else np.zeros(0, np.uint8) for t in ts]


def make_set(ts, C, **kw):
    s = snap.Set(chunk_bytes=C, **kw)
    for t in ts:
        s.register(t.data_ptr() if t.numel() else 0, t.numel())
    s.tensors = ts
    return s


def scribble(ts, seed, chunks=None, C=None):
    """Overwrite device bytes on the caller's stream, without synchronising:
    every byte (chunks=None) or the listed (buffer, chunk) pairs."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    for k, t in enumerate(ts):
        if not t.numel():
            continue
        if chunks is None:
            t ^= torch.randint(1, 256, (t.numel(),), dtype=torch.uint8, device="cuda", generator=g)
        else:
            for kk, i in chunks:
                if kk == k:
                    lo, hi = i * C, min((i + 1) * C, t.numel())
                    t[lo:hi] ^= torch.randint(1, 256, (hi - lo,), dtype=torch.uint8, device="cuda", generator=g)


def all_hashes(datas, C):
    return np.concatenate([oracle.chunk_hashes(d, C) for d in datas] + [np.zeros(0, np.uint32)])


@pytest.mark.parametrize("C,async_ctas", [(4096, 0), (65536, 0), (65536, 1), (65536, 7), (1 << 20, 148)])
def test_async_full_is_the_state_at_the_cut(C, async_ctas):
    ts, hs = device_state(SIZES, seed=31)
    s = make_set(ts, C, async_ctas=async_ctas)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    img.array[:] = 0xA5
    s.checkpoint_async(img, snap.FULL)
    scribble(ts, seed=32)  # the caller resumes at once
    used = s.checkpoint_wait()
    rc, exp = oracle.write_full(hs, C, generation=0)
    assert rc == 0 and used == exp.size
    assert np.array_equal(img.view(used), exp)
    n = sum(oracle.n_chunks(x, C) for x in SIZES)
    got, gen = s.committed_hashes(n)
    assert gen == 0 and np.array_equal(got, all_hashes(hs, C))
    now = readback(ts)
    assert all(not np.array_equal(a, b) for a, b in zip(now, hs) if a.size)
    st = s.stats()
    assert 0 < st["frozen_ms"] <= st["total_ms"]
    assert st["kernel_launches"] >= 2 and st["generation"] == 0
    # a synchronous checkpoint afterwards sees the scribbled state
    used = s.checkpoint(img, snap.FULL)
    assert np.array_equal(img.view(used), oracle.write_full(now, C, generation=1)[1])
    s.close()


@pytest.mark.parametrize("C", [4096, 65536])
def test_async_incremental_matches_oracle(C):
    ts, hs = device_state(SIZES, seed=41)
    s = make_set(ts, C)
    full = snap.HostBuffer(s.image_bytes(snap.FULL))
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    patch.array[:] = 0x5A
    used0 = s.checkpoint(full, snap.FULL)
    nch = [oracle.n_chunks(x, C) for x in SIZES]
    first = [(0, 0), (2, 0), (4, nch[4] - 1), (8, 1), (10, 3), (10, nch[10] - 1)]
    scribble(ts, 42, first, C)
    s1 = readback(ts)
    s.checkpoint_async(patch, snap.INCREMENTAL)
    second = [(1, 0), (5, 1), (10, 7), (10, 3)]
    scribble(ts, 43, second, C)  # during the background part
    used = s.checkpoint_wait()
    rc, exp, nd = oracle.write_patch(s1, C, [oracle.chunk_hashes(h, C) for h in hs], generation=1, parent=0)
    assert rc == 0 and used == exp.size and nd == len(set(first))
    assert np.array_equal(patch.view(used), exp)
    assert s.stats()["dirty_chunks"] == nd
    merged = full.view(used0).copy()
    snap.apply_patch(merged, patch.view(used))
    assert np.array_equal(merged, oracle.write_full(s1, C, generation=1)[1])
    # the next checkpoint diffs against the state at the cut, not the live one
    s2 = readback(ts)
    used2 = s.checkpoint(patch, snap.INCREMENTAL)
    rc, exp2, nd2 = oracle.write_patch(s2, C, [oracle.chunk_hashes(h, C) for h in s1], 2, 1)
    assert nd2 == len(set(second)) and np.array_equal(patch.view(used2), exp2)
    s.close()


def test_async_pending_set_is_busy_and_argument_errors():
    ts, hs = device_state(SIZES, seed=51)
    s = make_set(ts, 65536)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    assert s.checkpoint_async_status(img, snap.INCREMENTAL) == snap.ENOBASE
    assert s.checkpoint_wait_status(0)[0] == snap.EINVAL  # nothing pending
    pageable = np.zeros(s.image_bytes(snap.FULL), np.uint8)
    assert s.checkpoint_async_status(pageable, snap.FULL) == snap.EINVAL
    assert s.checkpoint_async_status(img, snap.FULL, cap=4096) == snap.EINVAL
    s.checkpoint_async(img, snap.FULL)
    assert s.checkpoint_status(img, snap.FULL)[0] == snap.EBUSY
    assert s.checkpoint_async_status(img, snap.FULL) == snap.EBUSY
    used = s.checkpoint_wait()
    assert np.array_equal(img.view(used), oracle.write_full(hs, 65536, 0)[1])
    assert s.checkpoint_wait_status(0)[0] == snap.EINVAL
    s.close()


def test_async_wait_timeout_leaves_it_pending():
    """One background CTA over 256 MiB takes far longer than a zero wait."""
    ts, hs = device_state([256 * MiB], seed=61)
    s = make_set(ts, 65536, async_ctas=1)
    s.prepare(shadow=True)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    s.checkpoint_async(img, snap.FULL)
    scribble(ts, 62)
    rc, _ = s.checkpoint_wait_status(0)
    if rc == snap.ETIMEDOUT:
        assert s.checkpoint_status(img, snap.FULL)[0] == snap.EBUSY
    else:
        assert rc == snap.OK
    if rc == snap.ETIMEDOUT:
        used = s.checkpoint_wait(120000)
    else:
        used = img.nbytes
    assert np.array_equal(img.view(used), oracle.write_full(hs, 65536, 0)[1])
    s.close()


def test_async_shadow_allocation_failure(monkeypatch):
    ts, hs = device_state(SIZES, seed=71)
    s = make_set(ts, 65536)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    monkeypatch.setenv("SNAP_FAULT", "shadow_alloc")
    assert s.checkpoint_async_status(img, snap.FULL) == snap.ENOMEM
    monkeypatch.delenv("SNAP_FAULT")
    used = s.checkpoint(img, snap.FULL)  # the set is still usable
    assert np.array_equal(img.view(used), oracle.write_full(hs, 65536, 0)[1])
    s.checkpoint_async(img, snap.FULL)
    used = s.checkpoint_wait()
    assert np.array_equal(img.view(used), oracle.write_full(hs, 65536, 1)[1])
    s.close()


def test_async_gpt2_state_full_parity():
    """GPT-2 small training state (593 allocations, 2,259,472,384 B): the
    cut is taken, the live state is overwritten while the image is produced
    in the background, and the image equals the oracle's image of the state
    at the cut, byte for byte."""
    spec = workloads.gpt2_state_spec()
    sizes = workloads.spec_bytes(spec)
    ts = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
    workloads.torch_fill_spec(ts, spec, seed=81)
    C = 65536
    s = make_set(ts, C)
    s.prepare(shadow=True)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    host = readback(ts)
    s.checkpoint_async(img, snap.FULL)
    scribble(ts, 83)
    used = s.checkpoint_wait()
    rc, exp = oracle.write_full(host, C, 0)
    assert rc == 0 and used == exp.size
    assert np.array_equal(img.view(used), exp)
    s.close()


def test_two_sets_in_two_threads_and_one_set_shared():
    """Sets are independent: two threads checkpoint two sets at once and both
    images equal the oracle's; on one set, a second concurrent call gets
    SNAP_EBUSY instead of interleaving with the first."""
    import threading
    ts1, hs1 = device_state(SIZES, seed=141)
    ts2, hs2 = device_state(SIZES, seed=142)
    s1, s2 = make_set(ts1, 65536), make_set(ts2, 65536)
    i1 = snap.HostBuffer(s1.image_bytes(snap.FULL))
    i2 = snap.HostBuffer(s2.image_bytes(snap.FULL))
    out = {}

    def run(name, s, img):
        out[name] = [s.checkpoint(img, snap.FULL) for _ in range(5)][-1]

    th = [threading.Thread(target=run, args=("a", s1, i1)), threading.Thread(target=run, args=("b", s2, i2))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert np.array_equal(i1.view(out["a"]), oracle.write_full(hs1, 65536, 4)[1])
    assert np.array_equal(i2.view(out["b"]), oracle.write_full(hs2, 65536, 4)[1])
    # one set: while an asynchronous checkpoint is pending every call is busy
    s1.checkpoint_async(i1, snap.FULL)
    statuses = []
    th = [threading.Thread(target=lambda: statuses.append(s1.checkpoint_status(i1, snap.FULL)[0]))
          for _ in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert statuses == [snap.EBUSY] * 4
    s1.checkpoint_wait()
    s1.close()
    s2.close()


def test_destroy_with_pending_work_waits_for_it():
    """Closing a set with an asynchronous checkpoint or a prioritised restore
    still in flight waits for the device work before freeing anything."""
    ts, hs = device_state([64 * MiB, 3 * MiB + 5], seed=151)
    s = make_set(ts, 65536, async_ctas=1)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    s.checkpoint_async(img, snap.FULL)
    s.close()  # no wait: destroy synchronises the background stream
    s = make_set(ts, 65536)
    used = s.checkpoint(img, snap.FULL)
    assert np.array_equal(img.view(used), oracle.write_full(hs, 65536, 0)[1])
    s.restore_async(img, [1])
    s.close()  # no restore_wait
    torch.cuda.synchronize()
    for a, b in zip(readback(ts), hs):
        assert np.array_equal(a, b)
