"""Degenerate states through every call: a set with no allocations, sets
whose allocations are all zero bytes long, and one whose first and last
allocations are.

Such a state has no chunk at all (or chunks only in the middle): its full
image is the 64-byte header plus one record per allocation with no hashes
and no data, and an incremental patch of it has no dirty chunk.  Every
image, patch and file written here must equal the oracle's byte for byte,
and every restore, verify and prioritised restore must succeed on it -- the
empty cases of the checkpoint and restore actions (Sec. 3.1.1)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2502_16631_b300 as snap
import workloads

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

C = 65536
STATES = {
    "empty": [],
    "one_zero": [0],
    "all_zero": [0, 0, 0],
    "zero_ends": [0, 5000, 2 * C + 48, 0],
}


def device_state(sizes, seed):
    ts, hs = [], []
    for k, n in enumerate(sizes):
        h = workloads.xorshift_bytes(n, seed, k)
        t = torch.empty(n + 16, dtype=torch.uint8, device="cuda")[:n]
        if n:
            t.copy_(torch.from_numpy(h))
        ts.append(t)
        hs.append(h)
    torch.cuda.synchronize()
    return ts, hs


def make_set(ts):
    s = snap.Set(chunk_bytes=C, ring_bytes=4 << 20)  # a small pinned ring: these states are tiny
    for t in ts:
        s.register(t.data_ptr() if t.numel() else 0, t.numel())
    return s


def readback(ts):
    torch.cuda.synchronize()
    return [t.cpu().numpy().copy() if t.numel() else np.zeros(0, np.uint8) for t in ts]


def hashes(hs):
    return [oracle.chunk_hashes(h, C) for h in hs]


def scribble(ts):
    for t in ts:
        if t.numel():
            t.fill_(0x3C)
    torch.cuda.synchronize()


@pytest.mark.parametrize("name", list(STATES))
def test_degenerate_state_sync_calls(name):
    """Full and incremental checkpoints into pinned and pageable images,
    restore from both, verify."""
    sizes = STATES[name]
    ts, hs = device_state(sizes, seed=301)
    s = make_set(ts)
    assert s.image_bytes(snap.FULL) == oracle.image_bytes(sizes, C)

    # pinned images, written through the mapping
    full = snap.HostBuffer(s.image_bytes(snap.FULL))
    full.array[:] = 0xA5
    used = s.checkpoint(full, snap.FULL)
    rc, exp = oracle.write_full(hs, C, generation=0)
    assert rc == 0 and used == exp.size and np.array_equal(full.view(used), exp)
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    patch.array[:] = 0x5A
    used_p = s.checkpoint(patch, snap.INCREMENTAL)
    rc, exp_p, nd = oracle.write_patch(hs, C, hashes(hs), generation=1, parent=0)
    assert rc == 0 and nd == 0 and s.stats()["dirty_chunks"] == 0
    assert used_p == exp_p.size and np.array_equal(patch.view(used_p), exp_p)

    # pageable images, through the ring
    full_p = np.full(s.image_bytes(snap.FULL), 0xA5, dtype=np.uint8)
    used2 = s.checkpoint(full_p, snap.FULL)
    assert np.array_equal(full_p[:used2], oracle.write_full(hs, C, generation=2)[1])
    patch_p = np.full(s.image_bytes(snap.INCREMENTAL), 0x5A, dtype=np.uint8)
    used3 = s.checkpoint(patch_p, snap.INCREMENTAL)
    assert np.array_equal(patch_p[:used3], oracle.write_patch(hs, C, hashes(hs), 3, 2)[1])

    # the generation-0 image + its patch is the generation-1 full image
    merged = full.view(used).copy()
    snap.apply_patch(merged, patch.view(used_p))
    assert np.array_equal(merged, oracle.write_full(hs, C, generation=1)[1])

    # restores from the pinned and from the pageable image, then verify
    for img, n in ((full, used), (full_p, used2)):
        scribble(ts)
        s.restore(img, n)
        for a, b in zip(readback(ts), hs):
            assert np.array_equal(a, b)
        assert s.verify(img, n) == 0
    n_chunks = sum(oracle.n_chunks(x, C) for x in sizes)
    got, gen = s.committed_hashes(n_chunks)
    assert gen == 2 and np.array_equal(got, np.concatenate(hashes(hs)) if n_chunks else got)


@pytest.mark.parametrize("name", list(STATES))
def test_degenerate_state_async_lazy_and_file(name, tmp_path):
    """Asynchronous checkpoint, prioritised restore and image files."""
    sizes = STATES[name]
    ts, hs = device_state(sizes, seed=302)
    s = make_set(ts)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    img.array[:] = 0xA5
    s.checkpoint_async(img, snap.FULL)
    used = s.checkpoint_wait()
    assert np.array_equal(img.view(used), oracle.write_full(hs, C, generation=0)[1])

    scribble(ts)
    first = [len(sizes) - 1] if sizes else []
    s.restore_async(img, first=first, nbytes=used)
    for k in range(len(sizes)):
        s.restore_ready(k)
    s.restore_wait()
    for a, b in zip(readback(ts), hs):
        assert np.array_equal(a, b)

    path = str(tmp_path / "state.snap")
    n = s.checkpoint_file(path, snap.FULL, sync=True)
    with open(path, "rb") as f:
        disk = np.frombuffer(f.read(), dtype=np.uint8)
    assert disk.size == n and np.array_equal(disk, oracle.write_full(hs, C, generation=1)[1])
    scribble(ts)
    s.restore_file(path)
    for a, b in zip(readback(ts), hs):
        assert np.array_equal(a, b)
    assert not os.path.exists(path + ".tmp")


def test_degenerate_tenants_served():
    """The serving loop completes full, incremental and restore requests of
    tenants that have no chunk (and one with chunks only in the middle)."""
    tenants = []
    for k, name in enumerate(STATES):
        ts, hs = device_state(STATES[name], seed=310 + k)
        tenants.append((make_set(ts), ts, hs))
    sv = snap.Server(pinned_budget=64 << 20, hbm_budget=1 << 40, chunk_bytes=C)
    try:
        imgs = [np.full(s.image_bytes(snap.FULL), 0xA5, dtype=np.uint8) for s, _, _ in tenants]
        patches = [np.full(s.image_bytes(snap.INCREMENTAL), 0x5A, dtype=np.uint8) for s, _, _ in tenants]

        def run(reqs):
            tickets = [sv.submit(s, kind, buf) for s, kind, buf in reqs]
            out = []
            for t in tickets:
                rc, status, st = sv.wait(t, 15000)
                assert rc == snap.OK and status == snap.OK, (rc, status)
                out.append(st)
            return out

        st = run([(s, snap.REQ_FULL, imgs[t]) for t, (s, _, _) in enumerate(tenants)])
        for t, (_, _, hs) in enumerate(tenants):
            assert np.array_equal(imgs[t][: st[t]["image_bytes"]], oracle.write_full(hs, C, generation=0)[1])
        st = run([(s, snap.REQ_INCREMENTAL, patches[t]) for t, (s, _, _) in enumerate(tenants)])
        for t, (_, _, hs) in enumerate(tenants):
            exp = oracle.write_patch(hs, C, hashes(hs), 1, 0)[1]
            assert st[t]["dirty_chunks"] == 0 and np.array_equal(patches[t][: st[t]["image_bytes"]], exp)
        for _, ts, _ in tenants:
            scribble(ts)
        run([(s, snap.REQ_RESTORE, imgs[t]) for t, (s, _, _) in enumerate(tenants)])
        for _, ts, hs in tenants:
            for a, b in zip(readback(ts), hs):
                assert np.array_equal(a, b)
    finally:
        sv.close()
