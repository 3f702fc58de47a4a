"""snap_checkpoint_coordinated on one GPU, with the other ranks stood in for
by the agree callback: success commits exactly what snap_checkpoint would; a
peer that fails after the run leaves this rank's base and generation where
they were; a peer that fails at the lock stops this rank before it copies."""
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
C = 65536


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


def make_set(ts):
    s = snap.Set(chunk_bytes=C)
    for t in ts:
        s.register(t.data_ptr() if t.numel() else 0, t.numel())
    s.tensors = ts
    return s


def readback(ts):
    torch.cuda.synchronize()
    return [t.cpu().numpy().copy() if t.numel() else np.zeros(0, np.uint8) for t in ts]


def alone(phase, status):
    return status


def peer_fails_at(at):
    calls = []

    def agree(phase, status):
        calls.append((phase, status))
        return snap.ECUDA if phase == at else status
    agree.calls = calls
    return agree


@pytest.mark.parametrize("pinned", [True, False])
def test_coordinated_commit_and_peer_failures(pinned):
    ts, hs = device_state(SIZES, seed=111)
    s = make_set(ts)
    n = sum(oracle.n_chunks(x, C) for x in SIZES)

    def image(mode):
        nb = s.image_bytes(mode)
        return snap.HostBuffer(nb) if pinned else np.zeros(nb, np.uint8)

    def view(img, used):
        return img.view(used) if pinned else img[:used]

    full = image(snap.FULL)
    rc, used = s.checkpoint_coordinated(full, alone, snap.FULL)
    assert rc == snap.OK
    assert np.array_equal(view(full, used), oracle.write_full(hs, C, 0)[1])
    h0, g0 = s.committed_hashes(n)
    assert g0 == 0

    # a peer fails after the run: EPEER here, nothing committed
    g = torch.Generator(device="cuda")
    g.manual_seed(112)
    ts[10][:C] ^= torch.randint(1, 256, (C,), dtype=torch.uint8, device="cuda", generator=g)
    cur = readback(ts)
    patch = image(snap.INCREMENTAL)
    agree = peer_fails_at(1)
    rc, _ = s.checkpoint_coordinated(patch, agree, snap.INCREMENTAL)
    assert rc == snap.EPEER and agree.calls == [(0, 0), (1, 0)]
    h1, g1 = s.committed_hashes(n)
    assert g1 == g0 and np.array_equal(h1, h0)

    # a peer fails at the lock: this rank never copies
    if pinned:
        patch.array[:] = 0xA5
    else:
        patch[:] = 0xA5
    agree = peer_fails_at(0)
    rc, _ = s.checkpoint_coordinated(patch, agree, snap.INCREMENTAL)
    assert rc == snap.EPEER and agree.calls == [(0, 0)]
    assert np.all(view(patch, 4096) == 0xA5)

    # a failing transport counts as a failure too
    def broken(phase, status):
        raise RuntimeError("transport down")
    rc, _ = s.checkpoint_coordinated(patch, broken, snap.INCREMENTAL)
    assert rc == snap.EPEER

    # the next coordinated incremental is still against generation 0
    rc, used = s.checkpoint_coordinated(patch, alone, snap.INCREMENTAL)
    assert rc == snap.OK
    exp = oracle.write_patch(cur, C, [oracle.chunk_hashes(h, C) for h in hs], 1, 0)[1]
    assert np.array_equal(view(patch, used), exp)
    assert s.committed_hashes(n)[1] == 1
    # local argument errors are agreed like any other failure
    agree = peer_fails_at(-1)
    rc, _ = s.checkpoint_coordinated(patch, agree, snap.FULL, cap=4096)
    assert rc == snap.EINVAL and agree.calls == [(0, snap.EINVAL)]
    s.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_coordinated_restore_validates_everywhere_first(pinned):
    ts, hs = device_state(SIZES, seed=121)
    s = make_set(ts)
    n = sum(oracle.n_chunks(x, C) for x in SIZES)
    rc, exp = oracle.write_full(hs, C, 7)
    img = snap.HostBuffer(exp.size) if pinned else np.empty(exp.size, np.uint8)
    (img.array if pinned else img)[:] = exp
    s.checkpoint(snap.HostBuffer(s.image_bytes(snap.FULL)), snap.FULL)  # a base at generation 0
    h0, g0 = s.committed_hashes(n)
    for t in ts:
        t.zero_()
    # a peer whose image is bad: nothing changes here
    agree = peer_fails_at(0)
    assert s.restore_coordinated(img, agree) == snap.EPEER and agree.calls == [(0, 0)]
    assert all(not t.numel() or int(t.max().item()) == 0 for t in ts)
    # a peer that fails during its run: this rank's bytes are back, its base stays
    agree = peer_fails_at(1)
    assert s.restore_coordinated(img, agree) == snap.EPEER and agree.calls == [(0, 0), (1, 0)]
    for a, b in zip(readback(ts), hs):
        assert np.array_equal(a, b)
    h1, g1 = s.committed_hashes(n)
    assert g1 == g0 and np.array_equal(h1, h0)
    # everyone succeeds: the image's generation and hashes are the base
    for t in ts:
        t.zero_()
    assert s.restore_coordinated(img, alone) == snap.OK
    for a, b in zip(readback(ts), hs):
        assert np.array_equal(a, b)
    h2, g2 = s.committed_hashes(n)
    assert g2 == 7 and np.array_equal(h2, np.concatenate([oracle.chunk_hashes(h, C) for h in hs]))
    # a bad image on this rank is agreed as a failure before anything moves
    bad = exp.copy()
    bad[0] ^= 1
    agree = peer_fails_at(-1)
    assert s.restore_coordinated(bad, agree) == snap.EFORMAT and agree.calls == [(0, snap.EFORMAT)]
    s.close()
