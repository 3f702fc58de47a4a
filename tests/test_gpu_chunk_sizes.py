"""Chunk sizes that are not powers of two, and the largest chunk size.

A set's chunk size C may be any multiple of 4 KiB from 4 KiB to 16 MiB.
Every other parity test uses powers of two; here C = 12 KiB and 20 KiB (a
lane's hash segment C/32 is then 384 or 640 bytes, and a gather stage of
32 x 256 bytes does not divide the chunk) and C = 16 MiB.  At the two small
sizes the state is large enough for several allocation groups, so the
incremental checkpoint takes the fused launch with the copy engines.  Hashes,
full images, patches (pinned and pageable), restores and verify all equal
the oracle's, byte for byte."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2502_16631_b300 as snap
import workloads

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

KiB, MiB = 1 << 10, 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _oracle_threads():
    oracle.set_threads(min(16, len(os.sched_getaffinity(0))))
    yield
    oracle.set_threads(1)


def sizes_for(C):
    if C >= 16 * MiB:
        return [40 * MiB + 48, 16 * MiB, 5, 0, 17 * MiB - 16, 3 * MiB]
    # about 223 MiB: three allocation groups of the pipelined incremental
    return [3 * C + 100, C, 1, 0, 7 * C - 16, 200000, 40 * MiB + 4, 60 * MiB - 12, 33 * MiB, 90 * MiB + 17]


def device_state(sizes, seed):
    ts = []
    for k, n in enumerate(sizes):
        t = torch.empty(n + 16, dtype=torch.uint8, device="cuda")[:n]
        if n:
            workloads.torch_random_bytes(t, seed * 1000 + k)
        ts.append(t)
    torch.cuda.synchronize()
    return ts


def readback(ts):
    torch.cuda.synchronize()
    return [t.cpu().numpy().copy() if t.numel() else np.zeros(0, np.uint8) for t in ts]


def mutate(ts, C, chunks, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    for k, i in chunks:
        lo, hi = i * C, min((i + 1) * C, ts[k].numel())
        ts[k][lo:hi] ^= torch.randint(1, 256, (hi - lo,), dtype=torch.uint8, device="cuda", generator=g)
    torch.cuda.synchronize()


def dirty_plan(sizes, C, seed):
    rng = np.random.default_rng(seed)
    out = set()
    for k, n in enumerate(sizes):
        nk = (n + C - 1) // C
        if nk:
            out |= {(k, 0), (k, nk - 1), (k, int(rng.integers(0, nk)))}
    return sorted(out)


@pytest.mark.parametrize("C", [12 * KiB, 20 * KiB, 16 * MiB])
def test_odd_and_largest_chunk_sizes_match_oracle(C):
    sizes = sizes_for(C)
    ts = device_state(sizes, seed=C // 4096)
    s = snap.Set(chunk_bytes=C, ring_bytes=64 * MiB)
    for t in ts:
        s.register(t.data_ptr() if t.numel() else 0, t.numel())

    # the standalone hasher on the largest allocation
    big = max(range(len(sizes)), key=lambda k: sizes[k])
    h = torch.zeros((sizes[big] + C - 1) // C, dtype=torch.int32, device="cuda")
    snap.hash_chunks(ts[big], C, h)
    base = readback(ts)
    assert np.array_equal(h.cpu().numpy().view(np.uint32), oracle.chunk_hashes(base[big], C))

    # full and incremental checkpoints into pinned images
    full = snap.HostBuffer(s.image_bytes(snap.FULL))
    full.array[:] = 0xA5
    used = s.checkpoint(full, snap.FULL)
    rc, exp = oracle.write_full(base, C, generation=0)
    assert rc == 0 and used == exp.size and np.array_equal(full.view(used), exp)
    dirty = dirty_plan(sizes, C, seed=7)
    mutate(ts, C, dirty, seed=8)
    cur = readback(ts)
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    patch.array[:] = 0x5A
    used_p = s.checkpoint(patch, snap.INCREMENTAL)
    st = s.stats()
    rc, exp_p, nd = oracle.write_patch(cur, C, [oracle.chunk_hashes(x, C) for x in base], 1, 0)
    assert rc == 0 and nd == len(dirty) and st["dirty_chunks"] == nd
    assert used_p == exp_p.size and np.array_equal(patch.view(used_p), exp_p)
    if C < 16 * MiB:  # the fused launch ran, its dirty runs moved by the copy engines
        assert st["kernel_launches"] == 4 and 0 < st["dma_copies"] <= nd
    merged = full.view(used).copy()
    snap.apply_patch(merged, patch.view(used_p))
    assert np.array_equal(merged, oracle.write_full(cur, C, generation=1)[1])

    # pageable images through the ring
    full_p = np.full(s.image_bytes(snap.FULL), 0xA5, dtype=np.uint8)
    used2 = s.checkpoint(full_p, snap.FULL)
    assert np.array_equal(full_p[:used2], oracle.write_full(cur, C, generation=2)[1])
    dirty2 = dirty_plan(sizes, C, seed=9)
    mutate(ts, C, dirty2, seed=10)
    cur2 = readback(ts)
    patch_p = np.full(s.image_bytes(snap.INCREMENTAL), 0x5A, dtype=np.uint8)
    used3 = s.checkpoint(patch_p, snap.INCREMENTAL)
    rc, exp3, nd3 = oracle.write_patch(cur2, C, [oracle.chunk_hashes(x, C) for x in cur], 3, 2)
    assert nd3 == len(dirty2) and np.array_equal(patch_p[:used3], exp3)

    # restore the generation-2 image (state `cur`) into scribbled buffers
    for t in ts:
        if t.numel():
            t.fill_(0x3C)
    s.restore(full_p, used2)
    for a, b in zip(readback(ts), cur):
        assert np.array_equal(a, b)
    assert s.verify(full_p, used2) == 0
    s.close()
