"""Serving loop: every request's result is the same alone and in the mix.

Tenant requests (full checkpoints, incremental checkpoints, restores) are
submitted together so that their tiles share batched launches, then the
same requests are replayed one at a time on identically prepared tenants.
Images, patches and restored bytes must be identical between the two runs
and equal to the CPU oracle (tolerance 0: this is byte work)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2502_16631_b300 as snap
import workloads

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

C = 65536
MiB = 1 << 20


def tenant_sizes(t):
    rng = np.random.default_rng(100 + t)
    return [int(x) for x in rng.integers(1, 6 * MiB, 6)] + [C * 3]


# Large-request case: tenants 0, 2 and 4 hold about 700 MiB in ten
# allocations, so with a 1 GiB staging pool (16 slots of 64 MiB) each of
# their full checkpoints, incremental checkpoints (most chunks dirty) and
# restores spans more windows than the scheduler gives one request per round
# (8); the other tenants stay small.
BIG_TENANTS = (0, 2, 4)
BIG_POOL = 1 << 30
BIG_SLOT = 64 * MiB


def big_tenant_sizes(t):
    rng = np.random.default_rng(200 + t)
    if t in BIG_TENANTS:
        return [int(x) // 16 * 16 + 16 * (k % 3) + 1 for k, x in enumerate(rng.integers(40 * MiB, 100 * MiB, 10))]
    return [int(x) for x in rng.integers(1, 6 * MiB, 4)] + [C * 3]


def make_tenants(n, seed, sizes_of=tenant_sizes):
    tenants = []
    for t in range(n):
        sizes = sizes_of(t)
        ts = []
        for k, nbytes in enumerate(sizes):
            d = torch.empty(nbytes + 16, dtype=torch.uint8, device="cuda")[:nbytes]
            d.copy_(torch.from_numpy(workloads.xorshift_bytes(nbytes, seed + t, k)))
            ts.append(d)
        s = snap.Set(chunk_bytes=C)
        for d in ts:
            s.register(d)
        tenants.append((s, ts))
    torch.cuda.synchronize()
    return tenants


def host(ts):
    torch.cuda.synchronize()
    return [d.cpu().numpy().copy() for d in ts]


def mutate(ts, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    for k, d in enumerate(ts):
        n = (d.numel() + C - 1) // C
        for i in range(0, n, 7):  # every 7th chunk
            lo, hi = i * C, min((i + 1) * C, d.numel())
            d[lo:hi] ^= torch.randint(1, 256, (hi - lo,), dtype=torch.uint8, device="cuda", generator=g)
    torch.cuda.synchronize()


def mutate_most(ts, seed):
    """Every chunk but each tenth changes in every byte (and every ragged
    last chunk): most of the tenant is dirty."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    for d in ts:
        nf = d.numel() // C
        if nf:
            rows = d[: nf * C].view(nf, C)
            idx = torch.tensor([i for i in range(nf) if i % 10], dtype=torch.long, device="cuda")
            if idx.numel():
                rows[idx] ^= torch.randint(1, 256, (idx.numel(), C), dtype=torch.uint8, device="cuda", generator=g)
        if d.numel() > nf * C:
            tail = d[nf * C:]
            tail ^= torch.randint(1, 256, (tail.numel(),), dtype=torch.uint8, device="cuda", generator=g)
    torch.cuda.synchronize()


PINNED = (0, 3, 4)  # tenants whose images are pinned (direct windows) when pinned=True


def scenario(mixed: bool, pinned: bool = False, big: bool = False):
    """Phase 1: full checkpoints of 6 tenants; phase 2: incremental (t0, t1),
    full (t2, t3), restore of the phase-1 image after scribbling (t4, t5).
    With `pinned`, the images of tenants PINNED are registered, so the server
    reads and writes them directly, and the others stay pageable (staged).
    With `big`, tenants BIG_TENANTS are large, tenant 0's incremental finds
    most chunks dirty, and the staging pool is BIG_POOL."""
    if big:
        tenants = make_tenants(6, seed=550, sizes_of=big_tenant_sizes)
        sv = snap.Server(pinned_budget=BIG_POOL, hbm_budget=1 << 40, chunk_bytes=C, ring_bytes=BIG_POOL)
    else:
        tenants = make_tenants(6, seed=500)
        sv = snap.Server(pinned_budget=64 * MiB, hbm_budget=1 << 40, chunk_bytes=C)
    imgs = [np.full(s.image_bytes(snap.FULL), 0xA5, dtype=np.uint8) for s, _ in tenants]
    patches = [np.full(s.image_bytes(snap.INCREMENTAL), 0x5A, dtype=np.uint8) for s, _ in tenants]
    registered = []
    if pinned:
        for t in PINNED:
            for a in (imgs[t], patches[t]):
                snap.host_register(a)
                registered.append(a)
    out = {"phase1_state": [host(ts) for _, ts in tenants]}

    def run(reqs):
        if mixed:
            tickets = [sv.submit(s, kind, buf) for s, kind, buf in reqs]
            res = [sv.wait(t, 120000) for t in tickets]
        else:
            res = [sv.wait(sv.submit(s, kind, buf), 120000) for s, kind, buf in reqs]
        for rc, status, st in res:
            assert rc == snap.OK and status == snap.OK, (rc, status)
        return [st for _, _, st in res]

    stats1 = run([(s, snap.REQ_FULL, imgs[t]) for t, (s, _) in enumerate(tenants)])
    out["full1"] = [imgs[t][: stats1[t]["image_bytes"]].copy() for t in range(6)]
    for t in (0, 1, 2, 3):
        if big and t == 0:
            mutate_most(tenants[t][1], seed=900 + t)
        else:
            mutate(tenants[t][1], seed=900 + t)
    for t in (4, 5):
        for d in tenants[t][1]:
            d.fill_(0x33)
    out["phase2_state"] = [host(ts) for _, ts in tenants]
    full2 = [np.full(s.image_bytes(snap.FULL), 0xA5, dtype=np.uint8) for s, _ in tenants]
    if pinned:
        for t in PINNED:
            snap.host_register(full2[t])
            registered.append(full2[t])
    reqs = [(tenants[0][0], snap.REQ_INCREMENTAL, patches[0]), (tenants[1][0], snap.REQ_INCREMENTAL, patches[1]),
            (tenants[2][0], snap.REQ_FULL, full2[2]), (tenants[3][0], snap.REQ_FULL, full2[3]),
            (tenants[4][0], snap.REQ_RESTORE, imgs[4]), (tenants[5][0], snap.REQ_RESTORE, imgs[5])]
    stats2 = run(reqs)
    out["incr"] = [patches[t][: stats2[t]["image_bytes"]].copy() for t in (0, 1)]
    out["dirty"] = [stats2[t]["dirty_chunks"] for t in (0, 1)]
    out["full2"] = [full2[t][: stats2[t]["image_bytes"]].copy() for t in (2, 3)]
    out["restored"] = [host(tenants[t][1]) for t in (4, 5)]
    out["latency_ms"] = [st["total_ms"] for st in stats1 + stats2]
    sv.close()
    for a in registered:
        snap.host_unregister(a)
    return out


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("big", [False, True])
def test_serving_mix_equals_alone_equals_oracle(pinned, big):
    """Alone == in the mix == oracle, with small tenants, and (big) with
    full, incremental and restore requests that each span more windows than
    one request may put into a round, so that the per-request round cap and
    the shortest-remaining-first order act while they run."""
    if big:
        for t in BIG_TENANTS:
            assert sum(big_tenant_sizes(t)) > 8 * BIG_SLOT  # more windows than the round cap
        # tenant 0's incremental (9 in 10 chunks dirty) has more dirty windows than the cap too
        assert 0.85 * sum(big_tenant_sizes(0)) > 8 * BIG_SLOT
    mixed = scenario(mixed=True, pinned=pinned, big=big)
    alone = scenario(mixed=False, pinned=pinned, big=big)
    for key in ("full1", "incr", "full2"):
        for a, b in zip(mixed[key], alone[key]):
            assert np.array_equal(a, b), key
    for ta, tb in zip(mixed["restored"], alone["restored"]):
        for a, b in zip(ta, tb):
            assert np.array_equal(a, b)
    # against the oracle
    for t in range(6):
        assert np.array_equal(mixed["full1"][t], oracle.write_full(mixed["phase1_state"][t], C, 0)[1])
    for j, t in enumerate((0, 1)):
        prev = [oracle.chunk_hashes(h, C) for h in mixed["phase1_state"][t]]
        rc, exp, nd = oracle.write_patch(mixed["phase2_state"][t], C, prev, 1, 0)
        assert nd == mixed["dirty"][j] and np.array_equal(mixed["incr"][j], exp)
    for j, t in enumerate((2, 3)):
        assert np.array_equal(mixed["full2"][j], oracle.write_full(mixed["phase2_state"][t], C, 1)[1])
    for j, t in enumerate((4, 5)):
        for a, b in zip(mixed["restored"][j], mixed["phase1_state"][t]):
            assert np.array_equal(a, b)
    assert all(x > 0 for x in mixed["latency_ms"])


def test_serving_budget_refusal():
    tenants = make_tenants(1, seed=600)
    s, _ = tenants[0]
    sv = snap.Server(pinned_budget=64 * MiB, hbm_budget=1 * MiB, chunk_bytes=C)
    img = np.zeros(s.image_bytes(snap.FULL), dtype=np.uint8)
    with pytest.raises(snap.SnapError) as e:
        sv.submit(s, snap.REQ_FULL, img)
    assert e.value.status == snap.EBUDGET
    sv.close()


def test_serving_incremental_without_base_fails_cleanly():
    tenants = make_tenants(1, seed=700)
    s, ts = tenants[0]
    sv = snap.Server(pinned_budget=64 * MiB, hbm_budget=1 << 40, chunk_bytes=C)
    patch = np.zeros(s.image_bytes(snap.INCREMENTAL), dtype=np.uint8)
    rc, status, _ = sv.wait(sv.submit(s, snap.REQ_INCREMENTAL, patch), 60000)
    assert rc == snap.OK and status == snap.ENOBASE
    img = np.zeros(s.image_bytes(snap.FULL), dtype=np.uint8)
    rc, status, st = sv.wait(sv.submit(s, snap.REQ_FULL, img), 60000)
    assert status == snap.OK
    assert np.array_equal(img[: st["image_bytes"]], oracle.write_full(host(ts), C, 0)[1])
    sv.close()
