"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Everything here is integer/byte work, so the bar is bit-exact: every image
byte, every hash and every restored byte equals what the oracle computes from
the same device bytes (read back with a plain device-to-host copy, not
through the library)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2502_16631_b300 as snap
import workloads

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

KiB, MiB, GiB = 1 << 10, 1 << 20, 1 << 30


@pytest.fixture(scope="module", autouse=True)
def _oracle_threads():
    oracle.set_threads(min(16, len(os.sched_getaffinity(0))))
    yield
    oracle.set_threads(1)


def device_state(sizes, seed=1, offset=0):
    """Device buffers with xorshift64* contents; returns (tensors, host copies).
    offset (multiple of 16) shifts each buffer inside a larger allocation."""
    ts, hs = [], []
    for k, s in enumerate(sizes):
        h = workloads.xorshift_bytes(s, seed, k)
        base = torch.empty(s + offset + 16, dtype=torch.uint8, device="cuda")
        t = base[offset: offset + s]
        if s:
            t.copy_(torch.from_numpy(h))
        ts.append(t)
        hs.append(h)
    torch.cuda.synchronize()
    return ts, hs


def readback(ts):
    torch.cuda.synchronize()
    return [t.cpu().numpy().copy() if t.numel() else np.zeros(0, np.uint8) for t in ts]


def make_set(ts, C=65536, **kw):
    s = snap.Set(chunk_bytes=C, **kw)
    for t in ts:
        s.register(t.data_ptr() if t.numel() else 0, t.numel())
    s.tensors = ts
    return s


# ------------------------------------------------------------ chunk hasher
@pytest.mark.parametrize("C", [4096, 16384, 65536, 1 << 20])
def test_hash_chunks_lengths(C):
    rng = np.random.default_rng(C)
    big = rng.integers(0, 256, 3 * C + 8192, dtype=np.uint8)
    dbig = torch.from_numpy(big).cuda()
    lengths = sorted(set([1, 2, 15, 16, 17, 31, 33, 100, 511, 513, 4095, 4096, 4097,
                          C - 16, C - 1, C, C + 1, C + 15, 2 * C + 48, 3 * C + 8192]
                         + list(rng.integers(1, 3 * C + 8192, 12))))
    out = torch.zeros(8, dtype=torch.int32, device="cuda")
    for n in lengths:
        n = int(n)
        nch = (n + C - 1) // C
        out = torch.zeros(nch, dtype=torch.int32, device="cuda")
        snap.hash_chunks(dbig, C, out, nbytes=n)
        got = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, oracle.chunk_hashes(big[:n], C)), (C, n)


def test_hash_chunks_every_small_length():
    rng = np.random.default_rng(5)
    big = rng.integers(0, 256, 4096 + 600, dtype=np.uint8)
    dbig = torch.from_numpy(big).cuda()
    out = torch.zeros(2, dtype=torch.int32, device="cuda")
    for n in range(1, 600):
        snap.hash_chunks(dbig, 4096, out, nbytes=n)
        assert int(out[0].item()) & 0xFFFFFFFF == oracle.crc32c(big[:n]), n


def test_hash_chunks_offsets_and_alignment():
    rng = np.random.default_rng(6)
    big = rng.integers(0, 256, 1 << 20, dtype=np.uint8)
    dbig = torch.from_numpy(big).cuda()
    out = torch.zeros(64, dtype=torch.int32, device="cuda")
    for off in (16, 48, 4096 + 32, 65536 + 16):
        n = (1 << 20) - off - 5
        snap.hash_chunks(dbig.data_ptr() + off, 65536, out, nbytes=n)
        exp = oracle.chunk_hashes(big[off: off + n], 65536)
        assert np.array_equal(out[: exp.size].cpu().numpy().view(np.uint32), exp)
    # a device pointer that is not 16-byte aligned is refused, not read
    rc = snap.lib().snap_hash_chunks(dbig.data_ptr() + 3, 100, 65536, out.data_ptr(), None)
    assert rc == snap.EINVAL


def test_hash_chunks_check_value():
    d = torch.tensor(list(b"123456789"), dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    snap.hash_chunks(d, 4096, out)
    assert int(out.item()) & 0xFFFFFFFF == 0xE3069283


# ------------------------------------------------------ full image, restore
SIZES_EDGE = [65536, 4096 * 3 + 16, 1, 0, 200000, 65536 * 2, 12345, 17, 65537, 3 * 65536 - 1]


@pytest.mark.parametrize("C", [4096, 65536, 1 << 20])
def test_full_checkpoint_matches_oracle(C):
    ts, _ = device_state(SIZES_EDGE, seed=11)
    s = make_set(ts, C)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    img.array[:] = 0xA5  # garbage: every padding byte must be written
    used = s.checkpoint(img, snap.FULL)
    rc, exp = oracle.write_full(readback(ts), C, generation=0)
    assert rc == 0 and used == exp.size
    assert np.array_equal(img.view(used), exp)
    # second checkpoint: generation 1
    used = s.checkpoint(img, snap.FULL)
    rc, exp = oracle.write_full(readback(ts), C, generation=1)
    assert np.array_equal(img.view(used), exp)


def test_config1_roundtrip():
    sizes = workloads.config1_sizes(1)
    ts, hs = device_state(sizes, seed=1)
    s = make_set(ts, 65536)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    used = s.checkpoint(img, snap.FULL)
    rc, exp = oracle.write_full(hs, 65536, 0)
    assert np.array_equal(img.view(used), exp)
    for t in ts:
        t.zero_()
    s.restore(img, used)
    for t, h in zip(readback(ts), hs):
        assert np.array_equal(t, h)
    assert s.verify(img, used) == 0
    # committed hashes = image hashes, generation adopted
    hh, gen = s.committed_hashes(sum((x + 65535) // 65536 for x in sizes))
    assert gen == 0
    assert np.array_equal(hh, np.concatenate([oracle.chunk_hashes(h, 65536) for h in hs]))


def test_restore_into_fresh_buffers_and_verify_counts():
    ts, hs = device_state(SIZES_EDGE, seed=12)
    s = make_set(ts, 4096)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    used = s.checkpoint(img, snap.FULL)
    fresh = [torch.zeros_like(t) for t in ts]
    s2 = make_set(fresh, 4096)
    s2.restore(img, used)
    for a, b in zip(readback(fresh), hs):
        assert np.array_equal(a, b)
    # corrupt two chunks on the device: verify counts exactly those
    fresh[4][5000] ^= 1
    fresh[0][0] ^= 0x80
    assert s2.verify(img, used) == 2


def test_plain_form_data_regions():
    ts, hs = device_state(SIZES_EDGE, seed=13)
    s = make_set(ts, 65536)
    n = s.image_bytes(snap.FULL)
    img = snap.HostBuffer(n)
    s.plain_checkpoint(img)
    rc, exp = oracle.write_full(hs, 65536, 0)
    # data regions equal the oracle's (headers/hashes are not written by the plain form)
    off = 64
    for h in hs:
        nk = (h.size + 65535) // 65536
        d = (off + 32 + 4 * nk + 4095) // 4096 * 4096
        assert np.array_equal(img.array[d: d + h.size], h)
        off = (d + h.size + 4095) // 4096 * 4096
    for t in ts:
        t.zero_()
    s.plain_restore(img)
    for a, b in zip(readback(ts), hs):
        assert np.array_equal(a, b)


# -------------------------------------------------------------- incremental
def mutate(ts, C, chunks, seed=9):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    for k, i in chunks:
        lo, hi = i * C, min((i + 1) * C, ts[k].numel())
        x = torch.randint(1, 256, (hi - lo,), dtype=torch.uint8, device="cuda", generator=g)
        ts[k][lo:hi] ^= x
    torch.cuda.synchronize()


@pytest.mark.parametrize("C", [4096, 65536])
def test_incremental_patch_matches_oracle(C):
    ts, _ = device_state(SIZES_EDGE, seed=14)
    s = make_set(ts, C)
    full = snap.HostBuffer(s.image_bytes(snap.FULL))
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    patch.array[:] = 0x5A
    used0 = s.checkpoint(full, snap.FULL)
    base = readback(ts)
    prev = [oracle.chunk_hashes(h, C) for h in base]
    nch = [(x + C - 1) // C for x in SIZES_EDGE]
    dirty = [(0, 0), (2, 0), (4, nch[4] - 1), (5, 1), (6, 0), (9, nch[9] - 1), (8, 1)]
    mutate(ts, C, dirty)
    used = s.checkpoint(patch, snap.INCREMENTAL)
    cur = readback(ts)
    rc, exp, nd = oracle.write_patch(cur, C, prev, generation=1, parent=0)
    assert rc == 0 and nd == len(set(dirty))
    assert used == exp.size
    assert np.array_equal(patch.view(used), exp)
    assert s.stats()["dirty_chunks"] == nd
    # previous image + patch == full image of the current state
    merged = full.view(used0).copy()
    snap.apply_patch(merged, patch.view(used))
    rc, full1 = oracle.write_full(cur, C, generation=1)
    assert np.array_equal(merged, full1)
    # a second incremental with nothing changed: headers and hashes only
    used2 = s.checkpoint(patch, snap.INCREMENTAL)
    rc, exp2, nd2 = oracle.write_patch(cur, C, [oracle.chunk_hashes(h, C) for h in cur], 2, 1)
    assert nd2 == 0 and np.array_equal(patch.view(used2), exp2)


def test_incremental_everything_dirty():
    C = 4096
    ts, _ = device_state([C * 5, C * 3 + 100, 77], seed=15)
    s = make_set(ts, C)
    full = snap.HostBuffer(s.image_bytes(snap.FULL))
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    used0 = s.checkpoint(full, snap.FULL)
    prev = [oracle.chunk_hashes(h, C) for h in readback(ts)]
    mutate(ts, C, [(k, i) for k, t in enumerate(ts) for i in range((t.numel() + C - 1) // C)])
    used = s.checkpoint(patch, snap.INCREMENTAL)
    cur = readback(ts)
    rc, exp, nd = oracle.write_patch(cur, C, prev, 1, 0)
    assert np.array_equal(patch.view(used), exp)
    merged = full.view(used0).copy()
    snap.apply_patch(merged, patch.view(used))
    assert np.array_equal(merged, oracle.write_full(cur, C, 1)[1])


def test_incremental_errors_keep_base():
    C = 4096
    ts, _ = device_state([C * 8], seed=16)
    s = make_set(ts, C)
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    rc, _ = s.checkpoint_status(patch, snap.INCREMENTAL)
    assert rc == snap.ENOBASE
    full = snap.HostBuffer(s.image_bytes(snap.FULL))
    s.checkpoint(full, snap.FULL)
    h0, g0 = s.committed_hashes(8)
    mutate(ts, C, [(0, i) for i in range(8)])
    # capacity too small for the patch: EINVAL, and nothing is committed
    rc, _ = s.checkpoint_status(patch, snap.INCREMENTAL, cap=C * 2)
    assert rc == snap.EINVAL
    h1, g1 = s.committed_hashes(8)
    assert np.array_equal(h0, h1) and g0 == g1
    used = s.checkpoint(patch, snap.INCREMENTAL)
    assert s.stats()["dirty_chunks"] == 8 and used > 8 * C


# ----------------------------------------------- pageable images via the ring
@pytest.mark.parametrize("C,ring", [(4096, 1 << 20), (65536, 2 << 20)])
def test_ring_pageable_images(C, ring):
    """Images in ordinary (pageable) host memory stream through a small
    pinned ring: many windows, slot reuse, ragged allocations."""
    sizes = [8 * C + 100, 3 * C, 1, 0, 200000, C + 1, 70 * C]
    ts, hs = device_state(sizes, seed=41)
    s = make_set(ts, C, ring_bytes=ring)
    s.prepare(layout=True, ring=True)
    full = np.full(s.image_bytes(snap.FULL), 0xA5, dtype=np.uint8)  # pageable
    used = s.checkpoint(full, snap.FULL)
    assert np.array_equal(full[:used], oracle.write_full(hs, C, 0)[1])
    assert s.verify(full, used) == 0
    # incremental into a pageable patch
    nch = [(n + C - 1) // C for n in sizes]
    dirty = [(0, 0), (0, nch[0] - 1), (4, 2), (6, 5), (6, 6), (6, 69), (2, 0)]
    mutate(ts, C, dirty)
    patch = np.full(s.image_bytes(snap.INCREMENTAL), 0x5A, dtype=np.uint8)
    used_p = s.checkpoint(patch, snap.INCREMENTAL)
    cur = readback(ts)
    rc, exp, nd = oracle.write_patch(cur, C, [oracle.chunk_hashes(h, C) for h in hs], 1, 0)
    assert nd == len(set(dirty)) and np.array_equal(patch[:used_p], exp)
    # restore the generation-0 image from pageable memory
    for t in ts:
        t.zero_()
    s.restore(full, used)
    for a, b in zip(readback(ts), hs):
        assert np.array_equal(a, b)
    assert s.committed_hashes(sum(nch))[1] == 0


def test_registered_numpy_image_is_used_directly():
    """A caller's numpy buffer pinned with host_register is an image like
    snap_host_alloc memory: the full image equals the oracle's, an
    incremental patch too, and the restore from it brings every byte back;
    unregistering twice is EINVAL."""
    C = 65536
    sizes = [3 * C + 100, C, 0, 5000, 2 * C]
    ts, hs = device_state(sizes, seed=61)
    s = make_set(ts, C)
    full = np.full(s.image_bytes(snap.FULL), 0xA5, dtype=np.uint8)
    patch = np.full(s.image_bytes(snap.INCREMENTAL), 0x5A, dtype=np.uint8)
    snap.host_register(full)
    snap.host_register(patch)
    try:
        used = s.checkpoint(full, snap.FULL)
        assert np.array_equal(full[:used], oracle.write_full(hs, C, 0)[1])
        mutate(ts, C, [(0, 1), (4, 1)])
        cur = readback(ts)
        used_p = s.checkpoint(patch, snap.INCREMENTAL)
        exp = oracle.write_patch(cur, C, [oracle.chunk_hashes(h, C) for h in hs], 1, 0)[1]
        assert used_p == exp.size and np.array_equal(patch[:used_p], exp)
        for d in ts:
            d.zero_()
        s.restore(full, used)
        for a, b in zip(readback(ts), hs):
            assert np.array_equal(a, b)
    finally:
        snap.host_unregister(full)
        snap.host_unregister(patch)
    with pytest.raises(snap.SnapError) as e:
        snap.host_unregister(full)
    assert e.value.status == snap.EINVAL


def test_partly_registered_image_is_staged_not_mapped():
    """An image buffer of which only a part is pinned (or which two separate
    registrations cover) is not read or written through its mapping: the
    synchronous calls stage it through the ring and still match the oracle,
    and the calls that need a mapping over the whole image (asynchronous
    checkpoint, prioritised restore) refuse it with EINVAL."""
    C = 65536
    sizes = [5 * C + 100, 2 * C, 0, 7000, 3 * C]
    ts, hs = device_state(sizes, seed=67)
    s = make_set(ts, C, ring_bytes=1 << 20)
    n = s.image_bytes(snap.FULL)
    import mmap
    m = mmap.mmap(-1, n + 8192)  # page-aligned, so the two halves share no page
    full = np.frombuffer(m, dtype=np.uint8)
    full[:] = 0xA5
    half = (n // 2) & ~4095
    lo, hi = full[:half], full[half:]
    snap.host_register(lo)
    try:
        exp = oracle.write_full(hs, C, 0)[1]
        used = s.checkpoint(full, snap.FULL)
        assert np.array_equal(full[:used], exp)
        assert s.checkpoint_async_status(full, snap.FULL) == snap.EINVAL
        assert s.restore_async_status(full, (), used) == snap.EINVAL
        for d in ts:
            d.zero_()
        s.restore(full, used)
        for a, b in zip(readback(ts), hs):
            assert np.array_equal(a, b)
        # two registrations side by side still leave the image in two regions
        # (the restore above adopted generation 0, so this checkpoint is 1)
        snap.host_register(hi)
        try:
            full[:used] = 0
            used = s.checkpoint(full, snap.FULL)
            assert np.array_equal(full[:used], oracle.write_full(hs, C, 1)[1])
            assert s.checkpoint_async_status(full, snap.FULL) == snap.EINVAL
            for d in ts:
                d.zero_()
            s.restore(full, used)
            for a, b in zip(readback(ts), hs):
                assert np.array_equal(a, b)
        finally:
            snap.host_unregister(hi)
    finally:
        snap.host_unregister(lo)
    s.close()
    del lo, hi, full
    m.close()
    s.close()


def test_ring_pageable_windows_smaller_than_slots():
    """A 640 MiB state through a 4 GiB ring: windows of about 20 MiB (1/32
    of the state) in 256 MiB slots, 32 or more of them, so the 16 slots are
    reused; the pageable full image equals the oracle's and the restore from
    it brings every byte back."""
    C = 65536
    sizes, ts = _pipeline_state(57)
    s = make_set(ts, C, ring_bytes=4 << 30)
    full = np.full(s.image_bytes(snap.FULL), 0xA5, dtype=np.uint8)
    base = readback(ts)
    used = s.checkpoint(full, snap.FULL)
    rc, exp = oracle.write_full(base, C, 0)
    assert rc == 0 and used == exp.size and np.array_equal(full[:used], exp)
    for t in ts:
        t.zero_()
    s.restore(full, used)
    for a, b in zip(readback(ts), base):
        assert np.array_equal(a, b)
    s.close()


def test_ring_pageable_incremental_many_windows():
    """A patch of thousands of dirty chunks into a pageable image: the ring
    path cuts the dirty ranks into one window per slot (16 here), each copied
    out by parallel parts of about 1 MiB; every third allocation has no dirty
    chunk, so parts start and end inside and between allocations."""
    C = 65536
    sizes, ts = _pipeline_state(53)
    s = make_set(ts, C, ring_bytes=1 << 30)
    full = np.empty(s.image_bytes(snap.FULL), dtype=np.uint8)
    s.checkpoint(full, snap.FULL)
    base = readback(ts)
    nch = [(n + C - 1) // C for n in sizes]
    rng = np.random.default_rng(54)
    dirty = sorted((k, i) for k, n in enumerate(nch) if k % 3 for i in range(n) if rng.random() < 0.7)
    assert len(dirty) > 4096  # windows of more than 16 MiB
    mutate(ts, C, dirty, seed=55)
    cur = readback(ts)
    patch = np.full(s.image_bytes(snap.INCREMENTAL), 0x5A, dtype=np.uint8)
    used = s.checkpoint(patch, snap.INCREMENTAL)
    rc, exp, nd = oracle.write_patch(cur, C, [oracle.chunk_hashes(h, C) for h in base], 1, 0)
    assert rc == 0 and nd == len(dirty) and s.stats()["dirty_chunks"] == nd
    assert used == exp.size and np.array_equal(patch[:used], exp)
    s.close()


# ------------------------------------------------------------- autotuner
@pytest.mark.parametrize("C", [4096, 65536])
def test_autotune_every_shape_agrees_then_parity(C):
    """The autotuner runs every launch shape (warps, stages, piece bytes,
    one or two CRC chains per lane) and fails if any two disagree on a
    single chunk hash; the adopted shape must still match the oracle."""
    sizes = [8 * C, 3 * C + 4096 + 16, 100000, 12345, C]
    ts, hs = device_state(sizes, seed=31)
    s = make_set(ts, C)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    t_inc = s.autotune(snap.INCREMENTAL)
    t_full = s.autotune(snap.FULL, img)
    assert t_inc["gbs"] > 0 and t_full["gbs"] > 0
    used = s.checkpoint(img, snap.FULL)
    assert np.array_equal(img.view(used), oracle.write_full(hs, C, 0)[1])
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    mutate(ts, C, [(0, 3), (3, 0)])
    used_p = s.checkpoint(patch, snap.INCREMENTAL)
    assert s.verify(patch, used_p) == 0
    rc, exp, nd = oracle.write_patch(readback(ts), C, [oracle.chunk_hashes(h, C) for h in hs], 1, 0)
    assert nd == 2 and np.array_equal(patch.view(used_p), exp)


def _shape(t):
    return tuple(t[k] for k in ("warps", "stages", "piece_bytes", "chains", "tma", "ctas_per_sm"))


def test_autotune_cache_is_read_back(tmp_path, monkeypatch):
    """A set tuned once stores its winners in $SNAP_TUNE_CACHE; a new set of
    the same GPU, chunk size and state size class starts with those shapes,
    and its images still equal the oracle's.  A hand-written entry with a
    shape no default uses is adopted the same way; an entry for another size
    class, or an invalid shape, is not."""
    import math
    C = 65536
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("SNAP_TUNE_CACHE", str(cache))
    sizes = [8 * C, 3 * C + 4096 + 16, 100000, 12345, C]
    ts, hs = device_state(sizes, seed=35)
    a = make_set(ts, C)
    img = snap.HostBuffer(a.image_bytes(snap.FULL))
    t_inc = a.autotune(snap.INCREMENTAL)
    t_full = a.autotune(snap.FULL, img)
    assert cache.exists() and len(cache.read_text().splitlines()) == 2
    ts2, hs2 = device_state(sizes, seed=36)
    b = make_set(ts2, C)
    assert _shape(b.tuning(snap.INCREMENTAL)) == _shape(t_inc)
    assert _shape(b.tuning(snap.FULL)) == _shape(t_full)
    img2 = snap.HostBuffer(b.image_bytes(snap.FULL))
    used = b.checkpoint(img2, snap.FULL)
    assert np.array_equal(img2.view(used), oracle.write_full(hs2, C, 0)[1])
    patch = snap.HostBuffer(b.image_bytes(snap.INCREMENTAL))
    mutate(ts2, C, [(0, 5), (2, 1)])
    used_p = b.checkpoint(patch, snap.INCREMENTAL)
    rc, exp, nd = oracle.write_patch(readback(ts2), C, [oracle.chunk_hashes(h, C) for h in hs2], 1, 0)
    assert nd == 2 and np.array_equal(patch.view(used_p), exp)
    # a hand-written entry: 16 warps, 3 stages, 32-byte pieces for the hash
    # pass (the default is 24 / 2 / 64), appended after the tuned one
    gpu = torch.cuda.get_device_name()
    cls = int(math.floor(math.log2(sum(sizes))))
    ctas = torch.cuda.get_device_properties(0).multi_processor_count
    entry = ('{"gpu": "%s", "op": 1, "chunk": %d, "class": %d, "warps": 16, "stages": 3, "piece": 32, '
             '"chains": 1, "tma": 0, "ctas": %d, "gbs": 1.0}\n')
    with open(cache, "a") as f:
        f.write(entry % (gpu, C, cls + 1, ctas))  # another size class: ignored
        f.write(entry.replace('"warps": 16', '"warps": 7') % (gpu, C, cls, ctas))  # not a tunable shape
        f.write(entry % (gpu, C, cls, ctas))
    ts3, hs3 = device_state(sizes, seed=37)
    c = make_set(ts3, C)
    t3 = c.tuning(snap.INCREMENTAL)
    assert (t3["warps"], t3["stages"], t3["piece_bytes"], t3["chains"], t3["tma"]) == (16, 3, 32, 1, 0)
    assert _shape(c.tuning(snap.FULL)) == _shape(t_full)
    used = c.checkpoint(img2, snap.FULL)
    assert np.array_equal(img2.view(used), oracle.write_full(hs3, C, 0)[1])
    assert c.verify(img2, used) == 0
    # without the cache file a new set keeps the defaults
    monkeypatch.delenv("SNAP_TUNE_CACHE")
    d = make_set(ts3, C)
    t4 = d.tuning(snap.INCREMENTAL)
    assert (t4["warps"], t4["stages"], t4["piece_bytes"]) == (24, 2, 64)
    for x in (a, b, c, d):
        x.close()


def test_device_wait_gives_up_and_the_set_recovers(monkeypatch):
    """The kernels' own give-up path, reached without a fault: with the test
    hook SNAP_TEST_STALL_TILE the warp that takes that tile waits on a stage
    whose bytes no copy delivers, so its bounded mbarrier wait (2 s) runs
    out; it records ERR_WAIT_TIMEOUT, drains and leaves, every other warp
    leaves at its next tile, and the call returns SNAP_ECUDA well inside the
    call deadline with nothing committed (Sec. 3.1.1: a lock that times out
    rolls back).  Checked on a full checkpoint (general kernel) and on verify
    (the hash-only kernel); the next calls succeed and match the oracle."""
    import time
    C = 65536
    sizes = [40 * C + 100, 3 * C, 12345]
    ts, hs = device_state(sizes, seed=71)
    s = make_set(ts, C)
    nch = sum((n + C - 1) // C for n in sizes)
    full = snap.HostBuffer(s.image_bytes(snap.FULL))
    used = s.checkpoint(full, snap.FULL)
    base, gen = s.committed_hashes(nch)
    base = base.copy()
    assert s.stats()["device_errors"] == 0
    mutate(ts, C, [(0, 7), (2, 0)])
    cur = readback(ts)
    img2 = snap.HostBuffer(s.image_bytes(snap.FULL))
    monkeypatch.setenv("SNAP_TEST_STALL_TILE", "5")
    t0 = time.perf_counter()
    rc, _ = s.checkpoint_status(img2, snap.FULL)
    dt = time.perf_counter() - t0
    assert rc == snap.ECUDA and s.stats()["device_errors"] == 1
    assert dt < 8.0  # two bounded waits of the stalled warp; the call deadline is 10 s
    b2, g2 = s.committed_hashes(nch)
    assert g2 == gen and np.array_equal(b2, base)
    with pytest.raises(snap.SnapError) as e:
        s.verify(full, used)
    assert e.value.status == snap.ECUDA and s.stats()["device_errors"] == 1
    monkeypatch.delenv("SNAP_TEST_STALL_TILE")
    used2 = s.checkpoint(img2, snap.FULL)
    assert s.stats()["device_errors"] == 0
    assert np.array_equal(img2.view(used2), oracle.write_full(cur, C, 1)[1])
    assert s.verify(img2, used2) == 0
    s.close()


def test_measurement_probes_report_rates():
    """The two measurement probes the bench reports its ceilings from: the
    SM-path link rate in each direction and both at once, and the host copy
    rate between pinned and pageable memory in each direction, both at once,
    and under link load -- each a positive rate below anything physical."""
    for d in (0, 1, 2):
        v = snap.link_ceiling(d, 64 << 20, 2)
        assert 1.0 < v < 500.0, (d, v)
    for d, th in ((0, 2), (1, 2), (2, 4)):
        v = snap.host_copy_ceiling(th, d, 64 << 20, 2)
        assert 0.1 < v < 2000.0, (d, v)
    v = snap.host_copy_ceiling(4, 2, 64 << 20, 1, with_link=True)
    assert 0.1 < v < 2000.0


def test_stats_report_phases():
    ts, _ = device_state([64 * 65536], seed=32)
    s = make_set(ts, 65536)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    s.checkpoint(img, snap.FULL)
    st = s.stats()
    assert st["copy_ms"] > 0 and st["kernel_launches"] >= 3 and st["total_ms"] >= st["copy_ms"]
    mutate(ts, 65536, [(0, 5)])
    s.checkpoint(patch, snap.INCREMENTAL)
    st = s.stats()
    assert st["hash_ms"] > 0 and st["diff_ms"] > 0 and st["dirty_chunks"] == 1


# ----------------------------------------------------------------- errors
def test_restore_rejects_mismatch_and_bad_images():
    ts, _ = device_state([65536, 5000], seed=17)
    s = make_set(ts, 65536)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    used = s.checkpoint(img, snap.FULL)
    other, _ = device_state([65536, 5001], seed=17)
    s2 = make_set(other, 65536)
    assert s2.restore_status(img, used) == snap.EMISMATCH
    s3 = make_set(other[:1], 65536)
    assert s3.restore_status(img, used) == snap.EMISMATCH
    s4 = make_set(ts, 4096)
    assert s4.restore_status(img, used) == snap.EMISMATCH
    img.array[3] ^= 1
    assert s.restore_status(img, used) == snap.EFORMAT
    img.array[3] ^= 1
    assert s.restore_status(img, used - 4096) == snap.EFORMAT
    assert s.restore_status(img, used) == snap.OK


def test_register_rejects_misaligned_pointer():
    t = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    s = snap.Set()
    with pytest.raises(snap.SnapError):
        s.register(t.data_ptr() + 4, 100)


def test_quiesce_timeout_then_recovers():
    """The lock waits for the caller's stream with a deadline (Sec. 3.1.1)."""
    st = torch.cuda.Stream()
    ts, hs = device_state([65536 * 4], seed=18)
    s = make_set(ts, 65536, stream=st, timeout_ms=100)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    with torch.cuda.stream(st):
        torch.cuda._sleep(int(2e9))  # about a second of queued work on the caller's stream
    rc, _ = s.checkpoint_status(img, snap.FULL)
    assert rc == snap.ETIMEDOUT
    with pytest.raises(snap.SnapError):
        s.committed_hashes(4)  # nothing was committed
    st.synchronize()
    used = s.checkpoint(img, snap.FULL)
    assert np.array_equal(img.view(used), oracle.write_full(hs, 65536, 0)[1])


def test_ring_consumer_stall_times_out_then_recovers(monkeypatch):
    """A ring consumer that stops draining, injected on the host
    (SNAP_FAULT=ring_stall: every copy-out task of a checkpoint waits until
    just past the call's deadline): the launcher's wait for a free slot runs
    out, the call returns SNAP_ETIMEDOUT soon after the deadline with nothing
    committed, and the next checkpoint, with the consumer draining again,
    equals the oracle's image (Sec. 3.1.1: a timeout rolls back)."""
    import time
    C = 65536
    sizes = [3 * 2**20 + 4096, 5 * 2**20, 12345]
    ts, hs = device_state(sizes, seed=61)
    s = make_set(ts, C, ring_bytes=2 << 20, timeout_ms=300)  # 8 slots of 256 KiB: 33 windows
    s.prepare(layout=True, ring=True)
    full = np.full(s.image_bytes(snap.FULL), 0xA5, dtype=np.uint8)  # pageable: through the ring
    monkeypatch.setenv("SNAP_FAULT", "ring_stall")
    t0 = time.perf_counter()
    rc, _ = s.checkpoint_status(full, snap.FULL)
    dt = time.perf_counter() - t0
    assert rc == snap.ETIMEDOUT and dt < 3.0
    nch = sum((n + C - 1) // C for n in sizes)
    with pytest.raises(snap.SnapError):
        s.committed_hashes(nch)  # nothing was committed
    monkeypatch.delenv("SNAP_FAULT")
    used = s.checkpoint(full, snap.FULL)
    assert np.array_equal(full[:used], oracle.write_full(hs, C, 0)[1])
    assert s.committed_hashes(nch)[1] == 0
    s.close()


def test_injected_allocation_failure_leaves_set_usable(monkeypatch):
    ts, hs = device_state([70000], seed=19)
    s = make_set(ts, 4096)
    monkeypatch.setenv("SNAP_FAULT", "hash_alloc")
    with pytest.raises(snap.SnapError) as e:
        s.image_bytes(snap.FULL)
    assert e.value.status == snap.ENOMEM
    monkeypatch.delenv("SNAP_FAULT")
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    used = s.checkpoint(img, snap.FULL)
    assert np.array_equal(img.view(used), oracle.write_full(hs, 4096, 0)[1])


def test_injected_graph_failure(monkeypatch):
    ts, hs = device_state([70000], seed=20)
    s = make_set(ts, 4096)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    monkeypatch.setenv("SNAP_FAULT", "graph")
    rc, _ = s.checkpoint_status(img, snap.FULL)
    assert rc == snap.ENOMEM
    monkeypatch.delenv("SNAP_FAULT")
    used = s.checkpoint(img, snap.FULL)
    assert np.array_equal(img.view(used), oracle.write_full(hs, 4096, 0)[1])


# ------------------------------------------------------------ config 2 size
def test_gpt2_state_full_parity():
    """GPT-2-small training state (593 allocations, 2,259,472,384 B): the
    batched persistent kernel's image equals the oracle's, byte for byte."""
    spec = workloads.gpt2_state_spec()
    sizes = workloads.spec_bytes(spec)
    ts = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
    workloads.torch_fill_spec(ts, spec, seed=2)
    s = make_set(ts, 65536)
    n = s.image_bytes(snap.FULL)
    img = snap.HostBuffer(n)
    used = s.checkpoint(img, snap.FULL)
    host = readback(ts)
    rc, exp = oracle.write_full(host, 65536, 0)
    assert rc == 0 and np.array_equal(img.view(used), exp)
    del exp
    for t in ts:
        t.zero_()
    s.restore(img, used)
    for a, b in zip(readback(ts), host):
        assert np.array_equal(a, b)


def test_link_ceiling_measures_both_directions():
    """The SM-path ceiling the gather and scatter are held to: positive in each
    direction and in both at once (whose combined rate is at least either
    direction's alone); bad arguments are rejected before anything is
    allocated."""
    d2h = snap.link_ceiling(0, 256 * MiB, 1)
    h2d = snap.link_ceiling(1, 256 * MiB, 1)
    both = snap.link_ceiling(2, 256 * MiB, 1)
    assert d2h > 1.0 and h2d > 1.0 and both > 0.9 * max(d2h, h2d)
    v = __import__("ctypes").c_double()
    assert snap.lib().snap_link_ceiling(-1, 3, 1 << 20, 1, v) == snap.EINVAL
    assert snap.lib().snap_link_ceiling(-1, 0, 4096, 1, v) == snap.EINVAL
    assert snap.lib().snap_link_ceiling(-1, 0, 1 << 20, 0, v) == snap.EINVAL


def _pipeline_state(seed):
    """About 630 MiB in 41 allocations of uneven sizes (zero bytes, a few
    bytes, ragged, one of 200 MiB): two hash launches of the pipelined
    incremental at 64 KiB chunks, nine at 16 KiB, where the 200 MiB
    allocation spans several launches and leaves one allocation group empty
    (with the default 24-warp hash shape on 140 SMs)."""
    rng = np.random.default_rng(seed)
    sizes = [int(x) for x in rng.integers(1, 24 * MiB, 36)] + [0, 17, 200 * MiB + 12345, 65536, 3]
    rng.shuffle(sizes)
    ts = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
    for k, t in enumerate(ts):
        if t.numel():
            workloads.torch_random_bytes(t, seed * 1000 + k)
    return sizes, ts


@pytest.mark.parametrize("form", ["fused", "fused16", "dma", "dma2", "stages"])
@pytest.mark.parametrize("C", [65536, 16384])
def test_pipelined_incremental_matches_oracle_and_the_serial_form(C, form, monkeypatch, tmp_path):
    """Large enough for several allocation groups: the pipelined patch (image
    capacity covers the largest patch) and the serial one (capacity one byte
    short of that bound) both equal the oracle's patch, byte for byte, at 0 %,
    a few, every other (alternating: no two dirty chunks adjacent) and 100 %
    dirty chunks.  Both pipelined forms: the fused one (one
    cooperative launch whose CTAs hash, lay out and gather group by group,
    the default), also with a 16-warp hash shape taken from the tuning cache
    (the general kernel instantiation, 512-thread CTAs) and with its dirty
    runs handed to the copy engines (SNAP_INCR_COPY_DMA: one copy per run of
    consecutive dirty chunks of an allocation; also dealt over two copy
    streams), and the launch-per-stage one (SNAP_FUSED_OFF)."""
    import math
    if form == "stages":
        monkeypatch.setenv("SNAP_FUSED_OFF", "1")
    if form == "dma2":
        monkeypatch.setenv("SNAP_DMA_STREAMS", "2")
    sizes, ts = _pipeline_state(31)
    if form == "fused16":
        cache = tmp_path / "tune.jsonl"
        cls = int(math.floor(math.log2(sum(sizes))))
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        cache.write_text('{"gpu": "%s", "op": 1, "chunk": %d, "class": %d, "warps": 16, "stages": 2, "piece": 64, '
                         '"chains": 1, "tma": 0, "ctas": %d, "gbs": 1.0}\n' % (torch.cuda.get_device_name(), C, cls, sms))
        monkeypatch.setenv("SNAP_TUNE_CACHE", str(cache))
    a = make_set(ts, C, incr_copy=snap.INCR_COPY_DMA if form.startswith("dma") else snap.INCR_COPY_SM)
    b = make_set(ts, C)
    if form == "fused16":
        assert a.tuning(snap.INCREMENTAL)["warps"] == 16
    full_a = snap.HostBuffer(a.image_bytes(snap.FULL))
    full_b = snap.HostBuffer(b.image_bytes(snap.FULL))
    bound = a.image_bytes(snap.INCREMENTAL)
    pa = snap.HostBuffer(bound)
    pb = snap.HostBuffer(bound)
    a.checkpoint(full_a, snap.FULL)
    b.checkpoint(full_b, snap.FULL)
    base = readback(ts)
    nch = [(n + C - 1) // C for n in sizes]
    rng = np.random.default_rng(32)
    dirty = set()
    for k, n in enumerate(nch):
        if n:
            dirty |= {(k, 0), (k, n - 1), (k, int(rng.integers(0, n)))}
    plans = [("none", set()), ("some", dirty),
             ("alternate", {(k, i) for k, n in enumerate(nch) for i in range(k % 2, n, 2)}),
             ("all", {(k, i) for k, n in enumerate(nch) for i in range(n)})]
    prev = [oracle.chunk_hashes(h, C) for h in base]
    gen = 1
    for name, chunks in plans:
        mutate(ts, C, sorted(chunks), seed=33 + gen)
        cur = readback(ts)
        used_a = a.checkpoint(pa, snap.INCREMENTAL)
        st_a = a.stats()
        used_b = b.checkpoint(pb, snap.INCREMENTAL, cap=bound - 1)
        st_b = b.stats()
        rc, exp, nd = oracle.write_patch(cur, C, prev, generation=gen, parent=gen - 1)
        assert rc == 0 and nd == len(chunks), name
        assert used_a == exp.size and np.array_equal(pa.view(used_a), exp), name
        assert used_b == exp.size and np.array_equal(pb.view(used_b), exp), name
        assert st_a["dirty_chunks"] == st_b["dirty_chunks"] == nd
        if form.startswith("dma"):  # the fused launch, then a stamp after the copies
            assert st_a["kernel_launches"] == 4
            assert (st_a["dma_copies"] > 0) == (nd > 0) and st_a["dma_copies"] <= nd
            if name == "all":  # one run per allocation with chunks
                assert st_a["dma_copies"] == sum(1 for n in nch if n)
            if name == "alternate":  # no two dirty chunks adjacent: a run per chunk
                assert st_a["dma_copies"] == nd
        elif form != "stages":  # one fused launch between the two phase stamps
            assert st_a["kernel_launches"] == 3 and st_a["dma_copies"] == 0
        else:  # the launch-per-stage sequence ran
            assert st_a["kernel_launches"] > st_b["kernel_launches"]
        prev = [oracle.chunk_hashes(h, C) for h in cur]
        gen += 1
    a.close()
    b.close()


@pytest.mark.parametrize("copy", ["sm", "dma"])
def test_fused_incremental_gives_up_and_the_set_recovers(copy, monkeypatch):
    """The fused incremental's device-side waits reach their error path
    without a fault: with the test hook SNAP_TEST_STALL_TILE one hash warp's
    bounded wait runs out; the metadata CTA waiting for that warp's group and
    the gather CTAs waiting for its metadata see the recorded error (or run
    out themselves) and leave (in the copy-engine form the host stops taking
    groups when the launch ends without publishing the next one); the call
    returns SNAP_ECUDA inside the call deadline with nothing committed, and
    the next incremental (fused again) equals the oracle's patch."""
    import time
    C = 65536
    sizes, ts = _pipeline_state(41)
    s = make_set(ts, C, incr_copy=snap.INCR_COPY_DMA if copy == "dma" else snap.INCR_COPY_SM)
    full = snap.HostBuffer(s.image_bytes(snap.FULL))
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    s.checkpoint(full, snap.FULL)
    prev = [oracle.chunk_hashes(h, C) for h in readback(ts)]
    nch = [(n + C - 1) // C for n in sizes]
    base, gen = s.committed_hashes(sum(nch))
    base = base.copy()
    mutate(ts, C, [(k, 0) for k, n in enumerate(nch) if n], seed=42)
    cur = readback(ts)
    monkeypatch.setenv("SNAP_TEST_STALL_TILE", "100")
    t0 = time.perf_counter()
    rc, _ = s.checkpoint_status(patch, snap.INCREMENTAL)
    dt = time.perf_counter() - t0
    assert rc == snap.ECUDA and s.stats()["device_errors"] & 1
    assert dt < 9.0  # the stalled warp's two bounded waits; the call deadline is 10 s
    h2, g2 = s.committed_hashes(sum(nch))
    assert g2 == gen and np.array_equal(h2, base)
    monkeypatch.delenv("SNAP_TEST_STALL_TILE")
    used = s.checkpoint(patch, snap.INCREMENTAL)
    launches = 4 if copy == "dma" else 3
    assert s.stats()["kernel_launches"] == launches and s.stats()["device_errors"] == 0  # the fused form, clean
    rc, exp, nd = oracle.write_patch(cur, C, prev, 1, 0)
    assert rc == 0 and used == exp.size and np.array_equal(patch.view(used), exp)
    s.close()


@pytest.mark.parametrize("copy", ["sm", "dma"])
def test_gpt2_state_pipelined_incremental_parity(copy):
    """GPT-2-small training state (2.26 GB, eight allocation groups): a 10 %
    clustered mutation; the pipelined patch equals the oracle's, and the
    previous full image plus the patch equals the full image of the state.
    Both ways of moving the dirty chunks: gather CTAs, and copy engines (one
    copy per run of consecutive dirty chunks, many of them single small
    tensors)."""
    spec = workloads.gpt2_state_spec()
    sizes = workloads.spec_bytes(spec)
    ts = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
    workloads.torch_fill_spec(ts, spec, seed=3)
    C = 65536
    s = make_set(ts, C, incr_copy=snap.INCR_COPY_DMA if copy == "dma" else snap.INCR_COPY_SM)
    full = snap.HostBuffer(s.image_bytes(snap.FULL))
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    used0 = s.checkpoint(full, snap.FULL)
    base = readback(ts)
    nch = [(n + C - 1) // C for n in sizes]
    c0 = np.concatenate([[0], np.cumsum(nch)])
    units = workloads.mutation_units(int(c0[-1]), 0.10, 4)
    chunks = [(int(np.searchsorted(c0, u, side="right") - 1), 0) for u in units]
    chunks = [(k, int(u - c0[k])) for (k, _), u in zip(chunks, units)]
    mutate(ts, C, chunks, seed=5)
    cur = readback(ts)
    used = s.checkpoint(patch, snap.INCREMENTAL)
    assert (s.stats()["dma_copies"] > 0) == (copy == "dma")
    rc, exp, nd = oracle.write_patch(cur, C, [oracle.chunk_hashes(h, C) for h in base], 1, 0)
    assert rc == 0 and nd == len(set(chunks))
    assert used == exp.size and np.array_equal(patch.view(used), exp)
    del exp
    merged = full.view(used0).copy()
    snap.apply_patch(merged, patch.view(used))
    assert np.array_equal(merged, oracle.write_full(cur, C, generation=1)[1])
    s.close()


def test_allocation_past_4_gib_offsets():
    """One allocation of 4 GiB + 12,345 B (chunk offsets past 2^32 bytes) next
    to a small one: image hashes and bytes of chunks around the 4 GiB mark and
    the ragged tail equal the oracle's, and restore brings them back."""
    C = 65536
    n_big = (4 << 30) + 12345
    big = torch.empty(n_big, dtype=torch.uint8, device="cuda")
    for p in range(0, n_big, 1 << 30):
        q = min(n_big, p + (1 << 30))
        workloads.torch_random_bytes(big[p:q], 200 + p // (1 << 30))
    small = torch.from_numpy(workloads.xorshift_bytes(100003, 9, 0)).cuda()
    s = make_set([small, big], C)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    used = s.checkpoint(img, snap.FULL)
    nb = (n_big + C - 1) // C
    picks = [0, 1, (1 << 32) // C - 1, (1 << 32) // C, (1 << 32) // C + 1, nb - 2, nb - 1]
    from struct import unpack_from
    rec1 = 64 + 32 + 4 * 2
    rec1 = (rec1 + 4095) // 4096 * 4096 + 100003
    rec1 = (rec1 + 4095) // 4096 * 4096  # record of the big allocation
    b, n, data_off, _ = unpack_from("<QQQQ", img.array, rec1)
    assert b == n_big and n == nb
    expect = {}
    for i in picks:
        lo, hi = i * C, min((i + 1) * C, n_big)
        chunk = big[lo:hi].cpu().numpy()
        expect[i] = chunk
        assert unpack_from("<I", img.array, rec1 + 32 + 4 * i)[0] == oracle.crc32c(chunk), i
        assert np.array_equal(img.array[data_off + lo: data_off + hi], chunk), i
    big.zero_()
    s.restore(img, used)
    for i in picks:
        lo, hi = i * C, min((i + 1) * C, n_big)
        assert np.array_equal(big[lo:hi].cpu().numpy(), expect[i]), i
    assert s.verify(img, used) == 0
    s.close()


def test_many_small_allocations_full_and_incremental():
    """5,000 allocations of 1 B - 20 KiB (most smaller than a chunk, many not a
    multiple of 16 B): full image and patch equal the oracle's, and restore
    into zeroed buffers reproduces every byte."""
    rng = np.random.default_rng(77)
    sizes = [int(x) for x in rng.integers(1, 20 * 1024, 5000)]
    # one arena, allocations at 16-byte aligned offsets (as a caching allocator gives)
    offs, o = [], 0
    for n in sizes:
        offs.append(o)
        o += (n + 15) // 16 * 16
    arena = torch.empty(o, dtype=torch.uint8, device="cuda")
    workloads.torch_random_bytes(arena, 78)
    ts = [arena[a: a + n] for a, n in zip(offs, sizes)]
    C = 4096
    s = make_set(ts, C)
    full = snap.HostBuffer(s.image_bytes(snap.FULL))
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    used = s.checkpoint(full, snap.FULL)
    base = readback(ts)
    assert np.array_equal(full.view(used), oracle.write_full(base, C, 0)[1])
    picks = sorted(set(int(k) for k in rng.integers(0, len(sizes), 300)))
    mutate(ts, C, [(k, 0) for k in picks], seed=79)
    cur = readback(ts)
    used_p = s.checkpoint(patch, snap.INCREMENTAL)
    rc, exp, nd = oracle.write_patch(cur, C, [oracle.chunk_hashes(h, C) for h in base], 1, 0)
    assert nd == len(picks) and np.array_equal(patch.view(used_p), exp)
    arena.zero_()
    s.restore(full, used)
    for a, b in zip(readback(ts), base):
        assert np.array_equal(a, b)
    s.close()


@pytest.mark.parametrize("C", [4096, 65536, 1 << 20])
def test_tma_hash_staging_parity(C):
    """The hash pass staged by 2D TMA tensor copies (tensor map per
    allocation, hardware swizzle) gives the oracle's hashes: full image,
    incremental patch and verify, with ragged allocations beside full ones."""
    sizes = SIZES_EDGE + [5 * C + 12345, 3 * C]
    ts, hs = device_state(sizes, seed=131)
    s = make_set(ts, C, hash_tma=True)
    full = snap.HostBuffer(s.image_bytes(snap.FULL))
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    used = s.checkpoint(full, snap.FULL)
    assert np.array_equal(full.view(used), oracle.write_full(hs, C, 0)[1])
    nch = [(x + C - 1) // C for x in sizes]
    dirty = [(k, n - 1) for k, n in enumerate(nch) if n] + [(len(sizes) - 2, 2)]
    mutate(ts, C, dirty, seed=132)
    cur = readback(ts)
    used_p = s.checkpoint(patch, snap.INCREMENTAL)
    rc, exp, nd = oracle.write_patch(cur, C, [oracle.chunk_hashes(h, C) for h in hs], 1, 0)
    assert nd == len(set(dirty)) and np.array_equal(patch.view(used_p), exp)
    assert s.verify(patch, used_p) == 0
    s.close()


def test_config3_20gib_full_parity():
    """The 20 GiB state of 2,000 allocations at full size, pipelined: the whole
    full image and the whole 1 % clustered patch equal the oracle's, byte for
    byte, on the device bytes read back with plain copies; the patch's dirty
    set equals the mutation set; the patch merged into the image equals the
    oracle's image of the mutated state; verify is clean."""
    C = 65536
    sizes = workloads.config3_sizes(1)
    need = sum(sizes)
    free_host = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    if free_host < 5 * need:
        pytest.skip("needs %d B of host memory" % (5 * need))
    align = 1 << 20
    starts, off = [], 0
    for n in sizes:
        starts.append(off)
        off += (n + align - 1) // align * align
    arena = torch.empty(off, dtype=torch.uint8, device="cuda")
    for p in range(0, off, 1 << 30):
        workloads.torch_random_bytes(arena[p: min(off, p + (1 << 30))], 300 + p // (1 << 30))
    ts = [arena[a: a + n] for a, n in zip(starts, sizes)]
    s = make_set(ts, C)
    full = snap.HostBuffer(s.image_bytes(snap.FULL))
    used = s.checkpoint(full, snap.FULL)
    host = readback(ts)
    rc, exp = oracle.write_full(host, C, 0)
    assert rc == 0 and used == exp.size
    assert np.array_equal(full.view(used), exp)
    del exp
    prev = [oracle.chunk_hashes(h, C) for h in host]
    del host
    # 1 % clustered mutation, pipelined incremental
    nch = [(n + C - 1) // C for n in sizes]
    c0 = np.concatenate([[0], np.cumsum(nch)])
    units = workloads.mutation_units(int(c0[-1]), 0.01, 302)
    ks = np.searchsorted(c0, units, side="right") - 1
    muts = [(int(k), int(u - c0[k])) for k, u in zip(ks, units)]
    mutate(ts, C, muts, seed=303)
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    used_p = s.checkpoint(patch, snap.INCREMENTAL)
    cur = readback(ts)
    rc, exp_p, nd = oracle.write_patch(cur, C, prev, 1, 0)
    assert rc == 0 and nd == len(units) == s.stats()["dirty_chunks"]
    assert used_p == exp_p.size and np.array_equal(patch.view(used_p), exp_p)
    by_alloc = {}
    for k, i in muts:
        by_alloc.setdefault(k, []).append(i)
    for k in range(len(sizes)):
        rc, idx = oracle.patch_dirty(exp_p, k)
        assert rc == 0 and idx.tolist() == sorted(by_alloc.get(k, [])), k
    del exp_p
    assert s.verify(patch, used_p) == 0
    merged = full.view(used).copy()
    snap.apply_patch(merged, patch.view(used_p))
    rc, exp = oracle.write_full(cur, C, 1)
    assert rc == 0 and np.array_equal(merged, exp)
    s.close()


def test_config4_llama7b_state_full_parity():
    """The Llama-7B-shaped state at full size (1,196 allocations,
    115,812,655,104 B) through the 4 GiB pinned ring into a pageable image,
    then restored into freshly allocated buffers (filled with a pattern
    first): the whole image equals the oracle's, compared window by window
    of records (about 2 GiB of state each) on the device bytes read back with
    plain copies; every restored allocation equals its bytes in the image;
    verify is clean."""
    import mmap
    from struct import unpack_from
    spec = workloads.llama7b_state_spec()
    sizes = workloads.spec_bytes(spec)
    need = sum(sizes)
    free_host = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    free_dev = torch.cuda.mem_get_info()[0]
    if free_host < need + (24 << 30) or free_dev < need + (8 << 30):
        pytest.skip("needs %d B of host and device memory" % need)
    C = 65536
    ts = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
    workloads.torch_fill_spec(ts, spec, seed=7)
    s = make_set(ts, C, ring_bytes=4 << 30)
    nimg = s.image_bytes(snap.FULL)
    m = mmap.mmap(-1, nimg, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS | getattr(mmap, "MAP_POPULATE", 0))
    img = np.frombuffer(m, dtype=np.uint8)
    used = s.checkpoint(img, snap.FULL)
    assert used == nimg == oracle.image_bytes(sizes, C)
    windows, k0 = [], 0
    while k0 < len(sizes):
        k1, acc = k0, 0
        while k1 < len(sizes) and (k1 == k0 or acc + sizes[k1] <= (2 << 30)):
            acc += sizes[k1]
            k1 += 1
        windows.append((k0, k1))
        k0 = k1
    end = 0
    for k0, k1 in windows:
        torch.cuda.synchronize()
        datas = [ts[k].cpu().numpy() for k in range(k0, k1)]
        rc, lo, win = oracle.write_full_window(sizes, datas, C, 0, k0, k1)
        assert rc == 0 and lo == end, (k0, k1)
        assert np.array_equal(img[lo: lo + win.size], win), (k0, k1)
        end = lo + win.size
    assert end == used
    s.close()
    del ts, datas
    torch.cuda.empty_cache()
    fresh = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
    for t in fresh:
        t.fill_(0xA5)  # whatever the allocator hands back, the restore must overwrite it
    s = make_set(fresh, C, ring_bytes=4 << 30)
    s.restore(img, used)
    torch.cuda.synchronize()
    for k, n in enumerate(sizes):
        rec = oracle.image_bytes(sizes[:k], C)  # record k's offset (the oracle's layout)
        d_off = unpack_from("<Q", m, rec + 16)[0]
        assert np.array_equal(fresh[k].cpu().numpy(), img[d_off: d_off + n]), k
    assert s.verify(img, used) == 0
    s.close()
    del img
    m.close()
