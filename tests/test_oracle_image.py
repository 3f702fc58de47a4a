"""Pins for the oracle's image writer, restore, verify and incremental patch.

The image layout is re-derived here from its written definition with
`struct` (not the oracle's own parser); hashes are checked with the SSE4.2
instruction; the invariants restore(checkpoint(x)) == x (Sec. 6,
deterministic restore) and apply_patch(prev_full, patch) == full(current)
(incremental checkpointing, Sec. 7) are checked end to end."""
import struct

import numpy as np
import pytest

import oracle
import workloads

PAGE = 4096


def up(x):
    return (x + PAGE - 1) // PAGE * PAGE


def layout(sizes, C):
    """(record offsets, data offsets, total) by the written layout rule."""
    off, recs, datas = 64, [], []
    for b in sizes:
        n = (b + C - 1) // C
        recs.append(off)
        d = up(off + 32 + 4 * n)
        datas.append(d)
        off = up(d + b)
    return recs, datas, off


def make(sizes, seed=1):
    return [workloads.xorshift_bytes(s, seed, k) for k, s in enumerate(sizes)]


SIZES = [65536, 4096 * 3 + 16, 1, 0, 200000, 65536 * 2, 12345]


@pytest.mark.parametrize("C", [4096, 65536])
def test_full_image_layout(C, hwcrc):
    datas = make(SIZES)
    rc, img = oracle.write_full(datas, C, generation=5)
    assert rc == 0
    recs, doffs, total = layout(SIZES, C)
    assert img.size == total == oracle.image_bytes(SIZES, C)
    raw = img.tobytes()
    magic, ver, flags, cb, n, tot, gen, par, hcrc, pad = struct.unpack_from("<8sIIQQQQQII", raw, 0)
    assert magic == b"SNAPIMG1" and ver == 1 and flags == 2 and cb == C
    assert n == len(SIZES) and tot == sum(SIZES) and gen == 5 and par == 0 and pad == 0
    assert hcrc == hwcrc.crc(raw[:56])
    covered = np.zeros(img.size, dtype=bool)
    covered[:64] = True
    for k, b in enumerate(SIZES):
        bk, nk, dk, res = struct.unpack_from("<QQQQ", raw, recs[k])
        assert (bk, nk, dk, res) == (b, (b + C - 1) // C, doffs[k], 0)
        h = np.frombuffer(raw, dtype="<u4", count=nk, offset=recs[k] + 32)
        assert np.array_equal(h, hwcrc.chunks(datas[k], C))
        assert raw[dk: dk + b] == datas[k].tobytes()
        covered[recs[k]: recs[k] + 32 + 4 * nk] = True
        covered[dk: dk + b] = True
    # everything else is zero padding
    assert not img[~covered].any()


@pytest.mark.parametrize("C", [4096, 65536])
def test_full_image_windows(C):
    """The record-window writer used for states too large to image whole:
    each window starts at the written layout's offset of its first record
    (0 when it holds the header), reads only its own allocations, and the
    windows of any split put end to end are the whole image."""
    datas = make(SIZES, seed=3)
    whole = oracle.write_full(datas, C, generation=4)[1]
    recs, _, total = layout(SIZES, C)
    n = len(SIZES)
    for cuts in ([0, n], [0, 1, n], [0, 2, 3, 5, n], list(range(n + 1)), [0, 4, 4, n]):
        parts = []
        for k0, k1 in zip(cuts, cuts[1:]):
            rc, lo, w = oracle.write_full_window(SIZES, datas[k0:k1], C, 4, k0, k1)
            assert rc == 0
            assert lo == (0 if k0 == 0 else recs[k0] if k0 < n else total)
            assert lo + w.size == (recs[k1] if k1 < n else total)
            parts.append(w)
        assert np.array_equal(np.concatenate(parts), whole)
    rc, lo, w = oracle.write_full_window(SIZES, [], C, 4, 0, 0)  # the header alone
    assert rc == 0 and lo == 0 and np.array_equal(w, whole[:64])


def test_image_bytes_closed_form():
    for C in (4096, 16384, 65536, 1 << 20):
        sizes = workloads.config1_sizes(3)
        assert oracle.image_bytes(sizes, C) == layout(sizes, C)[2]


def test_restore_roundtrip():
    datas = make(SIZES, seed=2)
    rc, img = oracle.write_full(datas, 65536)
    rc2, outs = oracle.restore(img, SIZES)
    assert rc == 0 and rc2 == 0
    for a, b in zip(datas, outs):
        assert np.array_equal(a, b)


def test_verify_detects_changes():
    datas = make(SIZES, seed=3)
    rc, img = oracle.write_full(datas, 4096)
    assert oracle.verify(img, datas) == (0, 0)
    bad = [d.copy() for d in datas]
    bad[4][100000] ^= 0x40
    bad[0][0] ^= 1
    assert oracle.verify(img, bad) == (0, 2)


def test_restore_rejects_bad_images():
    datas = make(SIZES, seed=4)
    _, img = oracle.write_full(datas, 65536)
    b = img.copy(); b[0] ^= 1
    assert oracle.restore(b, SIZES)[0] == oracle.EFORMAT            # magic
    b = img.copy(); b[40] ^= 1
    assert oracle.restore(b, SIZES)[0] == oracle.EFORMAT            # header CRC
    assert oracle.restore(img[:-1], SIZES)[0] == oracle.EFORMAT     # truncated
    assert oracle.restore(img[:63], SIZES)[0] == oracle.EFORMAT
    assert oracle.restore(img, SIZES[:-1])[0] == oracle.EMISMATCH   # count
    s2 = list(SIZES); s2[2] += 1
    assert oracle.restore(img, s2)[0] == oracle.EMISMATCH           # size
    b = img.copy(); b[64 + 16] ^= 8                                 # record data offset
    assert oracle.restore(b, SIZES)[0] == oracle.EFORMAT


def mutate(datas, C, chunks, seed=9):
    """XOR every byte of the given (alloc, chunk) pairs with a nonzero byte."""
    out = [d.copy() for d in datas]
    rng = np.random.default_rng(seed)
    for k, i in chunks:
        lo, hi = i * C, min((i + 1) * C, out[k].size)
        out[k][lo:hi] ^= rng.integers(1, 256, hi - lo, dtype=np.uint8)
    return out


@pytest.mark.parametrize("C", [4096, 65536])
def test_patch_apply_equals_full(C):
    datas = make(SIZES, seed=5)
    rc, full0 = oracle.write_full(datas, C, generation=0)
    prev = [oracle.chunk_hashes(d, C) for d in datas]
    nch = [(s + C - 1) // C for s in SIZES]
    dirty = [(0, 0), (2, 0), (4, nch[4] - 1), (5, 1), (6, 0), (4, 1)]
    cur = mutate(datas, C, dirty)
    rc, patch, nd = oracle.write_patch(cur, C, prev, generation=1, parent=0)
    assert rc == 0 and nd == len(set(dirty))
    for k in range(len(SIZES)):
        exp = sorted(i for kk, i in set(dirty) if kk == k)
        rc, idx = oracle.patch_dirty(patch, k)
        assert rc == 0 and list(idx) == exp
    rc, applied = oracle.apply_patch(full0, patch)
    assert rc == 0
    rc, full1 = oracle.write_full(cur, C, generation=1)
    assert np.array_equal(applied, full1)


def test_patch_layout_by_struct(hwcrc):
    C = 4096
    datas = make(SIZES, seed=6)
    prev = [oracle.chunk_hashes(d, C) for d in datas]
    dirty = [(0, 3), (0, 7), (4, 48), (6, 3)]       # (6, 3) is a partial last chunk
    cur = mutate(datas, C, dirty)
    rc, patch, nd = oracle.write_patch(cur, C, prev, generation=7, parent=6)
    raw = patch.tobytes()
    magic, ver, flags, cb, n, tot, gen, par, hcrc, pad = struct.unpack_from("<8sIIQQQQQII", raw, 0)
    assert flags == 3 and gen == 7 and par == 6 and hcrc == hwcrc.crc(raw[:56])
    off = 64
    for k, b in enumerate(SIZES):
        nk = (b + C - 1) // C
        bk, nk2, dk, res = struct.unpack_from("<QQQQ", raw, off)
        assert (bk, nk2, res) == (b, nk, 0)
        h = np.frombuffer(raw, dtype="<u4", count=nk, offset=off + 32)
        assert np.array_equal(h, hwcrc.chunks(cur[k], C))
        (ndk,) = struct.unpack_from("<I", raw, off + 32 + 4 * nk)
        idx = list(np.frombuffer(raw, dtype="<u4", count=ndk, offset=off + 36 + 4 * nk))
        assert idx == sorted(i for kk, i in dirty if kk == k)
        assert dk == up(off + 36 + 4 * nk + 4 * ndk)
        d = dk
        for i in idx:
            lo, hi = i * C, min((i + 1) * C, b)
            assert raw[d: d + hi - lo] == cur[k][lo:hi].tobytes()
            assert not any(raw[d + hi - lo: up(d + hi - lo)])
            d = up(d + hi - lo)
        off = d
    assert off == patch.size


def test_patch_zero_and_full_dirty():
    C = 4096
    datas = make(SIZES, seed=7)
    prev = [oracle.chunk_hashes(d, C) for d in datas]
    rc, p0, nd0 = oracle.write_patch(datas, C, prev, 1, 0)
    assert rc == 0 and nd0 == 0
    # zero dirty: record headers, hashes and empty lists only
    off = 64
    for s in SIZES:
        off = up(off + 32 + 4 * ((s + C - 1) // C) + 4)
    assert p0.size == off
    everything = [(k, i) for k, s in enumerate(SIZES) for i in range((s + C - 1) // C)]
    cur = mutate(datas, C, everything)
    rc, pall, nd = oracle.write_patch(cur, C, prev, 1, 0)
    assert nd == len(everything)
    rc, f0 = oracle.write_full(datas, C, 0)
    rc, app = oracle.apply_patch(f0, pall)
    rc, f1 = oracle.write_full(cur, C, 1)
    assert np.array_equal(app, f1)


def test_apply_patch_checks_generation_and_shape():
    C = 4096
    datas = make(SIZES, seed=8)
    _, f0 = oracle.write_full(datas, C, 3)
    prev = [oracle.chunk_hashes(d, C) for d in datas]
    _, p, _ = oracle.write_patch(mutate(datas, C, [(0, 1)]), C, prev, 5, 4)
    assert oracle.apply_patch(f0, p)[0] == oracle.EMISMATCH       # parent 4 != base 3
    _, p, _ = oracle.write_patch(mutate(datas, C, [(0, 1)]), C, prev, 4, 3)
    rc, app = oracle.apply_patch(f0, p)
    assert rc == 0
    assert oracle.read_header(app)[1]["generation"] == 4
    assert oracle.apply_patch(f0, f0)[0] == oracle.EFORMAT        # not a patch
    assert oracle.apply_patch(p, p)[0] == oracle.EFORMAT          # base is a patch
    other = make(SIZES[:-1], seed=8)
    _, f_other = oracle.write_full(other, C, 3)
    assert oracle.apply_patch(f_other, p)[0] == oracle.EMISMATCH  # count differs
    assert oracle.apply_patch(f0, p[:-4096])[0] == oracle.EFORMAT # truncated patch
