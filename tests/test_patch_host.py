"""The library's host-side patch merge (snap_apply_patch) on the CPU.

snap_apply_patch runs on the host only, so it is checked here without a
GPU: on images the oracle writes, merging a patch into its base must give
the oracle's full image of the new state byte for byte (the invariant
apply_patch(full(prev), patch) == full(current) of the incremental scheme),
and every malformed or mismatched input must be refused with the base left
exactly as it was (Sec. 3.1: a failed operation rolls back).  That includes
headers whose CRC is valid but whose allocation count no image could hold,
which must give EFORMAT rather than an attempt to size tables by it."""
import struct

import numpy as np
import pytest

import oracle
import paper_2502_16631_b300 as snap

MiB = 1 << 20


def upg(x):
    return (x + 4095) // 4096 * 4096


def state(sizes, rng):
    return [rng.integers(0, 256, n, dtype=np.uint8) for n in sizes]


def mutated(datas, C, rng, frac):
    out = [d.copy() for d in datas]
    for d in out:
        for i in range((d.size + C - 1) // C):
            if rng.random() < frac:
                lo, hi = i * C, min((i + 1) * C, d.size)
                d[lo:hi] ^= rng.integers(1, 256, hi - lo, dtype=np.uint8)
    return out


def hashes(datas, C):
    return [oracle.chunk_hashes(d, C) for d in datas]


def images(sizes, C, seed, frac=0.3, gen=4):
    rng = np.random.default_rng(seed)
    d0 = state(sizes, rng)
    d1 = mutated(d0, C, rng, frac)
    rc, base = oracle.write_full(d0, C, generation=gen)
    assert rc == 0
    rc, patch, nd = oracle.write_patch(d1, C, hashes(d0, C), gen + 1, gen)
    assert rc == 0
    return d0, d1, base, patch, nd


def set_header(img, **fields):
    """Rewrite header fields of an image and re-seal its header CRC."""
    keys = ("flags", "chunk_bytes", "n_allocs", "total", "generation", "parent")
    img = img.copy()
    hdr = list(struct.unpack_from("<IIQQQQQ", img, 8))
    vals = dict(zip(keys, hdr[1:]))
    vals.update(fields)
    struct.pack_into("<IIQQQQQ", img, 8, hdr[0], *[vals[k] for k in keys])
    struct.pack_into("<I", img, 56, oracle.crc32c(img[:56]))
    return img


def patch_records(patch):
    """(offset of the index list, n_dirty, n_chunks) of each patch record."""
    n_allocs, C = struct.unpack_from("<Q", patch, 24)[0], struct.unpack_from("<Q", patch, 16)[0]
    off, out = 64, []
    for _ in range(n_allocs):
        nbytes, n, data_off, _ = struct.unpack_from("<4Q", patch, off)
        nd = struct.unpack_from("<I", patch, off + 32 + 4 * n)[0]
        idx_off = off + 36 + 4 * n
        out.append((idx_off, nd, n))
        idx = np.frombuffer(patch[idx_off: idx_off + 4 * nd].tobytes(), dtype=np.uint32)
        off = data_off + sum(upg(min(C, nbytes - int(i) * C)) for i in idx)
    return out


SIZES = [3 * 4096 + 100, 0, 1, 65536, 200000, 17, 65536 * 2 + 4096, 5 * 4096]


@pytest.mark.parametrize("C", [4096, 65536])
@pytest.mark.parametrize("frac", [0.0, 0.3, 1.0])
def test_apply_patch_matches_oracle(C, frac):
    for seed in range(3):
        _, d1, base, patch, nd = images(SIZES, C, seed=seed * 10 + int(frac * 10), frac=frac)
        merged = base.copy()
        assert snap.apply_patch_status(merged, patch) == snap.OK
        rc, exp = oracle.write_full(d1, C, generation=5)
        assert np.array_equal(merged, exp)
        rc, also = oracle.apply_patch(base.copy(), patch)
        assert rc == 0 and np.array_equal(merged, also)


def test_apply_patch_empty_and_zero_byte_states():
    for sizes in ([], [0], [0, 0, 4096 * 2 + 5, 0]):
        _, d1, base, patch, _ = images(sizes, 4096, seed=3, frac=0.5)
        merged = base.copy()
        assert snap.apply_patch_status(merged, patch) == snap.OK
        assert np.array_equal(merged, oracle.write_full(d1, 4096, generation=5)[1])


def test_apply_patch_refuses_bad_inputs_and_keeps_the_base():
    C = 4096
    _, _, base, patch, nd = images(SIZES, C, seed=77, frac=0.5)
    assert nd >= 4
    recs = patch_records(patch)
    k = next(j for j, (_, d, _) in enumerate(recs) if d >= 2)
    idx_off, _, n = recs[k]

    unsorted = patch.copy()
    a, b = struct.unpack_from("<II", unsorted, idx_off)
    struct.pack_into("<II", unsorted, idx_off, b, a)
    past_end = patch.copy()
    struct.pack_into("<I", past_end, idx_off, n)
    too_many = patch.copy()
    struct.pack_into("<I", too_many, idx_off - 4, n + 1)
    bad_crc = patch.copy()
    bad_crc[56] ^= 1
    huge = 1 << 40
    cases = [
        ("truncated", base, patch[:-1], snap.EFORMAT),
        ("truncated to the header", base, patch[:64], snap.EFORMAT),
        ("wrong parent", base, set_header(patch, parent=9), snap.EMISMATCH),
        ("base is a patch", set_header(base, flags=3), patch, snap.EFORMAT),
        ("patch is a full image", base, set_header(patch, flags=2), snap.EFORMAT),
        ("chunk size differs", base, set_header(patch, chunk_bytes=8192), snap.EMISMATCH),
        ("state size differs", base, set_header(patch, total=1), snap.EMISMATCH),
        ("indices not ascending", base, unsorted, snap.EFORMAT),
        ("index past the last chunk", base, past_end, snap.EFORMAT),
        ("more dirty chunks than chunks", base, too_many, snap.EFORMAT),
        ("header CRC", base, bad_crc, snap.EFORMAT),
        ("allocation count no image can hold", set_header(base, n_allocs=huge), set_header(patch, n_allocs=huge),
         snap.EFORMAT),
        ("allocation count one past the records", set_header(base, n_allocs=len(SIZES) + 1),
         set_header(patch, n_allocs=len(SIZES) + 1), snap.EFORMAT),
    ]
    for name, b_img, p_img, want in cases:
        target = b_img.copy()
        assert snap.apply_patch_status(target, p_img) == want, name
        assert np.array_equal(target, b_img), name
    # and the untouched inputs still merge
    merged = base.copy()
    assert snap.apply_patch_status(merged, patch) == snap.OK


def test_binding_refuses_buffers_the_library_would_overrun():
    """The binding passes one (address, byte count) range per buffer, so it
    refuses a view that is not one contiguous range, a count beyond the
    buffer and, for a buffer the library writes, a read-only array -- before
    any library call."""
    C = 4096
    _, _, base, patch, _ = images(SIZES, C, seed=5)
    for bad_base in (base[::-1], np.lib.stride_tricks.as_strided(base, (base.size // 2,), (2,))):
        with pytest.raises(ValueError):
            snap.apply_patch(bad_base, patch)
    frozen = base.copy()
    frozen.flags.writeable = False
    with pytest.raises(ValueError):
        snap.apply_patch(frozen, patch)
    with pytest.raises(ValueError):
        snap.apply_patch(base.copy(), patch, base_bytes=base.size + 1)
    with pytest.raises(ValueError):
        snap.apply_patch(base.copy(), patch, patch_bytes=patch.size + 4096)
    ro_patch = patch.copy()
    ro_patch.flags.writeable = False  # a patch is only read
    merged = base.copy()
    snap.apply_patch(merged, ro_patch)
    assert np.array_equal(merged, oracle.write_full(images(SIZES, C, seed=5)[1], C, generation=5)[1])


def test_span_of_tensors_and_raw_addresses():
    torch = pytest.importorskip("torch")
    t = torch.zeros(64, 64, dtype=torch.uint8)
    assert snap._span(t) == (t.data_ptr(), 4096)
    assert snap._span(t[8:16]) == (t[8:16].data_ptr(), 512)
    with pytest.raises(ValueError):
        snap._span(t.t())
    with pytest.raises(ValueError):
        snap._span(t[:, :8])
    with pytest.raises(ValueError):
        snap._span(t, 4097)
    assert snap._span(12345, 7) == (12345, 7)
    with pytest.raises(TypeError):
        snap._span(12345)
