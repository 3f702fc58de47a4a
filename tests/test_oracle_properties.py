"""Property tests of the oracle's invariants on random allocation sets
(hypothesis): restore(full(x)) == x, apply_patch(full(a), patch(b vs a)) ==
full(b), the patch's dirty set is exactly the changed chunks, and verify
counts exactly the changed chunks.  Sizes straddle chunk boundaries, include
empty allocations and ragged tails."""
import numpy as np
from hypothesis import given, settings, strategies as st, HealthCheck

import oracle

SIZES = st.lists(st.one_of(st.integers(0, 40), st.integers(4000, 4200), st.integers(8180, 8200),
                           st.integers(0, 3 * 4096 + 17)), min_size=1, max_size=7)


def _arrays(sizes, seed):
    rng = np.random.default_rng(seed)
    return [rng.integers(0, 256, n, dtype=np.uint8) for n in sizes]


@settings(max_examples=40, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(sizes=SIZES, seed=st.integers(0, 2**31), chunk=st.sampled_from([4096, 8192]))
def test_full_image_roundtrip(sizes, seed, chunk):
    data = _arrays(sizes, seed)
    rc, img = oracle.write_full(data, chunk, 3)
    assert rc == 0 and img.size == oracle.image_bytes(sizes, chunk)
    rc, hdr = oracle.read_header(img)
    assert rc == 0 and hdr["generation"] == 3 and hdr["n_allocs"] == len(sizes)
    rc, back = oracle.restore(img, sizes)
    assert rc == 0
    for a, b in zip(back, data):
        assert np.array_equal(a, b)


@settings(max_examples=40, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(sizes=SIZES, seed=st.integers(0, 2**31), chunk=st.sampled_from([4096, 8192]),
       flips=st.lists(st.tuples(st.integers(0, 6), st.integers(0, 20000)), max_size=12))
def test_patch_is_exactly_the_changed_chunks(sizes, seed, chunk, flips):
    a = _arrays(sizes, seed)
    b = [x.copy() for x in a]
    for k, pos in flips:
        if k < len(b) and b[k].size:
            b[k][pos % b[k].size] ^= 0x5A
    # a byte flipped twice is back: the changed chunks are those that differ
    changed = {(k, i) for k in range(len(a)) for i in range(oracle.n_chunks(a[k].size, chunk))
               if not np.array_equal(a[k][i * chunk:(i + 1) * chunk], b[k][i * chunk:(i + 1) * chunk])}
    rc, full_a = oracle.write_full(a, chunk, 0)
    rc, patch, nd = oracle.write_patch(b, chunk, [oracle.chunk_hashes(x, chunk) for x in a], 1, 0)
    assert rc == 0 and nd == len(changed)
    for k in range(len(b)):
        rc, idx = oracle.patch_dirty(patch, k)
        assert rc == 0
        assert sorted(int(i) for i in idx) == sorted(i for kk, i in changed if kk == k)
    rc, merged = oracle.apply_patch(full_a, patch)
    assert rc == 0
    rc, full_b = oracle.write_full(b, chunk, 1)
    assert np.array_equal(merged, full_b)
    rc, bad = oracle.verify(full_a, b)
    assert rc == 0 and bad == len(changed)
