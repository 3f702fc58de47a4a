"""The seeded workload recipes: shapes, totals and determinism."""
import numpy as np

import workloads as w


def test_config1_sizes():
    s = w.config1_sizes(1)
    assert len(s) == 16 and sum(s) == 64 << 20
    assert all(x % 4096 == 0 and x > 0 for x in s)
    assert s == w.config1_sizes(1) and s != w.config1_sizes(2)


def test_config3_sizes():
    s = w.config3_sizes(1)
    assert len(s) == 2000 and sum(s) == 20 << 30
    assert all(x % 4096 == 0 for x in s)


def test_config5_tenants():
    t = w.config5_tenants(1)
    assert len(t) == 32
    for s in t:
        assert 8 <= len(s) <= 64 and sum(s) <= 4 << 30 and all(x % 4096 == 0 for x in s)


def test_model_shapes():
    assert sum(n for _, n in w.gpt2_small_tensors()) == 124_439_808
    assert len(w.gpt2_small_tensors()) == 148
    assert sum(n for _, n in w.llama7b_tensors()) == 6_738_415_616
    assert len(w.llama7b_tensors()) == 291
    g = w.gpt2_state_spec()
    assert len(g) == 593 and sum(w.spec_bytes(g)) == 2_259_472_384
    ll = w.llama7b_state_spec()
    assert len(ll) == 291 * 4 + 32 and sum(w.spec_bytes(ll)) == 115_812_655_104


def test_xorshift_stream_deterministic():
    a = w.xorshift_bytes(1000, 1, 3)
    assert np.array_equal(a, w.xorshift_bytes(1000, 1, 3))
    assert not np.array_equal(a, w.xorshift_bytes(1000, 1, 4))
    # the byte stream is the 64-bit outputs in little-endian order
    r = w.Rng(0)
    r.x = w.splitmix64(1 ^ 3)
    first = r.next_u64()
    assert int.from_bytes(a[:8].tobytes(), "little") == first


def test_mutation_units():
    u = w.mutation_units(10000, 0.1, 1)
    assert len(u) == 1000 and np.all(np.diff(u) > 0) and u[-1] < 10000
    assert np.array_equal(u, w.mutation_units(10000, 0.1, 1))
    # clustered: far fewer runs than units
    runs = 1 + np.count_nonzero(np.diff(u) > 1)
    assert runs < 200
    assert len(w.mutation_units(5000, 0.0, 1)) == 0
    assert len(w.mutation_units(5000, 1.0, 1)) == 5000
