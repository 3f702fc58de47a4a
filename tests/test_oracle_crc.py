"""Pins for the oracle's CRC-32C (table-driven, byte at a time).

Each pin is independent of the oracle's table: published values (the check
value and RFC 3720 Appendix B.4), a bit-at-a-time register, GF(2) polynomial
division on Python integers in the non-reflected convention, and the x86
SSE4.2 crc32 instruction."""
import numpy as np
import pytest
from hypothesis import given, settings, strategies as st

import oracle
from conftest import load_golden_vectors

POLY_NORMAL = 0x1EDC6F41          # x^32 + 0x1EDC6F41 (Castagnoli), normal form
POLY_REFLECTED = 0x82F63B78


def crc_bitwise(data: bytes) -> int:
    """One bit at a time through a reflected shift register (no table)."""
    c = 0xFFFFFFFF
    for b in data:
        for i in range(8):
            bit = ((c ^ (b >> i)) & 1)
            c >>= 1
            if bit:
                c ^= POLY_REFLECTED
    return c ^ 0xFFFFFFFF


def _reverse32(v: int) -> int:
    return int("{:032b}".format(v)[::-1], 2)


def crc_polydiv(data: bytes) -> int:
    """The definition as polynomial arithmetic over GF(2): with the message
    bits M(x) in transmission order (least significant bit of each byte
    first), the register after n bytes is I(x) x^(8n) + M(x) x^32 mod P(x),
    I = all ones; the reflected output is that remainder bit-reversed, then
    complemented."""
    n = len(data)
    m = 0
    for b in data:
        for i in range(8):
            m = (m << 1) | ((b >> i) & 1)
    a = (0xFFFFFFFF << (8 * n)) ^ (m << 32)
    p = (1 << 32) | POLY_NORMAL
    while a.bit_length() > 32:
        a ^= p << (a.bit_length() - 33)
    return _reverse32(a) ^ 0xFFFFFFFF


@pytest.mark.parametrize("name,data,expected", load_golden_vectors())
def test_published_vectors(name, data, expected, hwcrc):
    assert oracle.crc32c(data) == expected, name
    # the independent implementations agree with the published value too
    assert hwcrc.crc(data) == expected, name
    assert crc_bitwise(data) == expected, name
    assert crc_polydiv(data) == expected, name


def test_check_value():
    assert oracle.crc32c(b"123456789") == 0xE3069283


def test_empty_message():
    # zero bytes: init then final complement cancel
    assert oracle.crc32c(b"") == 0


def test_bitwise_all_short_lengths():
    rng = np.random.default_rng(7)
    buf = rng.integers(0, 256, 600, dtype=np.uint8).tobytes()
    for n in range(0, 600):
        assert oracle.crc32c(buf[:n]) == crc_bitwise(buf[:n]), n


def test_bitwise_long_lengths():
    rng = np.random.default_rng(8)
    for n in list(rng.integers(600, 2049, 12)) + [2048]:
        d = rng.integers(0, 256, int(n), dtype=np.uint8).tobytes()
        assert oracle.crc32c(d) == crc_bitwise(d)


def test_polydiv_lengths():
    rng = np.random.default_rng(9)
    for n in list(range(0, 70)) + [255, 256, 257, 1023, 1024]:
        d = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        assert oracle.crc32c(d) == crc_polydiv(d), n


def test_sse42_many_lengths(hwcrc):
    rng = np.random.default_rng(10)
    big = rng.integers(0, 256, 3 << 20, dtype=np.uint8)
    for n in list(range(0, 300)) + list(rng.integers(300, 3 << 20, 40)) + [65536, 65535, 65537, 3 << 20]:
        d = big[: int(n)]
        assert oracle.crc32c(d) == hwcrc.crc(d), n


def test_sse42_odd_offsets(hwcrc):
    rng = np.random.default_rng(11)
    big = rng.integers(0, 256, 1 << 18, dtype=np.uint8)
    for off in range(0, 33):
        for n in (1, 15, 16, 17, 4095, 65536 - off):
            d = big[off: off + n]
            assert oracle.crc32c(d) == hwcrc.crc(d)


def _shift_zeros(c: int, nbytes: int) -> int:
    """Raw register after feeding nbytes zero bytes, bit at a time."""
    for _ in range(8 * nbytes):
        c = (c >> 1) ^ (POLY_REFLECTED if c & 1 else 0)
    return c


@settings(max_examples=60, deadline=None)
@given(st.binary(max_size=300), st.binary(max_size=300))
def test_linearity_combine(a, b):
    """crc(A||B) = shift(crc_state(A), |B|) xor raw(B): the identity the
    GPU path's per-lane combine relies on, checked on the oracle."""
    sa = oracle.crc32c_update(0xFFFFFFFF, a)
    rb = oracle.crc32c_update(0, b)
    assert oracle.crc32c_update(0xFFFFFFFF, a + b) == _shift_zeros(sa, len(b)) ^ rb
    # the zero-shift identity: raw update over zeros equals the bit shift
    assert oracle.crc32c_update(sa, bytes(len(b))) == _shift_zeros(sa, len(b))


def test_single_bit_errors_detected():
    rng = np.random.default_rng(12)
    d = bytearray(rng.integers(0, 256, 4096, dtype=np.uint8).tobytes())
    base = oracle.crc32c(bytes(d))
    for pos in rng.integers(0, 4096 * 8, 200):
        d[pos // 8] ^= 1 << (pos % 8)
        assert oracle.crc32c(bytes(d)) != base
        d[pos // 8] ^= 1 << (pos % 8)


@pytest.mark.parametrize("C", [4096, 16384, 65536, 1 << 20])
def test_chunk_hashes_vs_hw(C, hwcrc):
    rng = np.random.default_rng(13)
    for nbytes in (0, 1, 17, C - 1, C, C + 1, 3 * C + 4097, 5 * C):
        d = rng.integers(0, 256, nbytes, dtype=np.uint8)
        h = oracle.chunk_hashes(d, C)
        assert h.size == (nbytes + C - 1) // C
        assert np.array_equal(h, hwcrc.chunks(d, C))


def test_threads_do_not_change_hashes(hwcrc):
    rng = np.random.default_rng(14)
    d = rng.integers(0, 256, 40 * 65536 + 123, dtype=np.uint8)
    ref = hwcrc.chunks(d, 65536)
    for t in (1, 3, 8):
        oracle.set_threads(t)
        assert np.array_equal(oracle.chunk_hashes(d, 65536), ref)
    oracle.set_threads(1)
