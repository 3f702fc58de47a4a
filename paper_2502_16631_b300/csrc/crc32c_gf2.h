// CRC-32C (Castagnoli) arithmetic for the GPU path and its host runtime.
//
// Representation: a CRC register value v stands for the polynomial
// V(x) = sum_i bit_i(v) * x^(31-i) over GF(2) (the reflected, LSB-first
// convention of CRC-32C), so the polynomial "1" is 0x80000000 and the
// Castagnoli modulus P(x) = x^32 + 0x1EDC6F41 appears as 0x82F63B78.
//
// Facts used by the kernels (linearity of the CRC over GF(2)):
//   update(v, M)           = v * x^(8|M|) + update(0, M)        (mod P)
//   update(v, 0^n)         = v * x^(8n)                          (mod P)
// so a chunk split into lane pieces S_0..S_m has
//   update(~0, chunk) = sum_l  update(init_l, S_l) * x^(8 * bytes after S_l)
// with init = ~0 for the first piece and 0 otherwise.  "Shift by n bytes" is
// multiplication by the constant x^(8n) mod P: a fixed GF(2) 32x32 matrix.
//
// All tables are generated at compile time from the polynomial.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define SNAP_HD __host__ __device__ __forceinline__
#else
#define SNAP_HD inline
#endif

namespace snapk {

constexpr uint32_t kPolyReflected = 0x82F63B78u;  // Castagnoli, reflected
constexpr uint32_t kOnePoly = 0x80000000u;        // the polynomial 1

// v * x mod P
SNAP_HD constexpr uint32_t gf2_mul_x(uint32_t v)
{
    return (v >> 1) ^ ((v & 1u) ? kPolyReflected : 0u);
}

// a * b mod P: shift-and-add over the terms of a, lowest degree first.
SNAP_HD constexpr uint32_t gf2_mulmod(uint32_t a, uint32_t b)
{
    uint32_t r = 0;
    for (int j = 0; j < 32; ++j) {
        r ^= (a & (kOnePoly >> j)) ? b : 0u;
        b = gf2_mul_x(b);
    }
    return r;
}

// Table of x^(8 * 2^i) mod P, i = 0..47 (byte shifts by powers of two).
struct Pow8Table {
    uint32_t v[48];
};

constexpr Pow8Table make_pow8_table()
{
    Pow8Table t{};
    uint32_t x8 = kOnePoly;
    for (int i = 0; i < 8; ++i) x8 = gf2_mul_x(x8);
    t.v[0] = x8;
    for (int i = 1; i < 48; ++i) t.v[i] = gf2_mulmod(t.v[i - 1], t.v[i - 1]);
    return t;
}

// x^(8n) mod P, from the power-of-two table.
SNAP_HD constexpr uint32_t gf2_x8n(uint64_t n, const Pow8Table &t)
{
    uint32_t r = kOnePoly;
    for (int i = 0; n; ++i, n >>= 1)
        if (n & 1u) r = gf2_mulmod(r, t.v[i]);
    return r;
}

// Slicing-by-4 tables: t[0][b] is the register after feeding byte b into a
// zero register (b's bits times x^8, reduced), and t[k][b] is t[k-1][b]
// fed with one more zero byte.
struct SliceTables {
    uint32_t t[4][256];
};

constexpr SliceTables make_slice_tables()
{
    SliceTables s{};
    for (uint32_t b = 0; b < 256; ++b) {
        uint32_t r = b;
        for (int k = 0; k < 8; ++k) r = gf2_mul_x(r);
        s.t[0][b] = r;
    }
    for (int k = 1; k < 4; ++k)
        for (uint32_t b = 0; b < 256; ++b) {
            uint32_t p = s.t[k - 1][b];
            s.t[k][b] = (p >> 8) ^ s.t[0][p & 0xFFu];
        }
    return s;
}

// Host-side CRC-32C used by the runtime for image headers; byte at a time.
inline uint32_t host_crc32c(const void *data, uint64_t n)
{
    static constexpr SliceTables tbl = make_slice_tables();
    const uint8_t *p = static_cast<const uint8_t *>(data);
    uint32_t c = 0xFFFFFFFFu;
    for (uint64_t i = 0; i < n; ++i) c = tbl.t[0][(c ^ p[i]) & 0xFFu] ^ (c >> 8);
    return c ^ 0xFFFFFFFFu;
}

}  // namespace snapk
