/* Test helper: CRC-32C computed by the x86 SSE4.2 crc32 instruction, an
 * implementation independent of the oracle's table (the instruction is
 * specified to compute the Castagnoli CRC, reflected, without the initial
 * and final complement, which are applied here). */
#include <nmmintrin.h>
#include <stdint.h>
#include <string.h>

uint32_t hw_crc32c(const uint8_t *p, uint64_t n)
{
    uint64_t c = 0xFFFFFFFFu;
    while (n >= 8) {
        uint64_t v;
        memcpy(&v, p, 8);
        c = _mm_crc32_u64(c, v);
        p += 8;
        n -= 8;
    }
    uint32_t c32 = (uint32_t)c;
    while (n--) c32 = _mm_crc32_u8(c32, *p++);
    return c32 ^ 0xFFFFFFFFu;
}

/* Chunk hashes of one buffer with the hardware instruction. */
void hw_chunk_hashes(const uint8_t *p, uint64_t bytes, uint64_t C, uint32_t *out)
{
    uint64_t n = (bytes + C - 1) / C;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t lo = i * C, hi = lo + C < bytes ? lo + C : bytes;
        out[i] = hw_crc32c(p + lo, hi - lo);
    }
}
