/* Input generator only (no snapshot arithmetic): xorshift64* byte stream.
 * State x != 0; each step: x ^= x >> 12; x ^= x << 25; x ^= x >> 27;
 * output x * 0x2545F4914F6CDD1D, emitted as 8 little-endian bytes. */
#include <stdint.h>
#include <string.h>

void fill_xorshift64star(uint8_t *out, uint64_t n, uint64_t x)
{
    uint64_t i = 0;
    while (i < n) {
        x ^= x >> 12;
        x ^= x << 25;
        x ^= x >> 27;
        uint64_t v = x * 0x2545F4914F6CDD1DULL;
        for (int b = 0; b < 8 && i < n; ++b, ++i) out[i] = (uint8_t)(v >> (8 * b));
    }
}
