// Large host-to-host copies between pinned staging slots and pageable
// images (ring and server).  Destination lines are written with
// non-temporal (streaming) stores, so the CPU neither reads the destination
// before writing it nor keeps it in cache: one read and one write of DRAM
// per byte instead of two reads and a write.  AVX-512 when the CPU has it,
// else AVX2, else memcpy; unaligned heads and tails go through memcpy.
#pragma once
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <immintrin.h>

namespace snapk {

__attribute__((target("avx512f"))) inline void stream_copy_avx512(uint8_t *d, const uint8_t *s, uint64_t n)
{
    uint64_t i = 0;
    for (; i + 256 <= n; i += 256) {
        const __m512i a = _mm512_loadu_si512(s + i);
        const __m512i b = _mm512_loadu_si512(s + i + 64);
        const __m512i c = _mm512_loadu_si512(s + i + 128);
        const __m512i e = _mm512_loadu_si512(s + i + 192);
        _mm512_stream_si512(reinterpret_cast<__m512i *>(d + i), a);
        _mm512_stream_si512(reinterpret_cast<__m512i *>(d + i + 64), b);
        _mm512_stream_si512(reinterpret_cast<__m512i *>(d + i + 128), c);
        _mm512_stream_si512(reinterpret_cast<__m512i *>(d + i + 192), e);
    }
    for (; i + 64 <= n; i += 64) _mm512_stream_si512(reinterpret_cast<__m512i *>(d + i), _mm512_loadu_si512(s + i));
    _mm_sfence();
    if (i < n) memcpy(d + i, s + i, n - i);
}

__attribute__((target("avx2"))) inline void stream_copy_avx2(uint8_t *d, const uint8_t *s, uint64_t n)
{
    uint64_t i = 0;
    for (; i + 128 <= n; i += 128) {
        const __m256i a = _mm256_loadu_si256(reinterpret_cast<const __m256i *>(s + i));
        const __m256i b = _mm256_loadu_si256(reinterpret_cast<const __m256i *>(s + i + 32));
        const __m256i c = _mm256_loadu_si256(reinterpret_cast<const __m256i *>(s + i + 64));
        const __m256i e = _mm256_loadu_si256(reinterpret_cast<const __m256i *>(s + i + 96));
        _mm256_stream_si256(reinterpret_cast<__m256i *>(d + i), a);
        _mm256_stream_si256(reinterpret_cast<__m256i *>(d + i + 32), b);
        _mm256_stream_si256(reinterpret_cast<__m256i *>(d + i + 64), c);
        _mm256_stream_si256(reinterpret_cast<__m256i *>(d + i + 96), e);
    }
    _mm_sfence();
    if (i < n) memcpy(d + i, s + i, n - i);
}

inline void stream_copy(void *dst, const void *src, uint64_t n)
{
    uint8_t *d = static_cast<uint8_t *>(dst);
    const uint8_t *s = static_cast<const uint8_t *>(src);
    if (n < (64u << 10)) {
        memcpy(d, s, n);
        return;
    }
    // align the destination to 64 bytes for the streaming stores
    const uint64_t head = (64u - ((uintptr_t)d & 63u)) & 63u;
    if (head) {
        memcpy(d, s, head);
        d += head;
        s += head;
        n -= head;
    }
    // SNAP_COPY_NT=0 selects plain memcpy (cached stores), for measurements
    static const int level = [] {
        const char *e = getenv("SNAP_COPY_NT");
        if (e && e[0] == '0') return 0;
        return __builtin_cpu_supports("avx512f") ? 2 : (__builtin_cpu_supports("avx2") ? 1 : 0);
    }();
    if (level == 2) stream_copy_avx512(d, s, n);
    else if (level == 1) stream_copy_avx2(d, s, n);
    else memcpy(d, s, n);
}

}  // namespace snapk
