// The host-memory ceiling of staged transfers.
//
// A pageable image cannot be reached by the GPU: its bytes cross a host copy
// between the image and a pinned, mapped staging slot (the ring's and the
// server's copy workers, host_copy.h), and the slot crosses the link.  Each
// staged byte therefore costs host DRAM one read and one write for the copy
// plus one access for the link transfer.  snap_host_copy_ceiling measures the
// first part with the workers' own copy routine: `threads` host threads copy
// a pinned buffer into a pageable one (direction 0, as a checkpoint drains a
// slot), the other way (1, as a restore fills one), or half the threads each
// way at once (2, the serving loop's mix), optionally while SM loads and
// stores move bytes over the link in both directions (with_link), which is
// the host DRAM traffic the copies share in the serving loop.
#include "snap.h"
#include "runtime_internal.h"
#include "host_copy.h"

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

namespace snapk {
namespace {

constexpr uint32_t kLoadBlock = 8192;

// Link load for with_link: even warps device -> host, odd warps host ->
// device, each over its own half of the buffers, repeated `passes` times.
__global__ void __launch_bounds__(256) k_link_load(const uint8_t *__restrict__ d_src, uint8_t *__restrict__ h_dst,
                                                   const uint8_t *__restrict__ h_src, uint8_t *__restrict__ d_dst,
                                                   uint64_t nblk, int passes)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5) / 2;
    const uint8_t *src = (gw & 1) ? h_src : d_src;
    uint8_t *dst = (gw & 1) ? d_dst : h_dst;
    for (int p = 0; p < passes; ++p)
        for (uint64_t b = gw >> 1; b < nblk; b += nw) {
            const uint4 *s4 = reinterpret_cast<const uint4 *>(src + b * kLoadBlock);
            uint4 *d4 = reinterpret_cast<uint4 *>(dst + b * kLoadBlock);
            uint4 v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = s4[lane + 32 * u];
#pragma unroll
            for (int u = 0; u < 16; ++u) d4[lane + 32 * u] = v[u];
        }
}

double seconds_now()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace
}  // namespace snapk

extern "C" int snap_host_copy_ceiling(int threads, int direction, uint64_t bytes, int reps, int with_link,
                                      double *gbs)
{
    using namespace snapk;
    if (!gbs || threads < 1 || threads > 256 || direction < 0 || direction > 2 || reps < 1 ||
        bytes < (1u << 20))
        return SNAP_EINVAL;
    if (direction == 2 && threads < 2) return SNAP_EINVAL;
    *gbs = 0.0;
    const uint64_t n = bytes & ~uint64_t(4095u);
    const bool both = direction == 2;
    const uint64_t nalloc = both ? 2 * n : n;  // direction 2: each half of the buffers serves one way
    uint8_t *pinned = nullptr;
    cudaError_t e = cudaHostAlloc((void **)&pinned, nalloc, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SNAP_ENOMEM;
    }
    uint8_t *pageable = static_cast<uint8_t *>(std::aligned_alloc(4096, nalloc));
    if (!pageable) {
        cudaFreeHost(pinned);
        return SNAP_ENOMEM;
    }
    std::memset(pageable, 0x5A, nalloc);  // fault every page in before timing
    std::memset(pinned, 0xA5, nalloc);

    // optional link load: about twice the copies' expected duration worth of passes
    uint8_t *d = nullptr, *hl = nullptr, *hld = nullptr;
    cudaStream_t st = nullptr;
    int dev = 0, sms = 148;
    const uint64_t lbytes = 1ull << 30;
    if (with_link) {
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaMalloc((void **)&d, 2 * lbytes);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&hl, 2 * lbytes, cudaHostAllocMapped | cudaHostAllocPortable);
        if (e == cudaSuccess) {
            hld = mapped_device_ptr(hl);
            if (!hld) e = cudaErrorInvalidValue;
        }
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    }
    double best = 0.0;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {  // the first round is a warm-up
        if (with_link) {
            // 1 GiB each way per pass at ~40 GB/s each way: ~25 ms a pass
            const int passes = std::max(2, (int)(2.0 * (double)n / (threads * 4e9) / 0.025) + 2);
            k_link_load<<<2 * sms * 4, 256, 0, st>>>(d, hld, hld + lbytes, d + lbytes, lbytes / kLoadBlock, passes);
            e = cudaGetLastError();
            if (e != cudaSuccess) break;
        }
        std::vector<std::thread> th;
        const double t0 = seconds_now();
        for (int t = 0; t < threads; ++t) {
            th.emplace_back([&, t] {
                const int group = both ? (t & 1) : direction;       // 0: pinned -> pageable
                const int nt = both ? (threads + 1 - group) / 2 : threads;
                const int idx = both ? t / 2 : t;
                const uint64_t base = both && group ? n : 0;
                const uint64_t lo = base + (n * idx / nt & ~uint64_t(63)), hi = base + (idx + 1 == nt ? n : (n * (idx + 1) / nt & ~uint64_t(63)));
                if (group == 0) stream_copy(pageable + lo, pinned + lo, hi - lo);
                else stream_copy(pinned + lo, pageable + lo, hi - lo);
            });
        }
        for (auto &x : th) x.join();
        const double dt = seconds_now() - t0;
        if (r > 0 && dt > 0) best = std::max(best, (double)(both ? 2 * n : n) / dt / 1e9);
        if (with_link) {
            e = cudaStreamSynchronize(st);
        }
    }
    if (st) cudaStreamDestroy(st);
    cudaFree(d);
    cudaFreeHost(hl);
    std::free(pageable);
    cudaFreeHost(pinned);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SNAP_ENOMEM : cuda_status(e);
    *gbs = best;
    return SNAP_OK;
}
