// The host-link ceiling of SM-initiated traffic.
//
// The gather and scatter kernels move the image over the host link with SM
// loads and stores to pinned, mapped host memory.  On the B300 machines this
// library was measured on, every SM store form (16-byte stores from all
// lanes, a TMA bulk store from shared memory, plain load/store with no
// shared memory) saturates at the same rate, below what the copy engines
// reach, so the roofline a link-bound kernel can meet is the SM path's own
// ceiling.  snap_link_ceiling measures it with the simplest form: each warp
// copies 8 KiB blocks with sixteen 16-byte loads in flight per lane, in one
// direction or in both at once (the ceiling of a launch that mixes
// checkpoints and restores, as the serving loop's rounds do).
#include "snap.h"
#include "runtime_internal.h"

#include <algorithm>

namespace snapk {

constexpr uint32_t kProbeBlock = 8192;

__global__ void __launch_bounds__(256) k_link_copy(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                                                   uint64_t nblk)
{
    const int lane = threadIdx.x & 31;
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t b = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nblk; b += nw) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src + b * kProbeBlock);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst + b * kProbeBlock);
        uint4 v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = s4[lane + 32 * u];
#pragma unroll
        for (int u = 0; u < 16; ++u) d4[lane + 32 * u] = v[u];
    }
}

// Both directions at once: even warps copy device -> host, odd warps host
// -> device, each over its own pair of buffers.
__global__ void __launch_bounds__(256) k_link_copy_both(const uint8_t *__restrict__ d_src, uint8_t *__restrict__ h_dst,
                                                        const uint8_t *__restrict__ h_src, uint8_t *__restrict__ d_dst,
                                                        uint64_t nblk)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5) / 2;
    const uint8_t *src = (gw & 1) ? h_src : d_src;
    uint8_t *dst = (gw & 1) ? d_dst : h_dst;
    for (uint64_t b = gw >> 1; b < nblk; b += nw) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src + b * kProbeBlock);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst + b * kProbeBlock);
        uint4 v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = s4[lane + 32 * u];
#pragma unroll
        for (int u = 0; u < 16; ++u) d4[lane + 32 * u] = v[u];
    }
}

}  // namespace snapk

extern "C" int snap_link_ceiling(int device, int direction, uint64_t bytes, int reps, double *gbs)
{
    using namespace snapk;
    if (!gbs || direction < 0 || direction > 2 || reps < 1 || bytes < kProbeBlock) return SNAP_EINVAL;
    *gbs = 0.0;
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return SNAP_ECUDA;
    if (cudaSetDevice(dev) != cudaSuccess) return SNAP_EINVAL;
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return SNAP_ECUDA;
    const uint64_t nblk = bytes / kProbeBlock;
    const uint64_t n = nblk * kProbeBlock;
    const bool both = direction == 2;
    // both directions: the second half of each buffer serves the other direction
    const uint64_t nalloc = both ? 2 * n : n;
    uint8_t *d = nullptr, *h = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc((void **)&d, nalloc);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&h, nalloc, cudaHostAllocMapped | cudaHostAllocPortable);
    uint8_t *hd = e == cudaSuccess ? mapped_device_ptr(h) : nullptr;
    if (e == cudaSuccess && !hd) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = cudaMemset(d, 0x5A, nalloc);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = 0.f;
    const int grid = prop.multiProcessorCount * 4;
    const uint8_t *src = direction == 0 ? d : hd;
    uint8_t *dst = direction == 0 ? hd : d;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {  // the first launch is a warm-up
        e = cudaEventRecord(a, st);
        if (e == cudaSuccess) {
            if (both) k_link_copy_both<<<2 * grid, 256, 0, st>>>(d, hd, hd + n, d + n, nblk);
            else k_link_copy<<<grid, 256, 0, st>>>(src, dst, nblk);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && r > 0 && ms > 0.f) best = std::max(best, (float)((both ? 2 : 1) * n / (ms * 1e-3) / 1e9));
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st) cudaStreamDestroy(st);
    cudaFree(d);
    cudaFreeHost(h);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SNAP_ENOMEM : cuda_status(e);
    *gbs = best;
    return SNAP_OK;
}
