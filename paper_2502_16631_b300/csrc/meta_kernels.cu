// Metadata kernels of libsnap: image record headers, the dirty-chunk diff
// with ordered (index-ascending) compaction, and the incremental patch
// layout.  Incremental checkpointing is the optimisation of CRIUgpu Sec. 7
// (Check-N-Run); the patch layout is the one snap_format.h states.
//
// Ordering is deterministic: the dirty list comes from a block-count / scan /
// scatter sequence over ascending chunk indices, never from atomics.
#include "snap_internal.h"

namespace snapk {

__device__ __forceinline__ uint64_t upg(uint64_t x) { return (x + 4095u) & ~uint64_t(4095u); }

__global__ void k_stamp(Result *res, int idx)
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    res->ts[idx] = t;
}

cudaError_t launch_stamp(Result *res, int idx, cudaStream_t st)
{
    k_stamp<<<1, 1, 0, st>>>(res, idx);
    return cudaGetLastError();
}

// ---------------------------------------------------- snapshot cut (shadow)
// The cut of an asynchronous checkpoint: every chunk of every allocation is
// copied device to device into the set's shadow buffer (packed layout,
// allocation k at shadow + state_off_k), so the caller may resume writing
// its allocations while the image is produced from the shadow.  Each warp
// copies whole chunks with 16-byte loads and stores, 4 in flight per lane.
__device__ __forceinline__ uint64_t find_alloc_chunk(const AllocDesc *a, uint64_t n, uint64_t chunk)
{
    uint64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a[mid].chunk0 <= chunk) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_shadow_copy(const AllocDesc *__restrict__ allocs, uint64_t n_allocs, uint64_t C, uint64_t n_chunks,
                              uint8_t *shadow)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t c = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < n_chunks; c += warps) {
        const AllocDesc a = allocs[find_alloc_chunk(allocs, n_allocs, c)];
        const uint64_t off = (c - a.chunk0) * C;
        const uint64_t L = (a.bytes - off) < C ? (a.bytes - off) : C;
        const uint4 *s = reinterpret_cast<const uint4 *>(a.ptr + off);
        uint4 *d = reinterpret_cast<uint4 *>(shadow + a.state_off + off);
        const uint64_t nb = L >> 4;
        uint64_t q = lane;
        for (; q + 96 < nb; q += 128) {
            const uint4 v0 = s[q], v1 = s[q + 32], v2 = s[q + 64], v3 = s[q + 96];
            d[q] = v0;
            d[q + 32] = v1;
            d[q + 64] = v2;
            d[q + 96] = v3;
        }
        for (; q < nb; q += 32) d[q] = s[q];
        const uint64_t rem = L & 15u;
        if ((uint64_t)lane < rem) {
            const uint8_t *sb = reinterpret_cast<const uint8_t *>(a.ptr + off);
            shadow[a.state_off + off + (nb << 4) + lane] = sb[(nb << 4) + lane];
        }
    }
}

cudaError_t launch_shadow_copy(const AllocDesc *allocs, uint64_t n_allocs, uint64_t C, uint64_t n_chunks,
                               uint8_t *shadow, int sms, cudaStream_t st)
{
    if (n_chunks == 0) return cudaSuccess;
    k_shadow_copy<<<sms * 8, 256, 0, st>>>(allocs, n_allocs, C, n_chunks, shadow);
    return cudaGetLastError();
}

// ------------------------------------------------ full image: record headers
// Block k writes allocation k's 32-byte record {bytes, n, data_off, 0} and
// zeroes the padding between its hash array and its data.  (The hashes, the
// data and the data padding are written by the gather tiles.)
__global__ void k_full_meta(const AllocDesc *__restrict__ allocs, uint64_t n_allocs, uint64_t C,
                            const CallParams *cp)
{
    uint8_t *image = cp->image;
    const uint64_t k = blockIdx.x;
    if (k >= n_allocs) return;
    const AllocDesc a = allocs[k];
    const uint64_t nk = (a.bytes + C - 1) / C;
    uint64_t *rec = reinterpret_cast<uint64_t *>(image + a.rec_off);
    if (threadIdx.x == 0) {
        rec[0] = a.bytes;
        rec[1] = nk;
        rec[2] = a.data_off;
        rec[3] = 0;
    }
    // [rec_off + 32 + 4n, data_off) is 4-byte aligned at both ends
    uint32_t *z = reinterpret_cast<uint32_t *>(image + a.rec_off + 32 + 4 * nk);
    const uint64_t nz = (a.data_off - (a.rec_off + 32 + 4 * nk)) / 4;
    for (uint64_t q = threadIdx.x; q < nz; q += blockDim.x) z[q] = 0u;
    // a zero-byte allocation has no chunk tile to pad its (empty) data
}

cudaError_t launch_full_meta(const AllocDesc *allocs, uint64_t n_allocs, uint64_t C, const CallParams *cp,
                             cudaStream_t st)
{
    if (n_allocs == 0) return cudaSuccess;
    k_full_meta<<<(unsigned)n_allocs, 128, 0, st>>>(allocs, n_allocs, C, cp);
    return cudaGetLastError();
}

// ----------------------------------------------------------- diff + compact
// dirty(c) = cur[c] != prev[c], over the chunk range [c0, c0 + n).  The
// range form lets an incremental checkpoint diff one group of allocations
// at a time; the dirty list stays globally ascending because the groups
// are diffed in chunk order, each continuing the running count.
__global__ void k_diff_count(const uint32_t *__restrict__ cur, const uint32_t *__restrict__ prev, uint64_t c0,
                             uint64_t n, unsigned int *blockcnt)
{
    const uint64_t i = (uint64_t)blockIdx.x * kDiffBlock + threadIdx.x;
    const int d = i < n && cur[c0 + i] != prev[c0 + i];
    const int cnt = __syncthreads_count(d);
    if (threadIdx.x == 0) blockcnt[blockIdx.x] = (unsigned)cnt;
}

// Block-wide exclusive scan of one value per thread (blockDim == 1024).
__device__ unsigned long long block_exscan(unsigned long long v, unsigned long long *total)
{
    __shared__ unsigned long long wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long s = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= o) s += y;
        }
        wsum[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    const unsigned long long before = (warp ? wsum[warp - 1] : 0ull) + x - v;
    *total = wsum[31];
    __syncthreads();
    return before;
}

// `run` holds the dirty entries listed so far (0 for a whole-state diff);
// the range's entries go after them, and gbeg / gcnt (optional) receive the
// range's first list position and count.
__global__ void k_diff_scan(const unsigned int *blockcnt, uint64_t nb, unsigned long long *blockoff,
                            unsigned long long *run, unsigned long long *gbeg, unsigned long long *gcnt)
{
    const unsigned long long carry0 = *run;
    __syncthreads();  // every thread has read `run` before thread 0 rewrites it
    unsigned long long carry = carry0;
    for (uint64_t base = 0; base < nb; base += kDiffBlock) {
        const uint64_t b = base + threadIdx.x;
        const unsigned long long v = b < nb ? blockcnt[b] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = block_exscan(v, &tot);
        if (b < nb) blockoff[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        if (gbeg) *gbeg = carry0;
        if (gcnt) *gcnt = carry - carry0;
        *run = carry;
    }
}

__global__ void k_diff_list(const uint32_t *__restrict__ cur, const uint32_t *__restrict__ prev, uint64_t c0,
                            uint64_t n, const unsigned long long *blockoff, uint32_t *dlist)
{
    __shared__ unsigned int wcnt[32];
    const uint64_t i = (uint64_t)blockIdx.x * kDiffBlock + threadIdx.x;
    const uint64_t c = c0 + i;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool d = i < n && cur[c] != prev[c];
    const unsigned int ball = __ballot_sync(0xFFFFFFFFu, d);
    if (lane == 0) wcnt[warp] = __popc(ball);
    __syncthreads();
    unsigned int before = 0;
    for (int q = 0; q < warp; ++q) before += wcnt[q];
    const unsigned int rank = before + __popc(ball & ((1u << lane) - 1u));
    if (d) dlist[blockoff[blockIdx.x] + rank] = (uint32_t)c;
}

cudaError_t launch_diff_range(const uint32_t *cur, const uint32_t *prev, uint64_t c0, uint64_t n,
                              unsigned int *blockcnt, unsigned long long *blockoff, uint32_t *dlist,
                              unsigned long long *run, unsigned long long *gbeg, unsigned long long *gcnt,
                              cudaStream_t st)
{
    const uint64_t nb = (n + kDiffBlock - 1) / kDiffBlock;
    if (nb) k_diff_count<<<(unsigned)nb, kDiffBlock, 0, st>>>(cur, prev, c0, n, blockcnt);
    k_diff_scan<<<1, kDiffBlock, 0, st>>>(blockcnt, nb, blockoff, run, gbeg, gcnt);
    if (nb) k_diff_list<<<(unsigned)nb, kDiffBlock, 0, st>>>(cur, prev, c0, n, blockoff, dlist);
    return cudaGetLastError();
}

cudaError_t launch_diff(const uint32_t *cur, const uint32_t *prev, uint64_t n, unsigned int *blockcnt,
                        unsigned long long *blockoff, uint32_t *dlist, Result *res, cudaStream_t st)
{
    // res->n_dirty is zero at the start of every launch sequence
    return launch_diff_range(cur, prev, 0, n, blockcnt, blockoff, dlist, &res->n_dirty, nullptr, nullptr, st);
}

// ------------------------------------------------------------ patch layout
// For allocation k with n_k chunks and nd_k dirty ones:
//   meta_k = 32 + 4 n_k + 4 + 4 nd_k bytes, padded to 4 KiB
//   data_k = sum over its dirty chunks of the chunk length padded to 4 KiB
// Record 0 starts at 64, every later record on a page boundary.
__device__ uint64_t lower_bound_u32(const uint32_t *a, uint64_t n, uint64_t key)
{
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if ((uint64_t)a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Allocations [a0, a0 + na); `run_off` carries the patch offset where
// allocation a0's record starts from the previous range (a0 == 0 starts
// after the 64-byte header).  The dirty list must already hold every dirty
// chunk of allocations < a0 + na, and no later one.
__global__ void k_patch_layout(const AllocDesc *__restrict__ allocs, uint64_t a0, uint64_t na, uint64_t C,
                               const uint32_t *__restrict__ dlist, uint64_t *patch_rec, uint64_t *patch_data,
                               uint64_t *dstart, const CallParams *cp, Result *res, unsigned long long *run_off)
{
    const uint64_t cap = cp->cap;
    const unsigned long long nd_all = res->n_dirty;
    unsigned long long carry = a0 == 0 ? 64ull : *run_off;
    __syncthreads();  // every thread has read `run_off` before thread 0 rewrites it
    const uint64_t a1 = a0 + na;
    for (uint64_t base = a0; base < a1; base += kDiffBlock) {
        const uint64_t k = base + threadIdx.x;
        unsigned long long R = 0, meta_pad = 0, ds = 0;
        if (k < a1) {
            const AllocDesc a = allocs[k];
            const uint64_t nk = (a.bytes + C - 1) / C;
            ds = lower_bound_u32(dlist, nd_all, a.chunk0);
            const uint64_t de = lower_bound_u32(dlist, nd_all, a.chunk0 + nk);
            const uint64_t nd = de - ds;
            uint64_t data = nd * C;
            if (nd && dlist[de - 1] == a.chunk0 + nk - 1) {
                const uint64_t last = a.bytes - (nk - 1) * C;
                data = data - C + upg(last);
            }
            const uint64_t meta = 32 + 4 * nk + 4 + 4 * nd;
            meta_pad = (k == 0) ? upg(64 + meta) - 64 : upg(meta);
            R = meta_pad + data;
        }
        unsigned long long tot;
        const unsigned long long ex = block_exscan(R, &tot);
        if (k < a1) {
            const unsigned long long rec = carry + ex;
            patch_rec[k] = rec;
            patch_data[k] = rec + meta_pad;
            dstart[k] = ds;
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        dstart[a1] = nd_all;
        *run_off = carry;
        res->patch_bytes = carry;
        if (carry > cap) res->cap_exceeded = 1ull;
    }
}

cudaError_t launch_patch_layout_range(const AllocDesc *allocs, uint64_t a0, uint64_t na, uint64_t C,
                                      const uint32_t *dlist, uint64_t *patch_rec, uint64_t *patch_data,
                                      uint64_t *dstart, const CallParams *cp, Result *res,
                                      unsigned long long *run_off, cudaStream_t st)
{
    k_patch_layout<<<1, kDiffBlock, 0, st>>>(allocs, a0, na, C, dlist, patch_rec, patch_data, dstart, cp, res,
                                             run_off);
    return cudaGetLastError();
}

cudaError_t launch_patch_layout(const AllocDesc *allocs, uint64_t n_allocs, uint64_t C, const uint32_t *dlist,
                                uint64_t *patch_rec, uint64_t *patch_data, uint64_t *dstart, const CallParams *cp,
                                Result *res, cudaStream_t st)
{
    // res->pad[0] serves as the running offset of a whole-state layout
    return launch_patch_layout_range(allocs, 0, n_allocs, C, dlist, patch_rec, patch_data, dstart, cp, res,
                                     &res->pad[0], st);
}

// Block k writes allocation k's patch metadata: record header, all new
// hashes, the dirty count, the ascending dirty index list and zero padding.
__global__ void k_patch_meta(const AllocDesc *__restrict__ allocs, uint64_t a0, uint64_t n_allocs, uint64_t C,
                             const uint32_t *__restrict__ cur, const uint32_t *__restrict__ dlist,
                             const uint64_t *__restrict__ patch_rec, const uint64_t *__restrict__ patch_data,
                             const uint64_t *__restrict__ dstart, const Result *res, const CallParams *cp)
{
    if (res->cap_exceeded) return;
    uint8_t *image = cp->image;
    const uint64_t k = a0 + blockIdx.x;
    if (k >= n_allocs) return;
    const AllocDesc a = allocs[k];
    const uint64_t nk = (a.bytes + C - 1) / C;
    const uint64_t rec = patch_rec[k], data = patch_data[k];
    const uint64_t ds = dstart[k], nd = dstart[k + 1] - ds;
    uint64_t *r64 = reinterpret_cast<uint64_t *>(image + rec);
    if (threadIdx.x == 0) {
        r64[0] = a.bytes;
        r64[1] = nk;
        r64[2] = data;
        r64[3] = 0;
    }
    uint32_t *h = reinterpret_cast<uint32_t *>(image + rec + 32);
    for (uint64_t i = threadIdx.x; i < nk; i += blockDim.x) h[i] = cur[a.chunk0 + i];
    if (threadIdx.x == 0) h[nk] = (uint32_t)nd;
    for (uint64_t j = threadIdx.x; j < nd; j += blockDim.x) h[nk + 1 + j] = dlist[ds + j] - (uint32_t)a.chunk0;
    const uint64_t zlo = rec + 36 + 4 * nk + 4 * nd;
    uint32_t *z = reinterpret_cast<uint32_t *>(image + zlo);
    const uint64_t nz = (data - zlo) / 4;
    for (uint64_t q = threadIdx.x; q < nz; q += blockDim.x) z[q] = 0u;
}

cudaError_t launch_patch_meta_range(const AllocDesc *allocs, uint64_t a0, uint64_t na, uint64_t C,
                                    const uint32_t *cur, const uint32_t *dlist, const uint64_t *patch_rec,
                                    const uint64_t *patch_data, const uint64_t *dstart, const Result *res,
                                    const CallParams *cp, cudaStream_t st)
{
    if (na == 0) return cudaSuccess;
    k_patch_meta<<<(unsigned)na, 256, 0, st>>>(allocs, a0, a0 + na, C, cur, dlist, patch_rec, patch_data, dstart,
                                               res, cp);
    return cudaGetLastError();
}

cudaError_t launch_patch_meta(const AllocDesc *allocs, uint64_t n_allocs, uint64_t C, const uint32_t *cur,
                              const uint32_t *dlist, const uint64_t *patch_rec, const uint64_t *patch_data,
                              const uint64_t *dstart, const Result *res, const CallParams *cp, cudaStream_t st)
{
    return launch_patch_meta_range(allocs, 0, n_allocs, C, cur, dlist, patch_rec, patch_data, dstart, res, cp, st);
}

}  // namespace snapk
