// snap_hash_chunks_noalloc: the chunk hasher for callers that must not
// allocate GPU memory.
//
// Who needs this: code that runs where cudaMalloc is off limits -- inside a
// CUDA-checkpoint or crash handler that must not disturb the allocator it
// is snapshotting, under a memory pool that is already exhausted or frozen,
// or in a process whose allocations are all owned by another framework.
// snap_hash_chunks allocates its scratch on first use; this variant never
// calls cudaMalloc, cudaFree, cudaHostAlloc or any allocating library
// routine.  Its scratch (the buffer descriptor table, the job descriptor,
// the tile cursor and the result block) lives in the file-scope device array
// below, which every GPU that loads libsnap holds until the process exits.
//
// Limits and sharing:
//  - at most kNoAllocMaxBuffers buffers per call (larger requests are
//    refused with SNAP_EINVAL before anything is launched);
//  - every call on a device uses the same array and leaves its contents
//    behind; each call rewrites all of it (descriptors, zeroed cursor and
//    result) before launching, so no state carries over -- but two calls
//    whose work overlaps on the GPU (different streams, or different host
//    threads on one device) race on the array.  The host side serialises
//    calls from one process with a mutex; the GPU side is the caller's to
//    order.
//  - the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress) and opts the kernel into its shared memory;
//  - every call copies its descriptor block to the device from a static,
//    pageable host block and synchronises the caller's stream before it
//    returns, so no call may be made while that stream is being captured
//    into a CUDA graph.
#include "snap.h"
#include "runtime_internal.h"

#include <cstring>
#include <mutex>

namespace snapk {
namespace {

constexpr uint32_t kNoAllocMaxBuffers = SNAP_NOALLOC_MAX_BUFFERS;

struct NoAllocScratch {
    unsigned long long cursor;
    unsigned long long pad;
    Result res;
    Job job;
    AllocDesc desc[kNoAllocMaxBuffers];
};

// The scratch.  In host code this name is only a stand-in for the symbol;
// its device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

struct DeviceSetup {
    bool ready = false;
    int sms = 0;
    NoAllocScratch *dev = nullptr;  // device address of g_noalloc_scratch
};

DeviceSetup g_setup[64];
NoAllocScratch g_host;  // host copy of the call block (pageable, static)
Result g_host_res;
std::mutex g_mu;

int setup_device(int dev)
{
    DeviceSetup &d = g_setup[dev];
    if (d.ready) return SNAP_OK;
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = init_tile_kernel();
    if (e != cudaSuccess) return cuda_status(e);
    d.dev = static_cast<NoAllocScratch *>(p);
    d.sms = sms;
    d.ready = true;
    return SNAP_OK;
}

}  // namespace
}  // namespace snapk

using namespace snapk;

extern "C" int snap_hash_chunks_noalloc(const void *const *dptrs, const uint64_t *bytes, uint32_t n_buffers,
                                        uint64_t chunk_bytes, uint32_t *hashes, void *stream)
{
    if (n_buffers > kNoAllocMaxBuffers) return SNAP_EINVAL;  // beyond the static scratch
    if (chunk_bytes < 4096 || chunk_bytes % 4096 || chunk_bytes > (16u << 20)) return SNAP_EINVAL;
    if (n_buffers && (!dptrs || !bytes)) return SNAP_EINVAL;
    uint64_t chunks = 0;
    for (uint32_t k = 0; k < n_buffers; ++k) {
        if ((uintptr_t)dptrs[k] & 15u) return SNAP_EINVAL;
        if (bytes[k] && !dptrs[k]) return SNAP_EINVAL;
        chunks += (bytes[k] + chunk_bytes - 1) / chunk_bytes;
    }
    if (chunks == 0) return SNAP_OK;
    if (!hashes || chunks > 0xFFFFFFFFull) return SNAP_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SNAP_ECUDA;

    std::lock_guard<std::mutex> lk(g_mu);
    int rc = setup_device(dev);
    if (rc) return rc;
    NoAllocScratch *d = g_setup[dev].dev;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // Rewrite the whole used part of the scratch: zero cursor and result,
    // the job, and one descriptor per buffer (chunk0 = running chunk count).
    NoAllocScratch &h = g_host;
    std::memset(&h, 0, offsetof(NoAllocScratch, desc));
    h.res.first_bad = ~0ull;
    uint64_t c0 = 0, skipped = 0;
    for (uint32_t k = 0; k < n_buffers; ++k) {
        if (bytes[k] == 0) {
            ++skipped;  // zero-byte buffers own no chunks: leave them out of the table
            continue;
        }
        AllocDesc &a = h.desc[k - skipped];
        std::memset(&a, 0, sizeof a);
        a.ptr = (uint64_t)(uintptr_t)dptrs[k];
        a.bytes = bytes[k];
        a.chunk0 = c0;
        c0 += (bytes[k] + chunk_bytes - 1) / chunk_bytes;
    }
    const uint64_t n_desc = n_buffers - skipped;
    h.job.allocs = d->desc;
    h.job.n_allocs = n_desc;
    h.job.chunk_bytes = chunk_bytes;
    h.job.n_tiles = chunks;
    h.job.op = OP_HASH;
    h.job.hash_out = hashes;
    h.job.res = &d->res;
    const size_t used = offsetof(NoAllocScratch, desc) + n_desc * sizeof(AllocDesc);

    const TileShape sh = default_hash_shape(g_setup[dev].sms);
    const CombineConsts cc = make_combine_consts(chunk_bytes, sh.piece);
    // pageable source: the call returns once the bytes are staged, so the
    // static host block may be reused by the next call
    cudaError_t e = cudaMemcpyAsync(d, &h, used, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_tiles(&d->job, 1, &d->cursor, cc, sh, &d->res, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&g_host_res, &d->res, sizeof(Result), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    return g_host_res.err ? SNAP_ECUDA : SNAP_OK;
}
