// snap_hash_chunks: the chunk hasher on its own, for any 16-byte aligned
// device buffer.  It runs the persistent tile kernel with one OP_HASH job;
// the job descriptor, allocation descriptor, tile cursor and result live in
// library-owned device scratch allocated once per device.
#include "snap.h"
#include "runtime_internal.h"

#include <cstring>
#include <mutex>

namespace snapk {
namespace {

struct HashScratch {
    alignas(128) uint8_t maps[kTmapPieces * kTmapBytes];  // the buffer's tensor maps (hash staging)
    AllocDesc desc;
    unsigned long long cursor;
    unsigned long long pad;
    Result res;
    Job job;
};

struct HashCtx {
    bool ready = false;
    int sms = 0;
    HashScratch *d = nullptr;   // device scratch
    HashScratch *h = nullptr;   // pinned staging
    Result *h_res = nullptr;
    std::mutex mu;
};

HashCtx g_ctx[64];

int ctx_init(HashCtx &c, int dev)
{
    if (c.ready) return SNAP_OK;
    cudaDeviceProp p{};
    cudaError_t e = cudaGetDeviceProperties(&p, dev);
    if (e == cudaSuccess) e = init_tile_kernel();
    if (e == cudaSuccess) e = cudaMalloc((void **)&c.d, sizeof(HashScratch));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&c.h, sizeof(HashScratch), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&c.h_res, sizeof(Result), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaFree(c.d);
        cudaFreeHost(c.h);
        cudaFreeHost(c.h_res);
        c.d = nullptr;
        c.h = nullptr;
        c.h_res = nullptr;
        return cuda_status(e);
    }
    c.sms = p.multiProcessorCount;
    c.ready = true;
    return SNAP_OK;
}

}  // namespace
}  // namespace snapk

using namespace snapk;

extern "C" int snap_hash_chunks(const void *dptr, uint64_t bytes, uint64_t chunk_bytes, uint32_t *hashes,
                                void *stream)
{
    if (chunk_bytes < 4096 || chunk_bytes % 4096 || chunk_bytes > (16u << 20)) return SNAP_EINVAL;
    if ((uintptr_t)dptr & 15u) return SNAP_EINVAL;
    if (bytes == 0) return SNAP_OK;
    if (!dptr || !hashes) return SNAP_EINVAL;
    const uint64_t n = (bytes + chunk_bytes - 1) / chunk_bytes;
    if (n > 0xFFFFFFFFull) return SNAP_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SNAP_ECUDA;
    HashCtx &c = g_ctx[dev];
    std::lock_guard<std::mutex> lk(c.mu);
    int rc = ctx_init(c, dev);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    HashScratch &h = *c.h;
    std::memset(&h, 0, sizeof h);
    h.desc.ptr = (uint64_t)(uintptr_t)dptr;
    h.desc.bytes = bytes;
    if (encode_hash_maps(h.desc.ptr, bytes, chunk_bytes, h.maps)) h.desc.tmap = (uint64_t)(uintptr_t)c.d->maps;
    h.res.first_bad = ~0ull;
    h.job.allocs = &c.d->desc;
    h.job.n_allocs = 1;
    h.job.chunk_bytes = chunk_bytes;
    h.job.n_tiles = n;
    h.job.op = OP_HASH;
    h.job.hash_out = hashes;
    h.job.res = &c.d->res;
    const TileShape sh = default_hash_shape(c.sms);
    const CombineConsts cc = make_combine_consts(chunk_bytes, sh.piece);
    cudaError_t e = cudaMemcpyAsync(c.d, c.h, sizeof(HashScratch), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_tiles(&c.d->job, 1, &c.d->cursor, cc, sh, &c.d->res, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.h_res, &c.d->res, sizeof(Result), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    return c.h_res->err ? SNAP_ECUDA : SNAP_OK;
}
