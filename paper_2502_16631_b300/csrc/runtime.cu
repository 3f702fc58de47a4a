// Host runtime of libsnap: sets, image layout, quiesce ("lock", CRIUgpu
// Sec. 3.1.1), graph-captured launch sequences, commit/rollback (Sec. 3.1:
// on failure the previous state stands), restore validation (Sec. 4.4: the
// target must match), the plain per-allocation copy form, and the
// standalone chunk hasher.
#include "snap.h"
#include "snap_format.h"
#include "snap_internal.h"
#include "crc32c_gf2.h"
#include "runtime_internal.h"

#include <cuda.h>  // CUtensorMap and its encoding parameters (the encoder comes through the runtime)

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>

using namespace snapk;

namespace snapk {

// ------------------------------------------------------------ small helpers
static inline uint64_t up_page(uint64_t x) { return (x + 4095u) & ~uint64_t(4095u); }

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

bool fault_injected(const char *what)
{
    const char *f = std::getenv("SNAP_FAULT");
    return f && std::strstr(f, what) != nullptr;
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return SNAP_OK;
    if (e == cudaErrorMemoryAllocation) return SNAP_ENOMEM;
    if (std::getenv("SNAP_LOG")) fprintf(stderr, "libsnap: CUDA error %s\n", cudaGetErrorString(e));
    return SNAP_ECUDA;
}

// Poll `ev` until complete or the deadline passes (bounded wait on the host).
int wait_event(cudaEvent_t ev, double deadline_ms)
{
    int spins = 0;
    for (;;) {
        const cudaError_t q = cudaEventQuery(ev);
        if (q == cudaSuccess) return SNAP_OK;
        if (q != cudaErrorNotReady) return cuda_status(q);
        if (now_ms() > deadline_ms) return SNAP_ETIMEDOUT;
        if (++spins < 2000) std::this_thread::yield();
        else std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// Device-visible address of a host buffer if it is pinned and mapped.
uint8_t *mapped_device_ptr(const void *host)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || at.devicePointer == nullptr) return nullptr;
    return static_cast<uint8_t *>(at.devicePointer);
}

// The host regions this library pinned and mapped for images
// (snap_host_alloc, snap_host_register): base -> bytes.  A caller's image is
// read or written by the kernels through its mapping only when the whole
// range the kernels touch lies inside one such region; a mapping of the
// first byte alone says nothing about the rest (a partly registered buffer,
// or two registrations with an unmapped gap between them).
namespace {
std::mutex g_pinned_mu;
std::map<uintptr_t, uint64_t> g_pinned;
}  // namespace

void pinned_add(const void *p, uint64_t bytes)
{
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    g_pinned[(uintptr_t)p] = bytes;
}

void pinned_remove(const void *p)
{
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    g_pinned.erase((uintptr_t)p);
}

bool pinned_covers(const void *p, uint64_t len)
{
    const uintptr_t a = (uintptr_t)p;
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    auto it = g_pinned.upper_bound(a);
    if (it == g_pinned.begin()) return false;
    --it;
    const uintptr_t lo = it->first;
    const uint64_t n = it->second;
    return a >= lo && a - lo <= n && len <= n - (a - lo);
}

uint8_t *mapped_image_ptr(const void *host, uint64_t len)
{
    if (!host || !pinned_covers(host, len)) return nullptr;
    return mapped_device_ptr(host);
}

uint64_t image_extent(const snap_set_s *s, int mode, uint64_t cap)
{
    return mode == SNAP_FULL ? s->full_bytes : std::min(cap, s->patch_bound);
}

void write_header(uint8_t *h, uint32_t flags, uint64_t C, uint64_t n, uint64_t total, uint64_t gen,
                  uint64_t parent)
{
    uint8_t b[64];
    std::memset(b, 0, sizeof b);
    std::memcpy(b, SNAP_IMG_MAGIC, 8);
    const uint32_t ver = SNAP_IMG_VERSION;
    std::memcpy(b + 8, &ver, 4);
    std::memcpy(b + 12, &flags, 4);
    std::memcpy(b + 16, &C, 8);
    std::memcpy(b + 24, &n, 8);
    std::memcpy(b + 32, &total, 8);
    std::memcpy(b + 40, &gen, 8);
    std::memcpy(b + 48, &parent, 8);
    const uint32_t crc = host_crc32c(b, 56);
    std::memcpy(b + 56, &crc, 4);
    std::memcpy(h, b, 64);
}

int parse_header(const uint8_t *img, uint64_t len, ImageHeader *h)
{
    if (!img || len < SNAP_IMG_HEADER_BYTES) return SNAP_EFORMAT;
    uint8_t b[64];
    std::memcpy(b, img, 64);
    if (std::memcmp(b, SNAP_IMG_MAGIC, 8) != 0) return SNAP_EFORMAT;
    uint32_t ver, crc, pad;
    std::memcpy(&ver, b + 8, 4);
    std::memcpy(&h->flags, b + 12, 4);
    std::memcpy(&h->chunk_bytes, b + 16, 8);
    std::memcpy(&h->n_allocs, b + 24, 8);
    std::memcpy(&h->total, b + 32, 8);
    std::memcpy(&h->generation, b + 40, 8);
    std::memcpy(&h->parent, b + 48, 8);
    std::memcpy(&crc, b + 56, 4);
    std::memcpy(&pad, b + 60, 4);
    if (ver != SNAP_IMG_VERSION || pad != 0 || crc != host_crc32c(b, 56)) return SNAP_EFORMAT;
    if (!(h->flags & SNAP_IMG_FLAG_DEVICE_STATE) || (h->flags & ~3u)) return SNAP_EFORMAT;
    if (h->chunk_bytes < 4096 || h->chunk_bytes % 4096 || h->chunk_bytes > (1ull << 30)) return SNAP_EFORMAT;
    return SNAP_OK;
}

// Walk an image's records (full or patch) against the set's allocations,
// collecting every chunk hash into `hashes` (global chunk order).  For a full
// image also checks that every data offset is where the layout puts it.
int walk_records_io(const snap_set_s *s, const ImageReader &rd, uint64_t len, const ImageHeader &h, uint32_t *hashes)
{
    if (h.chunk_bytes != s->C) return SNAP_EMISMATCH;
    if (h.n_allocs != s->allocs.size()) return SNAP_EMISMATCH;
    if (h.total != s->total_bytes) return SNAP_EMISMATCH;
    const bool patch = (h.flags & SNAP_IMG_FLAG_INCREMENTAL) != 0;
    uint64_t off = SNAP_IMG_HEADER_BYTES;
    for (size_t k = 0; k < s->allocs.size(); ++k) {
        const AllocDesc &a = s->desc[k];
        if (off + 32 > len) return SNAP_EFORMAT;
        uint64_t rec[4];
        if (!rd(off, rec, 32)) return SNAP_EIO;
        if (rec[0] != a.bytes) return SNAP_EMISMATCH;
        const uint64_t nk = (a.bytes + s->C - 1) / s->C;
        if (rec[1] != nk || rec[3] != 0) return SNAP_EFORMAT;
        if (nk > (len - off - 32) / 4) return SNAP_EFORMAT;
        if (hashes && nk && !rd(off + 32, hashes + a.chunk0, 4 * nk)) return SNAP_EIO;
        if (!patch) {
            if (rec[2] != a.data_off || off != a.rec_off) return SNAP_EFORMAT;
            if (a.data_off > len || a.bytes > len - a.data_off) return SNAP_EFORMAT;
            off = up_page(a.data_off + a.bytes);
        } else {
            if (off + 36 + 4 * nk > len) return SNAP_EFORMAT;
            uint32_t nd;
            if (!rd(off + 32 + 4 * nk, &nd, 4)) return SNAP_EIO;
            if (nd > nk || off + 36 + 4 * nk + 4ull * nd > len) return SNAP_EFORMAT;
            if (rec[2] != up_page(off + 36 + 4 * nk + 4ull * nd)) return SNAP_EFORMAT;
            uint64_t d = rec[2];
            int64_t last = -1;
            for (uint32_t j = 0; j < nd; ++j) {
                uint32_t i;
                if (!rd(off + 36 + 4 * nk + 4ull * j, &i, 4)) return SNAP_EIO;
                if (i >= nk || (int64_t)i <= last) return SNAP_EFORMAT;
                last = i;
                const uint64_t L = std::min<uint64_t>(s->C, a.bytes - (uint64_t)i * s->C);
                d += up_page(L);
            }
            off = d;
        }
    }
    if (off > len) return SNAP_EFORMAT;
    return SNAP_OK;
}

int walk_records(const snap_set_s *s, const uint8_t *img, uint64_t len, const ImageHeader &h, uint32_t *hashes)
{
    return walk_records_io(s, [img](uint64_t off, void *dst, uint64_t n) {
        std::memcpy(dst, img + off, n);
        return true;
    }, len, h, hashes);
}

// ------------------------------------------------------------- set layout
// Device arrays are (re)built lazily after registration changes.
static void free_device(snap_set_s *s)
{
    for (auto &g : s->graphs) if (g.exec) cudaGraphExecDestroy(g.exec);
    s->graphs.clear();
    cudaFree(s->d_allocs);
    cudaFree(s->d_tmaps);
    s->d_tmaps = nullptr;
    cudaFree(s->d_hash[0]);
    cudaFree(s->d_hash[1]);
    cudaFree(s->d_cmp);
    cudaFree(s->d_blockcnt);
    cudaFree(s->d_blockoff);
    cudaFree(s->d_dlist);
    cudaFree(s->d_patch_rec);
    cudaFree(s->d_patch_data);
    cudaFree(s->d_dstart);
    cudaFreeHost(s->h_hash_stage);
    s->d_allocs = nullptr;
    s->d_hash[0] = s->d_hash[1] = s->d_cmp = s->d_dlist = nullptr;
    s->d_blockcnt = nullptr;
    s->d_blockoff = nullptr;
    s->d_patch_rec = s->d_patch_data = s->d_dstart = nullptr;
    s->h_hash_stage = nullptr;
    async_free_layout(s);
    lazy_free_layout(s);
}

// Stage count a pipelined incremental checkpoint of this state aims at:
// one stage per max(64 MiB, 4,096 chunks) of state, at most kMaxGroups
// (each stage's dirty chunks are gathered by a few warps, one chunk per
// warp at a time, so a stage with only a handful of dirty chunks would
// leave the link idle); fewer than 2: no pipeline.
static void plan_groups(snap_set_s *s)
{
    const uint64_t kGroupBytes = std::max<uint64_t>(64ull << 20, 4096 * s->C);
    uint64_t cap = kMaxGroups;
    // SNAP_PIPE_GROUPS: a different stage cap (2 .. kMaxPipe), for measurements
    if (const char *e = std::getenv("SNAP_PIPE_GROUPS"))
        cap = std::max<uint64_t>(2, std::min<uint64_t>((uint64_t)kMaxPipe, std::strtoull(e, nullptr, 10)));
    s->n_groups = (int)std::min<uint64_t>(cap, s->total_bytes / kGroupBytes);
}

// The stages of a pipelined incremental checkpoint for hash launches of W
// warps (a warp hashes one chunk at a time).  Every launch but the last
// hashes a whole number of waves (multiples of W chunks), so that its warps
// run out of tiles together and no launch ends in a part-filled wave; the
// last hashes one wave plus the part-filled rest, which keeps the final
// stage (whose gather nothing overlaps) short.  Allocation group g is the
// allocations whose last chunk launch g hashes, a zero-byte allocation
// going with the one before it; a group is empty where one allocation
// spans several launches.  Returns the launch count (below 2: no pipeline).
static int plan_pipeline(snap_set_s *s, uint64_t W)
{
    const uint64_t N = s->n_chunks;
    const uint64_t waves = W ? N / W : 0;
    if (s->n_groups < 2 || waves < 2) return s->n_pipe = 1;
    const uint64_t H = std::min<uint64_t>({(uint64_t)s->n_groups, waves, (uint64_t)kMaxPipe});
    // launches 0 .. H-2 share waves-1 whole waves, the later ones taking
    // the extra wave where they do not divide evenly
    const uint64_t base = (waves - 1) / (H - 1), extra = (waves - 1) % (H - 1);
    s->hb[0] = 0;
    for (uint64_t h = 0; h + 1 < H; ++h) s->hb[h + 1] = s->hb[h] + (base + (h >= H - 1 - extra ? 1 : 0)) * W;
    s->hb[H] = N;
    const size_t n = s->desc.size();
    size_t k = 0;
    s->gal[0] = 0;
    s->gch[0] = 0;
    for (uint64_t h = 0; h < H; ++h) {
        if (h + 1 < H)
            while (k < n && s->desc[k].chunk0 + (s->desc[k].bytes + s->C - 1) / s->C <= s->hb[h + 1]) ++k;
        else
            k = n;
        s->gal[h + 1] = k;
        s->gch[h + 1] = k < n ? s->desc[k].chunk0 : N;
    }
    return s->n_pipe = (int)H;
}

// The driver's tensor-map encoder, looked up once through the runtime (no
// link against the driver library); null if unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled()
{
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiledFn) nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// The hash staging's tensor maps of one buffer: viewed as rows of C/32 bytes
// (floor(bytes / (C/32)) rows, so only whole rows: every full chunk is
// covered, ragged chunks take the cp.async path), one map per piece size
// 32 / 64 / 128 with the matching 32 / 64 / 128-byte swizzle, into `out`
// (kTmapPieces x kTmapBytes).  False if the buffer has no full chunk or a
// map cannot be encoded.
bool encode_hash_maps(uint64_t ptr, uint64_t bytes, uint64_t C, void *out)
{
    static_assert(sizeof(CUtensorMap) == kTmapBytes, "tensor map size");
    const EncodeTiledFn enc = encode_tiled();
    if (!enc || bytes < C || (ptr & 15u)) return false;
    const uint64_t row = C / 32;
    CUtensorMap *maps = static_cast<CUtensorMap *>(out);
    for (int pi = 0; pi < kTmapPieces; ++pi) {
        const cuuint32_t piece = 32u << pi;
        const cuuint64_t dim[2] = {row, bytes / row};
        const cuuint64_t stride[1] = {row};
        const cuuint32_t box[2] = {piece, 32};
        const cuuint32_t estride[2] = {1, 1};
        const CUtensorMapSwizzle sw = pi == 0 ? CU_TENSOR_MAP_SWIZZLE_32B
                                    : pi == 1 ? CU_TENSOR_MAP_SWIZZLE_64B
                                              : CU_TENSOR_MAP_SWIZZLE_128B;
        if (enc(&maps[pi], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, reinterpret_cast<void *>(ptr), dim, stride, box,
                estride, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

// Tensor maps for every allocation of the set (allocations without a full
// chunk, or whose maps cannot be encoded, keep tmap = 0).
static int build_tensor_maps(snap_set_s *s)
{
    const size_t n = s->desc.size();
    if (!encode_tiled() || n == 0) return SNAP_OK;
    std::vector<CUtensorMap> maps(n * kTmapPieces);
    std::vector<char> ok(n, 0);
    for (size_t k = 0; k < n; ++k)
        ok[k] = encode_hash_maps(s->desc[k].ptr, s->desc[k].bytes, s->C, &maps[k * kTmapPieces]);
    cudaError_t e = cudaMalloc((void **)&s->d_tmaps, maps.size() * sizeof(CUtensorMap));
    if (e == cudaSuccess) e = cudaMemcpy(s->d_tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(s->d_tmaps);
        s->d_tmaps = nullptr;
        return cuda_status(e);
    }
    for (size_t k = 0; k < n; ++k)
        s->desc[k].tmap = ok[k] ? (uint64_t)(uintptr_t)(s->d_tmaps + k * kTmapPieces * kTmapBytes) : 0;
    return SNAP_OK;
}

int build_layout(snap_set_s *s)
{
    if (!s->layout_dirty) return SNAP_OK;
    free_device(s);
    s->has_base = false;
    const uint64_t C = s->C;
    s->desc.resize(s->allocs.size());
    uint64_t off = SNAP_IMG_HEADER_BYTES, chunk = 0, state = 0, pack = 0;
    for (size_t k = 0; k < s->allocs.size(); ++k) {
        AllocDesc &a = s->desc[k];
        a.ptr = (uint64_t)(uintptr_t)s->allocs[k].ptr;
        a.bytes = s->allocs[k].bytes;
        a.tmap = 0;  // set by build_tensor_maps
        const uint64_t nk = (a.bytes + C - 1) / C;
        a.chunk0 = chunk;
        a.rec_off = off;
        a.data_off = up_page(off + 32 + 4 * nk);
        // packed (ring) offset: every allocation starts 256-byte aligned so
        // that the kernels' 16-byte accesses to a ring slot stay aligned
        a.state_off = pack;
        pack = (pack + a.bytes + 255u) & ~uint64_t(255u);
        off = up_page(a.data_off + a.bytes);
        chunk += nk;
        state += a.bytes;
    }
    s->n_chunks = chunk;
    s->total_bytes = state;
    plan_groups(s);
    s->full_bytes = off;
    if (chunk > 0xFFFFFFFFull) return SNAP_EINVAL;  // dirty lists hold u32 chunk indices
    // patch upper bound: full image + per allocation the dirty count, index list and a page
    s->patch_bound = off;
    for (size_t k = 0; k < s->allocs.size(); ++k) s->patch_bound += 4096 + 4 + 4 * ((s->desc[k].bytes + C - 1) / C);

    const size_t na = std::max<size_t>(1, s->desc.size());
    const size_t nc = std::max<uint64_t>(1, chunk);
    const size_t nb = (nc + kDiffBlock - 1) / kDiffBlock;
    if (fault_injected("hash_alloc")) return SNAP_ENOMEM;
    cudaError_t e = cudaSuccess;
    auto al = [&](void **p, size_t b) { if (e == cudaSuccess) e = cudaMalloc(p, b); };
    al((void **)&s->d_allocs, na * sizeof(AllocDesc));
    al((void **)&s->d_hash[0], nc * 4);
    al((void **)&s->d_hash[1], nc * 4);
    al((void **)&s->d_cmp, nc * 4);
    al((void **)&s->d_blockcnt, nb * sizeof(unsigned int));
    al((void **)&s->d_blockoff, nb * sizeof(unsigned long long));
    al((void **)&s->d_dlist, nc * 4);
    al((void **)&s->d_patch_rec, na * 8);
    al((void **)&s->d_patch_data, na * 8);
    al((void **)&s->d_dstart, (na + 1) * 8);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->h_hash_stage, nc * 4, cudaHostAllocDefault);
    if (e == cudaSuccess) {
        const int rc = build_tensor_maps(s);
        if (rc) {
            free_device(s);
            return rc;
        }
    }
    if (e == cudaSuccess && !s->desc.empty())
        e = cudaMemcpy(s->d_allocs, s->desc.data(), s->desc.size() * sizeof(AllocDesc), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_device(s);
        return cuda_status(e);
    }
    adopt_cached_shapes(s);
    s->layout_dirty = false;
    return SNAP_OK;
}

// ------------------------------------------------------------ call plumbing

// A previous call that timed out may still be running on the library
// stream; wait for it (bounded) before touching shared buffers again.
int settle(snap_set_s *s, double deadline)
{
    if (!s->in_flight) return SNAP_OK;
    const int rc = wait_event(s->ev[EV_END], deadline);
    if (rc == SNAP_OK) s->in_flight = false;
    return rc == SNAP_ETIMEDOUT ? SNAP_EBUSY : rc;
}

// Quiesce the caller's stream: every operation queued on it must finish
// before the snapshot reads device memory (the lock action, Sec. 3.1.1).
int quiesce(snap_set_s *s, double deadline)
{
    cudaError_t e = cudaEventRecord(s->ev_quiesce, s->user_stream);
    if (e != cudaSuccess) return cuda_status(e);
    return wait_event(s->ev_quiesce, deadline);
}

TileShape shape_for(const snap_set_s *s, int kind)
{
    TileShape sh = s->shape[kind];
    return sh;
}

// The graph for `kind`, captured from `body` on first use; parity selects
// which hash table is "current".
int get_graph(snap_set_s *s, int kind, int parity, const std::function<cudaError_t(cudaStream_t)> &body,
              GraphEntry **out)
{
    *out = nullptr;
    GraphEntry *g = nullptr;
    for (auto &x : s->graphs)
        if (x.kind == kind && x.parity == parity) g = &x;
    if (!g) {
        if (fault_injected("graph")) return SNAP_ENOMEM;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_status(e);
        cudaError_t eb = body(s->st);
        e = cudaStreamEndCapture(s->st, &graph);
        if (eb != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_status(eb != cudaSuccess ? eb : e);
        }
        uint64_t kernels = 0;
        size_t nn = 0;
        if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn) {
            std::vector<cudaGraphNode_t> nodes(nn);
            if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
                for (auto n : nodes) {
                    cudaGraphNodeType ty;
                    if (cudaGraphNodeGetType(n, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
                }
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_status(e);
        s->graphs.push_back(GraphEntry{kind, parity, exec, kernels});
        g = &s->graphs.back();
    }
    *out = g;
    return SNAP_OK;
}

static int run_graph(snap_set_s *s, int kind, int parity, const std::function<cudaError_t(cudaStream_t)> &body)
{
    GraphEntry *g = nullptr;
    const int rc = get_graph(s, kind, parity, body, &g);
    if (rc) return rc;
    s->call_kernels = g->kernels;
    return cuda_status(cudaGraphLaunch(g->exec, s->st));
}

// Fill the per-call block's header part (cursors, result, params).
static void reset_call(snap_set_s *s, uint8_t *image, uint64_t cap)
{
    CallBlock &cb = *s->h_cb;
    std::memset(&cb, 0, offsetof(CallBlock, jobs));
    cb.res.first_bad = ~0ull;
    cb.cp.image = image;
    cb.cp.cap = cap;
}

// Test hook: SNAP_TEST_STALL_TILE=<n> (unset in normal use) makes the warp
// that takes tile n of a direct full checkpoint's gather, of a verify or of
// a fused incremental's hash wait on a stage that no copy fills, so that the
// kernel's bounded wait runs out and its error path runs.
static uint64_t test_stall_tile()
{
    const char *e = std::getenv("SNAP_TEST_STALL_TILE");
    return e && *e ? std::strtoull(e, nullptr, 10) + 1 : 0;
}

static Job base_job(const snap_set_s *s, uint32_t op)
{
    Job j{};
    j.allocs = s->d_allocs;
    j.n_allocs = s->desc.size();
    j.chunk_bytes = s->C;
    j.tile_begin = 0;
    j.n_tiles = s->n_chunks;
    j.op = op;
    j.layout = LAYOUT_IMAGE;
    j.res = &s->d_cb->res;
    if (op == OP_GATHER || op == OP_VERIFY) j.test_stall = test_stall_tile();
    return j;
}

// Enqueue: copy the call block in, then body, then the result out.
static cudaError_t enqueue_prologue(snap_set_s *s, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(s->d_cb, s->h_cb, sizeof(CallBlock), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_stamp(&s->d_cb->res, TS_BEGIN, st);
    return e;
}
static cudaError_t enqueue_epilogue(snap_set_s *s, cudaStream_t st)
{
    cudaError_t e = launch_stamp(&s->d_cb->res, TS_COPY_END, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_res, &s->d_cb->res, sizeof(Result), cudaMemcpyDeviceToHost, st);
    return e;
}

// Milliseconds between two device stamps of the last launch sequence.
static double ts_ms(const snap_set_s *s, int a, int b)
{
    const unsigned long long ta = s->h_res->ts[a], tb = s->h_res->ts[b];
    return (ta && tb && tb >= ta) ? (double)(tb - ta) * 1e-6 : 0.0;
}

static float ev_ms(snap_set_s *s, int a, int b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s->ev[a], s->ev[b]) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

// Launch the graph, wait for it with the deadline, check the kernels' flags.
static int finish(snap_set_s *s, double deadline)
{
    cudaError_t e = cudaEventRecord(s->ev[EV_END], s->st);
    if (e != cudaSuccess) return cuda_status(e);
    const int rc = wait_event(s->ev[EV_END], deadline);
    if (rc == SNAP_ETIMEDOUT) {
        s->in_flight = true;
        return rc;
    }
    if (rc) return rc;
    s->device_err = s->h_res->err;
    if (s->h_res->err) return SNAP_ECUDA;
    return SNAP_OK;
}

int async_ctas(const snap_set_s *s)
{
    // the background gather is bound by the host link, which 8 CTAs
    // saturate on B300 (about 7 GB/s each); more would only take SMs from
    // the caller
    const int c = s->opts.async_ctas ? (int)s->opts.async_ctas : 8;
    return std::max(1, std::min(c, s->sms));
}

// Pipelined incremental checkpoint.  The hash pass (HBM-bound) runs as H
// launches on all but kPipeGatherCtas SMs, back to back on a second stream,
// each launch allowed to start in its predecessor's tail (programmatic
// stream serialization: it reads nothing the predecessor writes); a third
// stream takes each launch's completed allocations through diff, layout and
// metadata, and the library stream gathers their dirty chunks (link-bound)
// on the other SMs while later launches hash.  Groups are whole allocations
// in registration order, so the dirty list stays ascending and every offset
// of the patch is the one the whole-state layout gives: the bytes are those
// of the unpipelined sequence.  Used only when the image capacity covers the
// largest possible patch, because a group's bytes are written before later
// groups are laid out.
static int pipelined_incremental(snap_set_s *s, int cur, uint8_t *dimg, const TileShape &shh, GraphEntry **out)
{
    const int H = s->n_pipe;
    for (cudaStream_t *p : {&s->st_pipe, &s->st_meta})
        if (!*p) {
            const cudaError_t e = cudaStreamCreateWithFlags(p, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                *p = nullptr;
                return cuda_status(e);
            }
        }
    for (int i = 0; i < 2 * H + 1; ++i)
        if (!s->ev_pipe[i]) {
            const cudaError_t e = cudaEventCreateWithFlags(&s->ev_pipe[i], cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_status(e);
        }
    CallBlock &cb = *s->h_cb;
    for (int g = 0; g < H; ++g) {
        Job jh = base_job(s, OP_HASH);
        jh.tile_begin = s->hb[g];
        jh.n_tiles = s->hb[g + 1] - s->hb[g];
        jh.hash_out = s->d_hash[cur];
        cb.jobs[g] = jh;
        Job jg = base_job(s, OP_GATHER_DIRTY);
        jg.host = dimg;
        jg.tile_list = s->d_dlist;
        jg.tile_off_dev = &s->d_cb->gbeg[g];
        jg.n_tiles_dev = &s->d_cb->gcnt[g];
        jg.patch_data = s->d_patch_data;
        jg.dstart = s->d_dstart;
        jg.cap_exceeded = &s->d_cb->res.cap_exceeded;
        cb.jobs[H + g] = jg;
    }
    TileShape shg = s->shape[SHAPE_GATHER];
    shg.ctas = kPipeGatherCtas;
    const CombineConsts cch = make_combine_consts(s->C, shh.piece);
    const CombineConsts ccg = make_combine_consts(s->C, shg.piece);
    const uint32_t *curp = s->d_hash[cur], *prevp = s->d_hash[1 - cur];
    CallBlock *d = s->d_cb;
    return get_graph(s, GK_INCR_PIPE, cur, [&](cudaStream_t q) {
        cudaStream_t h = s->st_pipe;
        cudaError_t e = enqueue_prologue(s, q);
        // fork the hash stream off the capture
        if (e == cudaSuccess) e = cudaEventRecord(s->ev_pipe[0], q);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h, s->ev_pipe[0], 0);
        if (e == cudaSuccess) e = launch_stamp(&d->res, TS_DIFF_END, q);  // copy_ms spans the whole pipeline
        // three streams: h hashes launch after launch; m takes each
        // launch's completed allocations through diff, layout and metadata
        // (they continue the running dirty count and patch offset, so they
        // stay in order); q gathers each group once its metadata is written
        cudaStream_t m = s->st_meta;
        if (e == cudaSuccess) e = cudaStreamWaitEvent(m, s->ev_pipe[0], 0);
        for (int g = 0; g < H && e == cudaSuccess; ++g) {
            // the first launch follows the prologue's copy of the call block,
            // so it waits for it in full
            e = launch_tiles(d->jobs + g, 1, &d->cursor[g], cch, shh, &d->res, h, g > 0);
            if (e == cudaSuccess && g == H - 1) e = launch_stamp(&d->res, TS_HASH_END, h);
            if (e == cudaSuccess) e = cudaEventRecord(s->ev_pipe[1 + g], h);
        }
        for (int g = 0; g < H && e == cudaSuccess; ++g) {
            // m waits for every launch in turn, so group g's metadata runs
            // after launches 0 .. g have all completed (a launch that started
            // in its predecessor's tail may complete before it)
            e = cudaStreamWaitEvent(m, s->ev_pipe[1 + g], 0);
            const uint64_t a0 = s->gal[g], na = s->gal[g + 1] - s->gal[g];
            if (e != cudaSuccess || na == 0) continue;
            e = launch_diff_range(curp, prevp, s->gch[g], s->gch[g + 1] - s->gch[g], s->d_blockcnt, s->d_blockoff,
                                  s->d_dlist, &d->res.n_dirty, &d->gbeg[g], &d->gcnt[g], m);
            if (e == cudaSuccess)
                e = launch_patch_layout_range(s->d_allocs, a0, na, s->C, s->d_dlist, s->d_patch_rec,
                                              s->d_patch_data, s->d_dstart, &d->cp, &d->res, &d->run_off, m);
            if (e == cudaSuccess)
                e = launch_patch_meta_range(s->d_allocs, a0, na, s->C, curp, s->d_dlist, s->d_patch_rec,
                                            s->d_patch_data, s->d_dstart, &d->res, &d->cp, m);
            if (e == cudaSuccess) e = cudaEventRecord(s->ev_pipe[1 + H + g], m);
        }
        for (int g = 0; g < H && e == cudaSuccess; ++g) {
            if (s->gal[g + 1] == s->gal[g]) continue;
            e = cudaStreamWaitEvent(q, s->ev_pipe[1 + H + g], 0);
            if (e == cudaSuccess)
                e = launch_tiles(d->jobs + H + g, 1, &d->cursor[H + g], ccg, shg, &d->res, q);
        }
        // join the hash stream too (its last event precedes the last metadata,
        // but a join must name the stream's own last work)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(q, s->ev_pipe[H], 0);
        if (e == cudaSuccess) e = enqueue_epilogue(s, q);
        return e;
    }, out);
}

// The fused incremental checkpoint (one cooperative launch whose CTAs hash,
// lay out and gather group by group; see FusedIncr).  Groups are runs of
// whole allocations of about equal bytes (at least max(64 MiB, 1024 chunks)
// each, at most kFusedMaxGroups): unlike the launch-per-stage pipeline there
// is no launch boundary to align with the hash waves, so the groups can be
// finer, and the hash CTAs never stop between them.  Fills the group table
// of `f`; returns the group count (below 2: the state is too small).
static int plan_fused(const snap_set_s *s, FusedIncr &f)
{
    const uint64_t min_group = std::max<uint64_t>(64ull << 20, 1024 * s->C);
    const uint64_t G = std::min<uint64_t>((uint64_t)kFusedMaxGroups, s->total_bytes / min_group);
    if (G < 2) return 0;
    const uint64_t per = (s->total_bytes + G - 1) / G;
    int g = 0;
    uint64_t acc = 0;
    f.gal[0] = 0;
    f.gch[0] = 0;
    for (size_t k = 0; k < s->desc.size(); ++k) {
        acc += s->desc[k].bytes;
        if (acc >= (uint64_t)(g + 1) * per && (uint64_t)(g + 1) < G && k + 1 < s->desc.size()) {
            ++g;  // group g - 1 ends after allocation k
            f.gal[g] = k + 1;
            f.gch[g] = s->desc[k + 1].chunk0;
        }
    }
    f.gal[g + 1] = s->desc.size();
    f.gch[g + 1] = s->n_chunks;
    f.n_groups = g + 1;
    return f.n_groups;
}

// Whether the dirty runs of a fused incremental go to the copy engines
// (the default: on B300 the copy engines move device-to-host bytes at 57.3
// GB/s against 52.7 for SM stores, and the 8 SMs of the gather CTAs hash
// instead).
static bool want_dma(const snap_set_s *s)
{
    if (s->opts.incr_copy) return s->opts.incr_copy == SNAP_INCR_COPY_DMA;
    const char *e = std::getenv("SNAP_INCR_COPY");
    if (e && *e) return std::strcmp(e, "sm") != 0;
    return true;
}

// The copy-engine form's host side: the copy stream, its events, and a
// pinned, mapped block with the group records and room for one run per
// chunk (every run holds at least one dirty chunk).
static int dma_prepare(snap_set_s *s)
{
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kDmaStreams && e == cudaSuccess; ++i) {
        if (!s->st_dma[i]) e = cudaStreamCreateWithFlags(&s->st_dma[i], cudaStreamNonBlocking);
        if (e == cudaSuccess && !s->ev_dma[i]) e = cudaEventCreateWithFlags(&s->ev_dma[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess && !s->ev_graph_end) e = cudaEventCreateWithFlags(&s->ev_graph_end, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e);
    const uint64_t need = std::max<uint64_t>(s->n_chunks, 1);
    if (s->runs_cap >= need) return SNAP_OK;
    cudaFreeHost(s->h_rungrp);
    s->h_rungrp = nullptr;
    s->h_runs = nullptr;
    s->runs_cap = 0;
    void *p = nullptr;
    e = cudaHostAlloc(&p, sizeof(RunGroup) * kFusedMaxGroups + sizeof(DirtyRun) * need, cudaHostAllocMapped);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SNAP_ENOMEM;
    }
    s->h_rungrp = static_cast<RunGroup *>(p);
    s->h_runs = reinterpret_cast<DirtyRun *>(static_cast<uint8_t *>(p) + sizeof(RunGroup) * kFusedMaxGroups);
    s->runs_cap = need;
    return SNAP_OK;
}

static bool fused_ok(snap_set_s *s, const TileShape &shh, FusedIncr &f)
{
    if (std::getenv("SNAP_FUSED_OFF")) return false;  // the launch-per-stage pipeline, for measurements
    if (s->sms - 1 - kPipeGatherCtas < 1 || plan_fused(s, f) < 2) return false;
    return fused_incr_fits(shh, s->sms, s->device);
}

static int fused_incremental(snap_set_s *s, int cur, uint8_t *dimg, uint64_t cap, const TileShape &shh,
                             GraphEntry **out)
{
    CallBlock &cb = *s->h_cb;  // the counters were zeroed by reset_call; plan_fused filled the groups
    FusedIncr &f = cb.fused;
    f.prev = s->d_hash[1 - cur];
    f.dlist = s->d_dlist;
    f.patch_rec = s->d_patch_rec;
    f.patch_data = s->d_patch_data;
    f.dstart = s->d_dstart;
    f.host = dimg;
    f.cap = cap;
    f.dma = 0;
    if (want_dma(s) && dma_prepare(s) == SNAP_OK) {
        uint8_t *pub = mapped_device_ptr(s->h_rungrp);
        if (pub) {
            f.dma = 1;
            f.pub = reinterpret_cast<RunGroup *>(pub);
            f.runs = reinterpret_cast<DirtyRun *>(pub + sizeof(RunGroup) * kFusedMaxGroups);
            f.runs_cap = s->runs_cap;
            std::memset(s->h_rungrp, 0, sizeof(RunGroup) * kFusedMaxGroups);
        }
    }
    s->dma_call = f.dma != 0;
    // one metadata CTA, and kPipeGatherCtas gather CTAs unless the copy
    // engines take the dirty runs
    f.n_hash_ctas = s->sms - 1 - (f.dma ? 0 : kPipeGatherCtas);
    Job jh = base_job(s, OP_HASH);
    jh.hash_out = s->d_hash[cur];
    jh.fused = &s->d_cb->fused;
    jh.test_stall = test_stall_tile();  // the give-up test hook reaches the fused hash too
    cb.jobs[0] = jh;
    const CombineConsts cch = make_combine_consts(s->C, shh.piece);
    CallBlock *d = s->d_cb;
    return get_graph(s, GK_INCR_FUSED, cur, [&](cudaStream_t q) {
        cudaError_t e = enqueue_prologue(s, q);
        if (e == cudaSuccess) e = launch_fused_incr(d->jobs, &d->cursor[0], cch, shh, s->sms, &d->res, q);
        if (e == cudaSuccess) e = enqueue_epilogue(s, q);
        return e;
    }, out);
}

// Fill the call block of a checkpoint into the mapped image `dimg` and get
// (capturing it on first use) its graph: FULL = records + gather of every
// chunk with its CRC; INCREMENTAL = hash, diff against the committed table,
// patch layout + metadata, gather of the dirty chunks.  With `from_shadow`
// the kernels read the state from the shadow of an asynchronous checkpoint
// and run on async_ctas(s) CTAs.
int checkpoint_graph(snap_set_s *s, int mode, int cur, uint8_t *dimg, uint64_t cap, bool from_shadow,
                     GraphEntry **out)
{
    const AllocDesc *allocs = from_shadow ? s->d_allocs_shadow : s->d_allocs;
    reset_call(s, dimg, cap);
    s->dma_call = false;
    s->dma_copies = 0;
    TileShape shh = s->shape[SHAPE_HASH], shg = s->shape[SHAPE_GATHER];
    if (from_shadow) shh.ctas = shg.ctas = async_ctas(s);
    if (mode == SNAP_FULL) {
        Job j = base_job(s, OP_GATHER);
        j.allocs = allocs;
        j.host = dimg;
        j.hash_out = s->d_hash[cur];
        s->h_cb->jobs[0] = j;
        const CombineConsts cc = make_combine_consts(s->C, shg.piece);
        return get_graph(s, from_shadow ? GK_ASYNC_FULL : GK_FULL, cur, [&](cudaStream_t q) {
            cudaError_t e = enqueue_prologue(s, q);
            if (e == cudaSuccess) e = launch_full_meta(allocs, s->desc.size(), s->C, &s->d_cb->cp, q);
            if (e == cudaSuccess && s->n_chunks)
                e = launch_tiles(s->d_cb->jobs, 1, &s->d_cb->cursor[0], cc, shg, &s->d_cb->res, q);
            if (e == cudaSuccess) e = enqueue_epilogue(s, q);
            return e;
        }, out);
    }
    if (!from_shadow && s->n_groups >= 2 && cap >= s->patch_bound) {
        if (fused_ok(s, shh, s->h_cb->fused)) return fused_incremental(s, cur, dimg, cap, shh, out);
        TileShape shp = shh;
        shp.ctas = std::max(1, s->sms - kPipeGatherCtas);
        if (plan_pipeline(s, (uint64_t)shp.ctas * (uint64_t)shp.warps) >= 2)
            return pipelined_incremental(s, cur, dimg, shp, out);
    }
    Job jh = base_job(s, OP_HASH);
    jh.allocs = allocs;
    jh.hash_out = s->d_hash[cur];
    Job jg = base_job(s, OP_GATHER_DIRTY);
    jg.allocs = allocs;
    jg.host = dimg;
    jg.tile_list = s->d_dlist;
    jg.n_tiles_dev = &s->d_cb->res.n_dirty;
    jg.patch_data = s->d_patch_data;
    jg.dstart = s->d_dstart;
    jg.cap_exceeded = &s->d_cb->res.cap_exceeded;
    s->h_cb->jobs[0] = jh;
    s->h_cb->jobs[1] = jg;
    const CombineConsts cch = make_combine_consts(s->C, shh.piece);
    const CombineConsts ccg = make_combine_consts(s->C, shg.piece);
    const uint32_t *curp = s->d_hash[cur], *prevp = s->d_hash[1 - cur];
    return get_graph(s, from_shadow ? GK_ASYNC_INCR : GK_INCR, cur, [&](cudaStream_t q) {
        cudaError_t e = enqueue_prologue(s, q);
        if (e == cudaSuccess && s->n_chunks)
            e = launch_tiles(s->d_cb->jobs, 1, &s->d_cb->cursor[0], cch, shh, &s->d_cb->res, q);
        if (e == cudaSuccess) e = launch_stamp(&s->d_cb->res, TS_HASH_END, q);
        if (e == cudaSuccess)
            e = launch_diff(curp, prevp, s->n_chunks, s->d_blockcnt, s->d_blockoff, s->d_dlist, &s->d_cb->res, q);
        if (e == cudaSuccess)
            e = launch_patch_layout(allocs, s->desc.size(), s->C, s->d_dlist, s->d_patch_rec, s->d_patch_data,
                                    s->d_dstart, &s->d_cb->cp, &s->d_cb->res, q);
        if (e == cudaSuccess)
            e = launch_patch_meta(allocs, s->desc.size(), s->C, curp, s->d_dlist, s->d_patch_rec, s->d_patch_data,
                                  s->d_dstart, &s->d_cb->res, &s->d_cb->cp, q);
        if (e == cudaSuccess) e = launch_stamp(&s->d_cb->res, TS_DIFF_END, q);
        if (e == cudaSuccess && s->n_chunks)
            e = launch_tiles(s->d_cb->jobs + 1, 1, &s->d_cb->cursor[1], ccg, shg, &s->d_cb->res, q);
        if (e == cudaSuccess) e = enqueue_epilogue(s, q);
        return e;
    }, out);
}

// After the device finished a checkpoint graph: write the image header,
// fill the stats and commit the new hash table as the base (Sec. 3.1: only
// a completed checkpoint replaces the base).
int complete_checkpoint(snap_set_s *s, int mode, int cur, uint8_t *host_image, uint64_t *used, snap_stats &st)
{
    const uint64_t gen = s->next_gen;
    if (mode == SNAP_FULL) {
        write_header(host_image, SNAP_IMG_FLAG_DEVICE_STATE, s->C, s->desc.size(), s->total_bytes, gen, 0);
        st.image_bytes = s->full_bytes;
        st.copy_ms = ts_ms(s, TS_BEGIN, TS_COPY_END);
        st.dirty_chunks = s->n_chunks;
    } else {
        if (s->h_res->cap_exceeded) return SNAP_EINVAL;
        write_header(host_image, SNAP_IMG_FLAG_DEVICE_STATE | SNAP_IMG_FLAG_INCREMENTAL, s->C, s->desc.size(),
                     s->total_bytes, gen, s->base_gen);
        st.image_bytes = s->h_res->patch_bytes;
        st.dirty_chunks = s->h_res->n_dirty;
        st.hash_ms = ts_ms(s, TS_BEGIN, TS_HASH_END);
        st.diff_ms = ts_ms(s, TS_HASH_END, TS_DIFF_END);
        st.copy_ms = ts_ms(s, TS_DIFF_END, TS_COPY_END);
        st.dma_copies = s->dma_copies;
    }
    if (used) *used = st.image_bytes;
    s->prev_idx = cur;
    s->has_base = true;
    s->base_gen = gen;
    s->next_gen = gen + 1;
    st.state_bytes = s->total_bytes;
    st.total_chunks = s->n_chunks;
    st.generation = gen;
    return SNAP_OK;
}

}  // namespace snapk

// ===================================================================== ABI
extern "C" {

const char *snap_strerror(int st)
{
    switch (st) {
    case SNAP_OK: return "ok";
    case SNAP_EINVAL: return "invalid argument";
    case SNAP_ENOMEM: return "out of memory";
    case SNAP_ECUDA: return "CUDA error";
    case SNAP_ETIMEDOUT: return "timed out";
    case SNAP_ENOBASE: return "no committed base for an incremental checkpoint";
    case SNAP_EFORMAT: return "malformed image";
    case SNAP_EMISMATCH: return "image does not match the set";
    case SNAP_EBUSY: return "set busy";
    case SNAP_EBUDGET: return "request exceeds the server budgets";
    case SNAP_EIO: return "image file I/O error";
    case SNAP_EPEER: return "the coordinated call failed on another rank";
    default: return "unknown status";
    }
}

int snap_host_alloc(uint64_t bytes, void **out)
{
    if (!out || bytes == 0) return SNAP_EINVAL;
    *out = nullptr;
    if (fault_injected("pinned_alloc")) return SNAP_ENOMEM;
    cudaError_t e = cudaHostAlloc(out, bytes, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return SNAP_ENOMEM;
    }
    pinned_add(*out, bytes);
    return SNAP_OK;
}

int snap_host_free(void *p)
{
    if (!p) return SNAP_OK;
    pinned_remove(p);
    return cuda_status(cudaFreeHost(p));
}

int snap_host_register(void *p, uint64_t bytes)
{
    if (!p || bytes == 0) return SNAP_EINVAL;
    const cudaError_t e = cudaHostRegister(p, bytes, cudaHostRegisterMapped | cudaHostRegisterPortable);
    if (e == cudaSuccess) {
        pinned_add(p, bytes);
        return SNAP_OK;
    }
    cudaGetLastError();
    if (e == cudaErrorHostMemoryAlreadyRegistered || e == cudaErrorInvalidValue) return SNAP_EINVAL;
    return e == cudaErrorMemoryAllocation ? SNAP_ENOMEM : SNAP_ECUDA;
}

int snap_host_unregister(void *p)
{
    if (!p) return SNAP_EINVAL;
    const cudaError_t e = cudaHostUnregister(p);
    if (e == cudaSuccess) {
        pinned_remove(p);
        return SNAP_OK;
    }
    cudaGetLastError();
    return e == cudaErrorHostMemoryNotRegistered || e == cudaErrorInvalidValue ? SNAP_EINVAL : SNAP_ECUDA;
}

int snap_set_create(snap_set *out, const snap_opts *o)
{
    if (!out) return SNAP_EINVAL;
    *out = nullptr;
    snap_opts opt{};
    if (o) opt = *o;
    if (opt.chunk_bytes == 0) opt.chunk_bytes = 65536;
    if (opt.chunk_bytes < 4096 || opt.chunk_bytes % 4096 || opt.chunk_bytes > (16u << 20)) return SNAP_EINVAL;
    if (opt.timeout_ms == 0) opt.timeout_ms = 10000;
    if (opt.ring_bytes == 0) opt.ring_bytes = 4ull << 30;
    if (opt.incr_copy > SNAP_INCR_COPY_DMA) return SNAP_EINVAL;
    int dev = o ? opt.device : -1;
    if (dev < 0) {
        if (cudaGetDevice(&dev) != cudaSuccess) return SNAP_ECUDA;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || dev >= ndev) return SNAP_EINVAL;
    if (cudaSetDevice(dev) != cudaSuccess) return SNAP_ECUDA;
    auto *s = new (std::nothrow) snap_set_s();
    if (!s) return SNAP_ENOMEM;
    s->device = dev;
    s->C = opt.chunk_bytes;
    s->timeout_ms = opt.timeout_ms;
    s->user_stream = static_cast<cudaStream_t>(opt.stream);
    s->opts = opt;
    cudaDeviceProp prop{};
    cudaError_t e = cudaGetDeviceProperties(&prop, dev);
    s->sms = prop.multiProcessorCount;
    std::snprintf(s->gpu_name, sizeof s->gpu_name, "%s", prop.name);
    if (e == cudaSuccess) e = init_tile_kernel();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_quiesce, cudaEventDisableTiming);
    for (int i = 0; i < EV_COUNT && e == cudaSuccess; ++i) e = cudaEventCreate(&s->ev[i]);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_cb, sizeof(CallBlock));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->h_cb, sizeof(CallBlock), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->h_res, sizeof(Result), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        snap_set_destroy(s);
        return cuda_status(e);
    }
    default_shapes(s);
    *out = s;
    return SNAP_OK;
}

int snap_set_destroy(snap_set s)
{
    if (!s) return SNAP_EINVAL;
    cudaSetDevice(s->device);
    if (s->st) cudaStreamSynchronize(s->st);
    free_device(s);
    ring_free(s);
    async_free(s);
    lazy_free(s);
    for (auto &ev : s->ev_pipe)
        if (ev) cudaEventDestroy(ev);
    if (s->st_pipe) cudaStreamDestroy(s->st_pipe);
    if (s->st_meta) cudaStreamDestroy(s->st_meta);
    for (int i = 0; i < kDmaStreams; ++i) {
        if (s->st_dma[i]) {
            cudaStreamSynchronize(s->st_dma[i]);
            cudaStreamDestroy(s->st_dma[i]);
        }
        if (s->ev_dma[i]) cudaEventDestroy(s->ev_dma[i]);
    }
    if (s->ev_graph_end) cudaEventDestroy(s->ev_graph_end);
    cudaFreeHost(s->h_rungrp);
    cudaFree(s->d_cb);
    cudaFreeHost(s->h_cb);
    cudaFreeHost(s->h_res);
    if (s->ev_quiesce) cudaEventDestroy(s->ev_quiesce);
    for (int i = 0; i < EV_COUNT; ++i) if (s->ev[i]) cudaEventDestroy(s->ev[i]);
    if (s->st) cudaStreamDestroy(s->st);
    delete s;
    return SNAP_OK;
}

int snap_register(snap_set s, void *dptr, uint64_t bytes)
{
    if (!s) return SNAP_EINVAL;
    BusyGuard g(s);
    if (!g.ok) return SNAP_EBUSY;
    if (bytes && !dptr) return SNAP_EINVAL;
    if ((uintptr_t)dptr & 15u) return SNAP_EINVAL;
    if (s->allocs.size() >= (size_t)INT32_MAX) return SNAP_EINVAL;
    if (bytes) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, dptr) != cudaSuccess) {
            cudaGetLastError();
            return SNAP_EINVAL;
        }
        if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return SNAP_EINVAL;
        if (at.device != s->device) return SNAP_EINVAL;
    }
    s->allocs.push_back(HostAlloc{dptr, bytes});
    s->layout_dirty = true;
    s->has_base = false;
    return (int)(s->allocs.size() - 1);
}

int snap_set_prepare(snap_set s, int what)
{
    if (!s || (what & ~(SNAP_PREPARE_LAYOUT | SNAP_PREPARE_RING | SNAP_PREPARE_SHADOW))) return SNAP_EINVAL;
    BusyGuard g(s);
    if (!g.ok) return SNAP_EBUSY;
    cudaSetDevice(s->device);
    int rc = build_layout(s);
    if (rc == SNAP_OK && (what & SNAP_PREPARE_RING)) {
        Ring *r = nullptr;
        rc = ring_get(s, &r);
    }
    if (rc == SNAP_OK && (what & SNAP_PREPARE_SHADOW)) rc = async_prepare(s);
    return rc;
}

int snap_image_bytes(snap_set s, int mode, uint64_t *out)
{
    if (!s || !out) return SNAP_EINVAL;
    BusyGuard g(s);
    if (!g.ok) return SNAP_EBUSY;
    cudaSetDevice(s->device);
    const int rc = build_layout(s);
    if (rc) return rc;
    if (mode == SNAP_FULL) *out = s->full_bytes;
    else if (mode == SNAP_INCREMENTAL) *out = s->patch_bound;
    else return SNAP_EINVAL;
    return SNAP_OK;
}

// Copy streams the copy-engine form deals its runs over ($SNAP_DMA_STREAMS,
// default 1).
static int dma_streams()
{
    const char *e = std::getenv("SNAP_DMA_STREAMS");
    const int n = e && *e ? std::atoi(e) : 1;
    return std::max(1, std::min(n, kDmaStreams));
}

// Copy-engine form, host side: while the fused launch runs, take its groups
// in order as the metadata CTA publishes them and hand each dirty run to
// the copy engines (one asynchronous copy each, into the caller's pinned
// image, the runs dealt round-robin over dma_streams() copy streams).
// Each entry is checked against the allocation table and the image extent
// `cap` before its copy is issued (*bad on a failed check: nothing more is
// issued).  A launch that ends without publishing a group sets
// *unpublished (it has normally recorded its error in the result, which
// finish() reports).  On return the library stream is ordered after every
// copy issued, and after them a stamp marks the end of the copy phase.
static int dma_dirty_runs(snap_set_s *s, uint8_t *image, uint64_t cap, double deadline, bool *bad,
                          bool *unpublished)
{
    const FusedIncr &f = s->h_cb->fused;
    const uint64_t nst = (uint64_t)dma_streams();
    *bad = false;
    *unpublished = false;
    cudaError_t e = cudaEventRecord(s->ev_graph_end, s->st);
    if (e != cudaSuccess) return cuda_status(e);
    int rc = SNAP_OK;
    uint64_t copies = 0;
    for (int g = 0; g < f.n_groups && rc == SNAP_OK && !*bad; ++g) {
        volatile RunGroup *p = s->h_rungrp + g;
        unsigned spins = 0;
        while (!p->ready) {
            if (cudaEventQuery(s->ev_graph_end) == cudaSuccess) break;  // the launch has ended
            if (now_ms() > deadline) {
                rc = SNAP_ETIMEDOUT;
                break;
            }
            if (++spins > 64) std::this_thread::yield();
        }
        if (rc != SNAP_OK) break;
        if (!p->ready) {
            *unpublished = true;
            break;
        }
        std::atomic_thread_fence(std::memory_order_acquire);
        const uint64_t b = p->begin, n = p->count;
        if (b > s->runs_cap || n > s->runs_cap - b) {
            *bad = true;
            break;
        }
        for (uint64_t j = b; j < b + n; ++j) {
            const volatile DirtyRun *v = s->h_runs + j;
            const uint64_t k = v->alloc, i = v->chunk, d0 = v->dst0, d1 = v->dst1;
            if (k >= s->desc.size() || d1 <= d0 || d1 > cap || d0 < SNAP_IMG_HEADER_BYTES) {
                *bad = true;
                break;
            }
            const AllocDesc &a = s->desc[k];
            const uint64_t len = d1 - d0;
            if (i >= (a.bytes + s->C - 1) / s->C || len > a.bytes - i * s->C) {
                *bad = true;
                break;
            }
            e = cudaMemcpyAsync(image + d0, reinterpret_cast<const uint8_t *>(a.ptr) + i * s->C, len,
                                cudaMemcpyDeviceToHost, s->st_dma[copies % nst]);
            if (e != cudaSuccess) {
                rc = cuda_status(e);
                break;
            }
            ++copies;
        }
    }
    s->dma_copies = copies;
    e = cudaSuccess;
    for (uint64_t q = 0; q < nst && e == cudaSuccess; ++q) {
        e = cudaEventRecord(s->ev_dma[q], s->st_dma[q]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->st, s->ev_dma[q], 0);
    }
    if (e == cudaSuccess) e = launch_stamp(&s->d_cb->res, TS_COPY_END, s->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&s->h_res->ts[TS_COPY_END], &s->d_cb->res.ts[TS_COPY_END], sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s->st);
    ++s->call_kernels;
    if (rc == SNAP_OK && e != cudaSuccess) rc = cuda_status(e);
    return rc;
}

// Run a checkpoint's graph into the caller's mapped image (host address
// `image`) and wait for it; the copy-engine form's copies are issued from
// this thread while the launch runs.
static int run_checkpoint(snap_set_s *s, GraphEntry *ge, uint8_t *image, uint64_t cap, double deadline)
{
    s->call_kernels = ge->kernels;
    int rc = cuda_status(cudaGraphLaunch(ge->exec, s->st));
    if (rc) return rc;
    bool bad = false, unpublished = false;
    int rc_dma = SNAP_OK;
    // the copies stay inside the pinned range the direct path was chosen for
    if (s->dma_call)
        rc_dma = dma_dirty_runs(s, image, image_extent(s, SNAP_INCREMENTAL, cap), deadline, &bad, &unpublished);
    rc = finish(s, deadline);
    // a bad run entry, or a launch that ended without publishing every group
    // and without recording why: the patch is incomplete
    if (bad || (unpublished && rc == SNAP_OK)) {
        s->device_err |= ERR_BAD_TILE;
        if (rc == SNAP_OK) rc = SNAP_ECUDA;
    }
    return rc != SNAP_OK ? rc : rc_dma;
}

int snap_checkpoint(snap_set s, void *host_image, uint64_t cap, int mode, uint64_t *used)
{
    const double t0 = now_ms();
    if (!s || !host_image || ((uintptr_t)host_image & 15u)) return SNAP_EINVAL;
    if (mode != SNAP_FULL && mode != SNAP_INCREMENTAL) return SNAP_EINVAL;
    BusyGuard g(s);
    if (!g.ok) return SNAP_EBUSY;
    cudaSetDevice(s->device);
    const double deadline = t0 + s->timeout_ms;
    int rc = settle(s, deadline);
    if (rc) return rc;
    rc = build_layout(s);
    if (rc) return rc;
    if (mode == SNAP_INCREMENTAL && !s->has_base) return SNAP_ENOBASE;
    if (mode == SNAP_FULL && cap < s->full_bytes) return SNAP_EINVAL;
    if (mode == SNAP_INCREMENTAL && cap < SNAP_IMG_HEADER_BYTES) return SNAP_EINVAL;

    uint8_t *dimg = mapped_image_ptr(host_image, image_extent(s, mode, cap));
    rc = quiesce(s, deadline);
    if (rc) return rc;
    const double tq = now_ms();
    if (!dimg) {
        ImageIO io;
        io.mem = static_cast<uint8_t *>(host_image);
        return ring_checkpoint(s, io, cap, mode, used, t0, tq, deadline);
    }

    const int cur = 1 - s->prev_idx;
    GraphEntry *ge = nullptr;
    rc = checkpoint_graph(s, mode, cur, dimg, cap, false, &ge);
    if (rc) return rc;
    rc = run_checkpoint(s, ge, static_cast<uint8_t *>(host_image), cap, deadline);
    if (rc) return rc;
    snap_stats st{};
    rc = complete_checkpoint(s, mode, cur, static_cast<uint8_t *>(host_image), used, st);
    if (rc) return rc;
    st.quiesce_ms = tq - t0;
    st.kernel_launches = s->call_kernels;
    st.total_ms = now_ms() - t0;
    st.frozen_ms = st.total_ms;
    s->last = st;
    return SNAP_OK;
}

// One rank of a coordinated checkpoint: the lock / run / commit / abort
// steps of snap_coordinate over the synchronous checkpoint path.  The run
// commits like snap_checkpoint; abort puts the previous base back.
struct CoordCkpt {
    snap_set_s *s;
    void *image;
    uint64_t cap;
    int mode;
    uint64_t *used;
    snap_agree_fn agree;
    void *agree_ctx;
    bool busy = false;
    double t0 = 0, tq = 0, deadline = 0;
    uint8_t *dimg = nullptr;
    int prev_idx = 0;
    bool has_base = false;
    uint64_t base_gen = 0, next_gen = 0;
};

static int coord_lock(void *p)
{
    CoordCkpt &c = *static_cast<CoordCkpt *>(p);
    snap_set_s *s = c.s;
    if (!s || !c.image || ((uintptr_t)c.image & 15u)) return SNAP_EINVAL;
    if (c.mode != SNAP_FULL && c.mode != SNAP_INCREMENTAL) return SNAP_EINVAL;
    if (s->busy.exchange(true)) return SNAP_EBUSY;
    c.busy = true;
    cudaSetDevice(s->device);
    c.deadline = c.t0 + s->timeout_ms;
    int rc = settle(s, c.deadline);
    if (rc == SNAP_OK) rc = build_layout(s);
    if (rc) return rc;
    if (c.mode == SNAP_INCREMENTAL && !s->has_base) return SNAP_ENOBASE;
    if (c.mode == SNAP_FULL && c.cap < s->full_bytes) return SNAP_EINVAL;
    if (c.mode == SNAP_INCREMENTAL && c.cap < SNAP_IMG_HEADER_BYTES) return SNAP_EINVAL;
    c.dimg = mapped_image_ptr(c.image, image_extent(s, c.mode, c.cap));
    rc = quiesce(s, c.deadline);
    c.tq = now_ms();
    return rc;
}

static int coord_run(void *p)
{
    CoordCkpt &c = *static_cast<CoordCkpt *>(p);
    snap_set_s *s = c.s;
    c.prev_idx = s->prev_idx;
    c.has_base = s->has_base;
    c.base_gen = s->base_gen;
    c.next_gen = s->next_gen;
    if (!c.dimg) {
        ImageIO io;
        io.mem = static_cast<uint8_t *>(c.image);
        return ring_checkpoint(s, io, c.cap, c.mode, c.used, c.t0, c.tq, c.deadline);
    }
    const int cur = 1 - s->prev_idx;
    GraphEntry *ge = nullptr;
    int rc = checkpoint_graph(s, c.mode, cur, c.dimg, c.cap, false, &ge);
    if (rc) return rc;
    rc = run_checkpoint(s, ge, static_cast<uint8_t *>(c.image), c.cap, c.deadline);
    if (rc) return rc;
    snap_stats st{};
    rc = complete_checkpoint(s, c.mode, cur, static_cast<uint8_t *>(c.image), c.used, st);
    if (rc) return rc;
    st.quiesce_ms = c.tq - c.t0;
    st.kernel_launches = s->call_kernels;
    st.total_ms = now_ms() - c.t0;
    st.frozen_ms = st.total_ms;
    s->last = st;
    return SNAP_OK;
}

static void coord_abort(void *p)
{
    CoordCkpt &c = *static_cast<CoordCkpt *>(p);
    c.s->prev_idx = c.prev_idx;
    c.s->has_base = c.has_base;
    c.s->base_gen = c.base_gen;
    c.s->next_gen = c.next_gen;
}

static int coord_agree(void *p, int phase, int status)
{
    CoordCkpt &c = *static_cast<CoordCkpt *>(p);
    return c.agree(c.agree_ctx, phase, status);
}

int snap_checkpoint_coordinated(snap_set s, void *host_image, uint64_t cap, int mode, uint64_t *used,
                                snap_agree_fn agree, void *agree_ctx)
{
    if (!s || !agree) return SNAP_EINVAL;
    CoordCkpt c{s, host_image, cap, mode, used, agree, agree_ctx};
    c.t0 = now_ms();
    snap_coord_ops ops{};
    ops.lock = coord_lock;
    ops.run = coord_run;
    ops.abort = coord_abort;
    ops.agree = coord_agree;
    const int rc = coordinate(ops, &c);
    if (c.busy) s->busy.store(false);
    return rc;
}

}  // extern "C"

namespace snapk {

// The lock of a restore: validate the image against the set (header, every
// record, the hashes into the stage) and quiesce the caller's stream.
static int restore_lock(snap_set_s *s, const uint8_t *img, uint64_t bytes, ImageHeader &h, double deadline)
{
    int rc = settle(s, deadline);
    if (rc) return rc;
    rc = build_layout(s);
    if (rc) return rc;
    rc = parse_header(img, bytes, &h);
    if (rc) return rc;
    if (h.flags & SNAP_IMG_FLAG_INCREMENTAL) return SNAP_EFORMAT;  // merge patches first
    if (bytes < s->full_bytes && h.n_allocs == s->desc.size() && h.chunk_bytes == s->C && h.total == s->total_bytes)
        return SNAP_EFORMAT;
    rc = walk_records(s, img, bytes, h, s->h_hash_stage);
    if (rc) return rc;
    return quiesce(s, deadline);
}

// The restore itself, after restore_lock; commits the image's hashes and
// generation as the base.
static int restore_run(snap_set_s *s, const uint8_t *img, uint64_t bytes, const ImageHeader &h, double t0, double tq,
                       double deadline)
{
    uint8_t *dimg = mapped_image_ptr(img, bytes);
    if (!dimg) {
        ImageIO io;
        io.mem = const_cast<uint8_t *>(img);  // read only: restore copies image -> ring
        return ring_restore(s, io, h, t0, tq, deadline);
    }
    const int cur = 1 - s->prev_idx;
    reset_call(s, dimg, bytes);
    Job j = base_job(s, OP_SCATTER);
    j.host = dimg;
    s->h_cb->jobs[0] = j;
    const TileShape sh = s->shape[SHAPE_SCATTER];
    const CombineConsts cc = make_combine_consts(s->C, sh.piece);
    int rc = run_graph(s, GK_RESTORE, cur, [&](cudaStream_t q) {
        cudaError_t e = enqueue_prologue(s, q);
        if (e == cudaSuccess && s->n_chunks)
            e = cudaMemcpyAsync(s->d_hash[cur], s->h_hash_stage, s->n_chunks * 4, cudaMemcpyHostToDevice, q);
        if (e == cudaSuccess && s->n_chunks)
            e = launch_tiles(s->d_cb->jobs, 1, &s->d_cb->cursor[0], cc, sh, &s->d_cb->res, q);
        if (e == cudaSuccess) e = enqueue_epilogue(s, q);
        return e;
    });
    if (rc == SNAP_OK) rc = finish(s, deadline);
    if (rc) return rc;
    s->prev_idx = cur;
    s->has_base = true;
    s->base_gen = h.generation;
    s->next_gen = h.generation + 1;
    snap_stats st{};
    st.state_bytes = s->total_bytes;
    st.image_bytes = s->full_bytes;
    st.total_chunks = s->n_chunks;
    st.generation = h.generation;
    st.quiesce_ms = tq - t0;
    st.copy_ms = ts_ms(s, TS_BEGIN, TS_COPY_END);
    st.kernel_launches = s->call_kernels;
    st.total_ms = now_ms() - t0;
    st.frozen_ms = st.total_ms;
    s->last = st;
    return SNAP_OK;
}

// One rank of a coordinated restore (snap_coordinate's steps).
struct CoordRestore {
    snap_set_s *s;
    const uint8_t *img;
    uint64_t bytes;
    snap_agree_fn agree;
    void *agree_ctx;
    bool busy = false;
    ImageHeader h{};
    double t0 = 0, tq = 0, deadline = 0;
    int prev_idx = 0;
    bool has_base = false;
    uint64_t base_gen = 0, next_gen = 0;
};

static int coord_restore_lock(void *p)
{
    CoordRestore &c = *static_cast<CoordRestore *>(p);
    if (!c.s || !c.img || ((uintptr_t)c.img & 15u)) return SNAP_EINVAL;
    if (c.s->busy.exchange(true)) return SNAP_EBUSY;
    c.busy = true;
    cudaSetDevice(c.s->device);
    c.deadline = c.t0 + c.s->timeout_ms;
    const int rc = restore_lock(c.s, c.img, c.bytes, c.h, c.deadline);
    c.tq = now_ms();
    return rc;
}

static int coord_restore_run(void *p)
{
    CoordRestore &c = *static_cast<CoordRestore *>(p);
    c.prev_idx = c.s->prev_idx;
    c.has_base = c.s->has_base;
    c.base_gen = c.s->base_gen;
    c.next_gen = c.s->next_gen;
    return restore_run(c.s, c.img, c.bytes, c.h, c.t0, c.tq, c.deadline);
}

static void coord_restore_abort(void *p)
{
    CoordRestore &c = *static_cast<CoordRestore *>(p);
    c.s->prev_idx = c.prev_idx;
    c.s->has_base = c.has_base;
    c.s->base_gen = c.base_gen;
    c.s->next_gen = c.next_gen;
}

static int coord_restore_agree(void *p, int phase, int status)
{
    CoordRestore &c = *static_cast<CoordRestore *>(p);
    return c.agree(c.agree_ctx, phase, status);
}

}  // namespace snapk

extern "C" {

int snap_restore(const void *host_image, uint64_t bytes, snap_set s)
{
    const double t0 = now_ms();
    if (!s || !host_image || ((uintptr_t)host_image & 15u)) return SNAP_EINVAL;
    BusyGuard g(s);
    if (!g.ok) return SNAP_EBUSY;
    cudaSetDevice(s->device);
    const double deadline = t0 + s->timeout_ms;
    const uint8_t *img = static_cast<const uint8_t *>(host_image);
    ImageHeader h{};
    const int rc = restore_lock(s, img, bytes, h, deadline);
    if (rc) return rc;
    return restore_run(s, img, bytes, h, t0, now_ms(), deadline);
}

int snap_restore_coordinated(const void *host_image, uint64_t bytes, snap_set s, snap_agree_fn agree,
                             void *agree_ctx)
{
    if (!s || !agree) return SNAP_EINVAL;
    CoordRestore c{s, static_cast<const uint8_t *>(host_image), bytes, agree, agree_ctx};
    c.t0 = now_ms();
    snap_coord_ops ops{};
    ops.lock = coord_restore_lock;
    ops.run = coord_restore_run;
    ops.abort = coord_restore_abort;
    ops.agree = coord_restore_agree;
    const int rc = coordinate(ops, &c);
    if (c.busy) s->busy.store(false);
    return rc;
}

int snap_verify(const void *host_image, uint64_t bytes, snap_set s, uint64_t *n_mismatch)
{
    const double t0 = now_ms();
    if (!s || !host_image || !n_mismatch) return SNAP_EINVAL;
    BusyGuard g(s);
    if (!g.ok) return SNAP_EBUSY;
    cudaSetDevice(s->device);
    const double deadline = t0 + s->timeout_ms;
    int rc = settle(s, deadline);
    if (rc) return rc;
    rc = build_layout(s);
    if (rc) return rc;
    const uint8_t *img = static_cast<const uint8_t *>(host_image);
    ImageHeader h{};
    rc = parse_header(img, bytes, &h);
    if (rc) return rc;
    rc = walk_records(s, img, bytes, h, s->h_hash_stage);
    if (rc) return rc;
    rc = quiesce(s, deadline);
    if (rc) return rc;
    const double tq = now_ms();
    reset_call(s, nullptr, 0);
    Job j = base_job(s, OP_VERIFY);
    j.hash_cmp = s->d_cmp;
    s->h_cb->jobs[0] = j;
    const TileShape sh = s->shape[SHAPE_HASH];
    const CombineConsts cc = make_combine_consts(s->C, sh.piece);
    rc = run_graph(s, GK_VERIFY, 0, [&](cudaStream_t q) {
        cudaError_t e = enqueue_prologue(s, q);
        if (e == cudaSuccess && s->n_chunks)
            e = cudaMemcpyAsync(s->d_cmp, s->h_hash_stage, s->n_chunks * 4, cudaMemcpyHostToDevice, q);
        if (e == cudaSuccess && s->n_chunks)
            e = launch_tiles(s->d_cb->jobs, 1, &s->d_cb->cursor[0], cc, sh, &s->d_cb->res, q);
        if (e == cudaSuccess) e = enqueue_epilogue(s, q);
        return e;
    });
    if (rc == SNAP_OK) rc = finish(s, deadline);
    if (rc) return rc;
    *n_mismatch = s->h_res->mismatches;
    snap_stats st{};
    st.state_bytes = s->total_bytes;
    st.total_chunks = s->n_chunks;
    st.mismatches = s->h_res->mismatches;
    st.generation = h.generation;
    st.quiesce_ms = tq - t0;
    st.hash_ms = ts_ms(s, TS_BEGIN, TS_COPY_END);
    st.kernel_launches = s->call_kernels;
    st.total_ms = now_ms() - t0;
    st.frozen_ms = st.total_ms;
    s->last = st;
    return SNAP_OK;
}

int snap_committed_hashes(snap_set s, uint32_t *out, uint64_t n, uint64_t *generation)
{
    if (!s || (!out && n)) return SNAP_EINVAL;
    BusyGuard g(s);
    if (!g.ok) return SNAP_EBUSY;
    cudaSetDevice(s->device);
    if (!s->has_base || s->layout_dirty) return SNAP_ENOBASE;
    if (n < s->n_chunks) return SNAP_EINVAL;
    if (s->n_chunks) {
        cudaError_t e = cudaMemcpy(out, s->d_hash[s->prev_idx], s->n_chunks * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (generation) *generation = s->base_gen;
    return SNAP_OK;
}

int snap_last_stats(snap_set s, snap_stats *out)
{
    if (!s || !out) return SNAP_EINVAL;
    *out = s->last;
    out->device_errors = s->device_err;
    return SNAP_OK;
}

int snap_apply_patch(void *base_image, uint64_t base_bytes, const void *patch, uint64_t patch_bytes)
{
    return apply_patch_host(static_cast<uint8_t *>(base_image), base_bytes, static_cast<const uint8_t *>(patch),
                            patch_bytes);
}

// ------------------------------------------------------------- plain form
int snap_plain_checkpoint(snap_set s, void *host_image, uint64_t cap)
{
    const double t0 = now_ms();
    if (!s || !host_image) return SNAP_EINVAL;
    BusyGuard g(s);
    if (!g.ok) return SNAP_EBUSY;
    cudaSetDevice(s->device);
    const double deadline = t0 + s->timeout_ms;
    int rc = settle(s, deadline);
    if (rc) return rc;
    rc = build_layout(s);
    if (rc) return rc;
    if (cap < s->full_bytes) return SNAP_EINVAL;
    rc = quiesce(s, deadline);
    if (rc) return rc;
    uint8_t *img = static_cast<uint8_t *>(host_image);
    cudaError_t e = cudaEventRecord(s->ev[EV_BEGIN], s->st);
    for (size_t k = 0; k < s->desc.size() && e == cudaSuccess; ++k)
        if (s->desc[k].bytes)
            e = cudaMemcpyAsync(img + s->desc[k].data_off, s->allocs[k].ptr, s->desc[k].bytes, cudaMemcpyDeviceToHost,
                                s->st);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev[EV_COPY_END], s->st);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaEventRecord(s->ev[EV_END], s->st);
    if (e != cudaSuccess) return cuda_status(e);
    rc = wait_event(s->ev[EV_END], deadline);
    if (rc == SNAP_ETIMEDOUT) s->in_flight = true;
    if (rc) return rc;
    snap_stats st{};
    st.state_bytes = s->total_bytes;
    st.copy_ms = ev_ms(s, EV_BEGIN, EV_COPY_END);
    st.total_ms = now_ms() - t0;
    st.frozen_ms = st.total_ms;
    s->last = st;
    return SNAP_OK;
}

int snap_plain_restore(const void *host_image, uint64_t bytes, snap_set s)
{
    const double t0 = now_ms();
    if (!s || !host_image) return SNAP_EINVAL;
    BusyGuard g(s);
    if (!g.ok) return SNAP_EBUSY;
    cudaSetDevice(s->device);
    const double deadline = t0 + s->timeout_ms;
    int rc = settle(s, deadline);
    if (rc) return rc;
    rc = build_layout(s);
    if (rc) return rc;
    if (bytes < s->full_bytes) return SNAP_EINVAL;
    rc = quiesce(s, deadline);
    if (rc) return rc;
    const uint8_t *img = static_cast<const uint8_t *>(host_image);
    cudaError_t e = cudaEventRecord(s->ev[EV_BEGIN], s->st);
    for (size_t k = 0; k < s->desc.size() && e == cudaSuccess; ++k)
        if (s->desc[k].bytes)
            e = cudaMemcpyAsync(s->allocs[k].ptr, img + s->desc[k].data_off, s->desc[k].bytes, cudaMemcpyHostToDevice,
                                s->st);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev[EV_COPY_END], s->st);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev[EV_END], s->st);
    if (e != cudaSuccess) return cuda_status(e);
    rc = wait_event(s->ev[EV_END], deadline);
    if (rc == SNAP_ETIMEDOUT) s->in_flight = true;
    if (rc) return rc;
    snap_stats st{};
    st.state_bytes = s->total_bytes;
    st.copy_ms = ev_ms(s, EV_BEGIN, EV_COPY_END);
    st.total_ms = now_ms() - t0;
    st.frozen_ms = st.total_ms;
    s->last = st;
    return SNAP_OK;
}

}  // extern "C"
