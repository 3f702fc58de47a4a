// Internal structures shared by the kernels (kernels.cu, meta_kernels.cu)
// and the host runtime (runtime.cu).  Not part of the public ABI.
#pragma once
#include <stdint.h>
#include <stddef.h>
#include <cuda_runtime.h>

namespace snapk {

// One registered allocation, as the kernels see it (device array).
struct AllocDesc {
    uint64_t ptr;        // device address (16-byte aligned)
    uint64_t bytes;      // size in bytes
    uint64_t chunk0;     // global index of its first chunk
    uint64_t rec_off;    // full image: offset of its 32-byte record
    uint64_t data_off;   // full image: offset of its data (4 KiB aligned)
    uint64_t state_off;  // offset in the packed concatenation of all allocations
                         // (each allocation starts on a 256-byte boundary)
    uint64_t tmap;       // device address of its three TMA tensor maps (pieces of
                         // 32, 64, 128 bytes; kTmapBytes each) for the hash
                         // staging, or 0: stage with cp.async instead
};

// A 2D view of an allocation for the hash staging: rows of C/32 bytes (one
// lane segment each), box = piece bytes x 32 rows, so stage k of full chunk
// i is the box at (k * piece, 32 * i).  The box lands in shared memory with
// the hardware swizzle that equals the stage layout's XOR swizzle.
constexpr uint32_t kTmapBytes = 128;
constexpr int kTmapPieces = 3;  // 32, 64, 128

// What a job does with each of its chunk tiles.
enum JobOp : uint32_t {
    OP_HASH = 0,          // CRC every chunk -> hash_out
    OP_GATHER = 1,        // CRC + copy device -> host, hashes -> hash_out (and image)
    OP_VERIFY = 2,        // CRC, compare with hash_cmp
    OP_GATHER_DIRTY = 3,  // copy dirty chunks device -> patch data slots
    OP_SCATTER = 4,       // copy host -> device
};

// Where a job's host bytes live.
enum JobLayout : uint32_t {
    LAYOUT_IMAGE = 0,   // full-image layout (data at AllocDesc.data_off)
    LAYOUT_PACKED = 1,  // packed window: host = base + state_off + i*C - window_off
};

// Device-side outcome of a launch sequence.
struct Result {
    unsigned long long err;          // ResultErr bits set by a kernel that gave up
    unsigned long long mismatches;   // verify
    unsigned long long first_bad;    // verify: smallest mismatching chunk (or ~0)
    unsigned long long n_dirty;      // incremental: dirty chunk count
    unsigned long long patch_bytes;  // incremental: patch size
    unsigned long long cap_exceeded; // incremental: patch larger than the image capacity
    unsigned long long pad[2];
    unsigned long long ts[8];        // %globaltimer stamps between the phases (ns)
};

enum StampId { TS_BEGIN = 0, TS_HASH_END, TS_DIFF_END, TS_COPY_END };

enum ResultErr : unsigned long long {
    ERR_WAIT_TIMEOUT = 1ull,   // an mbarrier wait passed its deadline
    ERR_BAD_TILE = 2ull,       // a tile resolved outside its allocation table
    ERR_SMEM_BASE = 4ull,      // dynamic shared memory not where the CRC lookups expect it
};

struct FusedIncr;

// One job: a set of chunk tiles with one operation.
struct Job {
    const AllocDesc *allocs;
    uint64_t n_allocs;
    uint64_t chunk_bytes;
    uint64_t tile_begin;           // identity tiles: first global chunk
    uint64_t n_tiles;              // identity tiles: count
    const uint32_t *tile_list;     // list tiles (ascending global chunks), or null
    const unsigned long long *n_tiles_dev;  // list tiles: count on the device
    const unsigned long long *tile_off_dev; // list tiles: first list entry, on the device (or null: 0)
    uint8_t *host;                 // device-visible address of the host image / window
    uint64_t window_off;           // LAYOUT_PACKED
    uint32_t op;                   // JobOp
    uint32_t layout;               // JobLayout
    uint32_t *hash_out;            // device hash table (global chunk index), or null
    const uint32_t *hash_cmp;      // OP_VERIFY: expected hashes (global chunk index)
    const uint64_t *patch_data;    // OP_GATHER_DIRTY: per-allocation data offset in the patch
    const uint64_t *dstart;        // OP_GATHER_DIRTY: per-allocation first dirty rank
    const unsigned long long *cap_exceeded;  // OP_GATHER_DIRTY: skip if set
    Result *res;                   // per-job counters (verify)
    uint64_t test_stall;           // test hook, 0 in every normal call: the warp that takes
                                   // tile test_stall - 1 waits on a stage no copy fills, so
                                   // its bounded wait runs out (ERR_WAIT_TIMEOUT)
    FusedIncr *fused;              // OP_HASH of a fused incremental checkpoint, else null
};

// A fused incremental checkpoint: one cooperative launch of the tile kernel
// whose CTAs take three roles.  CTAs [0, n_hash_ctas) hash every chunk in
// ascending order (the job's tiles) and count each completed chunk against
// its group; CTA n_hash_ctas waits for each group in turn and diffs it
// (ascending dirty list), lays out its allocations' patch records and
// writes their metadata into the patch; the remaining CTAs wait for each
// group's metadata and copy its dirty chunks into their patch slots (or,
// with `dma`, there are none: the metadata CTA lists the group's dirty runs
// for the copy engines instead, see DirtyRun).  A
// group is a run of whole allocations, chunks [gch[g], gch[g+1]) and
// allocations [gal[g], gal[g+1]).  Every wait is bounded (ERR_WAIT_TIMEOUT);
// the cooperative launch keeps every CTA resident, so no role waits on a CTA
// that is not running.
constexpr int kFusedMaxGroups = 64;

// Copy-engine form of the fused incremental's dirty copy: the metadata CTA
// lists each group's dirty runs (maximal ranges of consecutive dirty chunks
// of one allocation; their patch slots are contiguous) in pinned, mapped
// host memory and publishes the group; a host thread hands every run to the
// copy engines (one asynchronous device-to-host copy each) while the SMs
// hash the later groups.  Host and device agree on these two layouts.
struct DirtyRun {
    uint64_t alloc;  // allocation index
    uint64_t chunk;  // first chunk of the run, within the allocation
    uint64_t dst0;   // patch offset of the run's first byte
    uint64_t dst1;   // patch offset one past its last data byte
};
struct RunGroup {
    unsigned long long begin, count;  // the group's runs: entries [begin, begin + count)
    unsigned long long ready;         // written last, 1 once begin and count and the entries are
    unsigned long long pad;
};

struct FusedIncr {
    const uint32_t *prev;      // committed hashes
    uint32_t *dlist;           // ascending dirty chunk list
    uint64_t *patch_rec, *patch_data, *dstart;
    uint8_t *host;             // device-visible address of the patch image
    uint64_t cap;              // its capacity
    int n_groups, n_hash_ctas;
    int dma;                   // 1: no gather CTAs; runs are listed for the copy engines
    int pad_;
    DirtyRun *runs;            // dma: device-visible address of the run table (mapped host)
    RunGroup *pub;             // dma: device-visible address of the per-group records (mapped host)
    uint64_t runs_cap;         // dma: entries of the run table
    uint64_t gch[kFusedMaxGroups + 1];
    uint64_t gal[kFusedMaxGroups + 1];
    // counters and results, zero at the start of every call
    unsigned long long grp_done[kFusedMaxGroups];    // chunks hashed per group
    unsigned long long meta_ready[kFusedMaxGroups];  // 1 once a group's metadata is written
    unsigned long long gcur[kFusedMaxGroups];        // gather cursor per group
    unsigned long long gbeg[kFusedMaxGroups], gcnt[kFusedMaxGroups];  // its dirty-list range
};

constexpr int kMaxJobs = 64;
constexpr int kMaxWarps = 16;      // general tile kernel
constexpr int kMaxHashWarps = 32;  // hash/verify-only tile kernel

// Launch shape of the persistent tile kernel.
struct TileShape {
    int warps;        // warps per CTA
    int stages;       // staging buffers per warp
    int piece;        // bytes per segment per stage: 32, 64, 128 or 256
    int ctas;         // grid size (persistent CTAs)
    int chains = 1;   // hashing: independent CRC chains per lane (1 or 2)
    int tma = 0;      // hashing: 1 = stage full chunks with 2D TMA tensor copies where
                      // the allocation has tensor maps, 0 = per-lane cp.async (the
                      // autotuner picks per set: within 3 % of each other at the
                      // best shapes, TMA ahead at large chunks)
};

// Combine constants, computed on the host for a chunk size and piece size.
struct CombineConsts {
    uint32_t kseg[32];    // x^(8*(C - (l+1)*C/32)): segmented lane l of a full chunk
    uint32_t kseg2[64];   // x^(8*(C - (v+1)*C/64)): segment v of 64 (two chains per lane)
    uint32_t kint[32];    // x^(8*(31-l)*P): interleaved lane l, end of a full chunk
    uint32_t kgap;        // x^(8*31*P): interleaved gap between a lane's pieces
    uint32_t pad[3];
};

// Per-call values read by the metadata kernels from device memory, so that
// one captured graph serves every call (the host rewrites them per call).
struct CallParams {
    uint8_t *image;  // device-visible address of the host image
    uint64_t cap;    // its capacity in bytes
};

size_t tile_smem_bytes(const TileShape &sh);
constexpr size_t kMaxSmem = 232448;  // 227 KiB opt-in per CTA

// Kernel launchers.  All run on `st`.
// `overlap_prev`: launched with programmatic stream serialization, so its
// CTAs may start while the previous tile kernel on `st` finishes its last
// tiles; only for a launch that reads nothing the previous one writes.
cudaError_t launch_tiles(const Job *jobs_dev, int n_jobs, unsigned long long *cursor,
                         const CombineConsts &cc, const TileShape &sh, Result *kres,
                         cudaStream_t st, bool overlap_prev = false);
// The fused incremental checkpoint: one cooperative launch of `grid` CTAs
// of shape `sh` (hash-role CTAs = fused->n_hash_ctas of them), job = its
// OP_HASH job (with `fused` set).  fused_incr_fits: whether the device can
// keep `grid` CTAs of that shape resident at once.
cudaError_t launch_fused_incr(const Job *job_dev, unsigned long long *cursor, const CombineConsts &cc,
                              const TileShape &sh, int grid, Result *kres, cudaStream_t st);
bool fused_incr_fits(const TileShape &sh, int grid, int device);

// Two job groups with their own cursors: jobs [0, n_jobs_a) (device to
// host) and [n_jobs_a, n_jobs) (host to device), worked on concurrently.
cudaError_t launch_tiles2(const Job *jobs_dev, int n_jobs, int n_jobs_a, unsigned long long *cursor_a,
                          unsigned long long *cursor_b, const CombineConsts &cc, const TileShape &sh, Result *kres,
                          cudaStream_t st, bool overlap_prev = false);
CombineConsts make_combine_consts(uint64_t chunk_bytes, int piece);
cudaError_t init_tile_kernel();
cudaError_t launch_full_meta(const AllocDesc *allocs, uint64_t n_allocs, uint64_t chunk_bytes,
                             const CallParams *cp, cudaStream_t st);
cudaError_t launch_diff(const uint32_t *cur, const uint32_t *prev, uint64_t n_chunks,
                        unsigned int *blockcnt, unsigned long long *blockoff, uint32_t *dlist,
                        Result *res, cudaStream_t st);
cudaError_t launch_patch_layout(const AllocDesc *allocs, uint64_t n_allocs, uint64_t chunk_bytes,
                                const uint32_t *dlist, uint64_t *patch_rec, uint64_t *patch_data,
                                uint64_t *dstart, const CallParams *cp, Result *res, cudaStream_t st);
// Range forms for a checkpoint processed in groups of allocations: diff the
// chunks [c0, c0 + n) after the `run` entries already listed (gbeg / gcnt
// get the range's first position and count); lay out and write the records
// of allocations [a0, a0 + na), continuing the patch offset in run_off.
cudaError_t launch_diff_range(const uint32_t *cur, const uint32_t *prev, uint64_t c0, uint64_t n,
                              unsigned int *blockcnt, unsigned long long *blockoff, uint32_t *dlist,
                              unsigned long long *run, unsigned long long *gbeg, unsigned long long *gcnt,
                              cudaStream_t st);
cudaError_t launch_patch_layout_range(const AllocDesc *allocs, uint64_t a0, uint64_t na, uint64_t chunk_bytes,
                                      const uint32_t *dlist, uint64_t *patch_rec, uint64_t *patch_data,
                                      uint64_t *dstart, const CallParams *cp, Result *res,
                                      unsigned long long *run_off, cudaStream_t st);
cudaError_t launch_patch_meta_range(const AllocDesc *allocs, uint64_t a0, uint64_t na, uint64_t chunk_bytes,
                                    const uint32_t *cur, const uint32_t *dlist, const uint64_t *patch_rec,
                                    const uint64_t *patch_data, const uint64_t *dstart, const Result *res,
                                    const CallParams *cp, cudaStream_t st);
cudaError_t launch_patch_meta(const AllocDesc *allocs, uint64_t n_allocs, uint64_t chunk_bytes,
                              const uint32_t *cur, const uint32_t *dlist, const uint64_t *patch_rec,
                              const uint64_t *patch_data, const uint64_t *dstart,
                              const Result *res, const CallParams *cp, cudaStream_t st);

// Device-to-device copy of every allocation into the packed shadow buffer
// (the cut of an asynchronous checkpoint).
cudaError_t launch_shadow_copy(const AllocDesc *allocs, uint64_t n_allocs, uint64_t chunk_bytes, uint64_t n_chunks,
                               uint8_t *shadow, int sms, cudaStream_t st);

// One-thread kernel recording the device clock into res->ts[idx]; stream
// order makes it a phase boundary inside a captured graph.
cudaError_t launch_stamp(Result *res, int idx, cudaStream_t st);

constexpr int kDiffBlock = 1024;

}  // namespace snapk
