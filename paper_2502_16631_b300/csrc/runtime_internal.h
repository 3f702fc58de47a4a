// Host-side state of libsnap (runtime.cu, ring.cu, tune.cu, server.cu).
#pragma once
#include "snap.h"
#include "snap_internal.h"

#include <atomic>
#include <functional>
#include <vector>

namespace snapk {

struct HostAlloc {
    void *ptr;
    uint64_t bytes;
};

struct ImageHeader {
    uint32_t flags;
    uint64_t chunk_bytes, n_allocs, total, generation, parent;
};

// A pipelined incremental checkpoint aims at about this many stages (hash
// launches of equal whole waves of tiles; the allocations each completes),
// and has at most kMaxPipe.
constexpr int kMaxGroups = 16;
constexpr int kMaxPipe = 2 * kMaxGroups;
// CTAs that gather dirty chunks while the other SMs hash the next group: the
// device-to-host link saturates with 8 gather CTAs on B300.
constexpr int kPipeGatherCtas = 8;
// Copy streams of the fused incremental's copy-engine form: at most this
// many, one by default ($SNAP_DMA_STREAMS): runs dealt over four streams made
// the 1 % incremental of a 20 GiB state 19 % slower on B300, not faster.
constexpr int kDmaStreams = 4;

// Everything one launch sequence needs that changes from call to call; the
// host fills a pinned copy and the captured graph's first node copies it in.
struct CallBlock {
    unsigned long long cursor[2 * kMaxPipe + 2];  // tile cursors of the sequence's launches
    unsigned long long gbeg[kMaxPipe];             // pipelined incremental: each group's
    unsigned long long gcnt[kMaxPipe];             //   dirty-list range
    unsigned long long run_off;                     //   and the running patch offset
    FusedIncr fused;                                // fused incremental: groups and counters
    Result res;
    CallParams cp;
    Job jobs[kMaxJobs];
};

enum EventId { EV_BEGIN = 0, EV_HASH_END, EV_DIFF_END, EV_COPY_END, EV_END, EV_COUNT };
enum GraphKind { GK_FULL = 0, GK_INCR, GK_RESTORE, GK_VERIFY, GK_ASYNC_FULL, GK_ASYNC_INCR, GK_INCR_PIPE,
                 GK_INCR_FUSED };
enum ShapeKind { SHAPE_GATHER = 0, SHAPE_HASH, SHAPE_SCATTER, SHAPE_COUNT };

struct GraphEntry {
    int kind;
    int parity;
    cudaGraphExec_t exec;
    uint64_t kernels;  // kernel nodes in the graph
};

struct Ring;

}  // namespace snapk

struct snap_set_s {
    int device = 0;
    int sms = 148;
    char gpu_name[256] = {0};
    uint64_t C = 65536;
    uint32_t timeout_ms = 10000;
    cudaStream_t user_stream = nullptr;  // the caller's stream (quiesced)
    cudaStream_t st = nullptr;           // library stream
    snap_opts opts{};

    std::vector<snapk::HostAlloc> allocs;
    std::vector<snapk::AllocDesc> desc;
    bool layout_dirty = true;
    uint64_t n_chunks = 0, total_bytes = 0, full_bytes = 0, patch_bound = 0;

    // device arrays (rebuilt with the layout)
    snapk::AllocDesc *d_allocs = nullptr;
    uint8_t *d_tmaps = nullptr;  // kTmapPieces tensor maps per allocation (hash staging)
    uint32_t *d_hash[2] = {nullptr, nullptr};  // committed table = d_hash[prev_idx]
    uint32_t *d_cmp = nullptr;                 // verify: expected hashes
    unsigned int *d_blockcnt = nullptr;
    unsigned long long *d_blockoff = nullptr;
    uint32_t *d_dlist = nullptr;
    uint64_t *d_patch_rec = nullptr, *d_patch_data = nullptr, *d_dstart = nullptr;
    uint32_t *h_hash_stage = nullptr;          // pinned, n_chunks hashes

    // per-call block
    snapk::CallBlock *d_cb = nullptr;
    snapk::CallBlock *h_cb = nullptr;
    snapk::Result *h_res = nullptr;

    // committed state
    int prev_idx = 0;
    bool has_base = false;
    uint64_t base_gen = 0;
    uint64_t next_gen = 0;

    // pipelined incremental: n_groups = the stage count the state's bytes
    // call for (2 or more: pipelined); at capture, n_pipe hash launches over
    // chunks [hb[g], hb[g+1]), and allocation groups [gal[g], gal[g+1])
    // (chunks [gch[g], gch[g+1])) = the allocations launch g completes;
    // two more streams and their fork/join events
    int n_groups = 0, n_pipe = 0;
    uint64_t hb[snapk::kMaxPipe + 1] = {};
    uint64_t gal[snapk::kMaxPipe + 1] = {}, gch[snapk::kMaxPipe + 1] = {};
    cudaStream_t st_pipe = nullptr, st_meta = nullptr;
    cudaEvent_t ev_pipe[2 * snapk::kMaxPipe + 1] = {};

    // fused incremental, copy-engine form: the group records and run table
    // (one pinned, mapped block), the copy stream, and the current call's
    // choice and copy count
    snapk::RunGroup *h_rungrp = nullptr;  // kFusedMaxGroups records, then runs_cap runs
    snapk::DirtyRun *h_runs = nullptr;
    uint64_t runs_cap = 0;
    cudaStream_t st_dma[snapk::kDmaStreams] = {};
    cudaEvent_t ev_dma[snapk::kDmaStreams] = {};
    cudaEvent_t ev_graph_end = nullptr;
    bool dma_call = false;
    uint64_t dma_copies = 0;

    std::vector<snapk::GraphEntry> graphs;
    snapk::TileShape shape[snapk::SHAPE_COUNT];
    std::atomic<bool> busy{false};
    bool in_flight = false;
    cudaEvent_t ev_quiesce = nullptr;
    cudaEvent_t ev[snapk::EV_COUNT] = {};
    snap_stats last{};
    uint64_t call_kernels = 0;  // kernels launched by the current call

    snapk::Ring *ring = nullptr;
    uint64_t device_err = 0;  // kernel error bits (Result.err) of the most recent call

    // asynchronous checkpoint (async.cu)
    uint8_t *d_shadow = nullptr;                // packed copy of the state at the cut
    snapk::AllocDesc *d_allocs_shadow = nullptr;  // the allocation table pointing into it
    uint64_t shadow_bytes = 0;
    cudaStream_t st_bg = nullptr;               // lowest-priority stream for the background part
    cudaEvent_t ev_bg = nullptr;               // end of the background part
    std::atomic<bool> async_pending{false};
    std::atomic<bool> async_waiting{false};
    int async_mode = 0, async_cur = 0;
    uint8_t *async_image = nullptr;
    double async_t0 = 0, async_tq = 0, async_tcut = 0;

    // prioritised restore (lazy.cu)
    uint32_t *h_order = nullptr;                  // pinned: chunk indices in restore order
    unsigned long long *d_wave_cursor = nullptr;  // one tile cursor per wave
    cudaEvent_t ev_wave[SNAP_RESTORE_MAX_WAVES] = {};
    cudaEvent_t ev_rstart = nullptr;
    std::vector<int> wave_of;                     // wave of each allocation
    int n_waves = 0;
    std::atomic<bool> restore_pending{false};
    std::atomic<bool> restore_waiting{false};
    int restore_cur = 0;
    uint64_t restore_gen = 0;
    double restore_t0 = 0, restore_tq = 0, restore_tlaunch = 0;
};

namespace snapk {

double now_ms();
bool fault_injected(const char *what);
int cuda_status(cudaError_t e);
int wait_event(cudaEvent_t ev, double deadline_ms);
uint8_t *mapped_device_ptr(const void *host);
// Pinned image regions (snap_host_alloc / snap_host_register): the mapped
// device address of [host, host+len) if that whole range lies inside one
// recorded region, else nullptr (the caller then stages through the ring,
// or refuses where only a mapping will do).
void pinned_add(const void *p, uint64_t bytes);
void pinned_remove(const void *p);
bool pinned_covers(const void *p, uint64_t len);
uint8_t *mapped_image_ptr(const void *host, uint64_t len);
// Bytes of the caller's image a checkpoint's kernels may touch: the full
// image, or for a patch the smaller of its capacity and the largest patch.
uint64_t image_extent(const snap_set_s *s, int mode, uint64_t cap);
void write_header(uint8_t *h, uint32_t flags, uint64_t C, uint64_t n, uint64_t total, uint64_t gen, uint64_t parent);
int parse_header(const uint8_t *img, uint64_t len, ImageHeader *h);
int walk_records(const snap_set_s *s, const uint8_t *img, uint64_t len, const ImageHeader &h, uint32_t *hashes);
// Reads n image bytes at off into dst; false on an I/O failure.
using ImageReader = std::function<bool(uint64_t off, void *dst, uint64_t n)>;
int walk_records_io(const snap_set_s *s, const ImageReader &rd, uint64_t len, const ImageHeader &h,
                    uint32_t *hashes);

// The host end of the ring's pipeline: a pageable image in memory, or an
// image file (file.cu).  For a file, a failed or short transfer records
// SNAP_EIO in `err` and later transfers are skipped; zero() is a no-op for
// a file, whose unwritten ranges read as zero (it is truncated to size first).
struct ImageIO {
    uint8_t *mem = nullptr;
    int fd = -1;
    std::atomic<int> err{0};
    void put(uint64_t off, const void *src, uint64_t n);
    void get(uint64_t off, void *dst, uint64_t n);
    void zero(uint64_t off, uint64_t n);
};
int apply_patch_host(uint8_t *base, uint64_t base_len, const uint8_t *patch, uint64_t patch_len);

// launch shapes (tune.cu)
void default_shapes(snap_set_s *s);
TileShape default_hash_shape(int ctas);
// the shapes the tuning cache ($SNAP_TUNE_CACHE) holds for this set's
// (GPU, operation, chunk size, state size class), adopted when its layout is built
void adopt_cached_shapes(snap_set_s *s);

// pageable images through the pinned ring (ring.cu)
int ring_checkpoint(snap_set_s *s, ImageIO &io, uint64_t cap, int mode, uint64_t *used, double t0, double tq,
                    double deadline);
int ring_restore(snap_set_s *s, ImageIO &io, const ImageHeader &h, double t0, double tq, double deadline);
void ring_free(snap_set_s *s);
int ring_get(snap_set_s *s, Ring **out);  // allocate the ring on first use

// A window: global chunks [c0, c1) = packed-state bytes [b0, b1).
struct Window {
    uint64_t c0, c1, b0, b1;
};
std::vector<Window> make_windows(const snap_set_s *s, uint64_t slot_bytes, bool taper = false);
void copy_window_part(const snap_set_s *s, const Window &w, uint8_t *slot, uint8_t *image, uint64_t p0, uint64_t p1,
                      bool to_image);
uint64_t parts_for(uint64_t bytes, int threads);

// (Re)build a set's device layout after registrations (runtime.cu).
int build_layout(snap_set_s *s);

// Holds a set's busy flag for the duration of a call.
struct BusyGuard {
    snap_set_s *s;
    bool ok;
    explicit BusyGuard(snap_set_s *s_) : s(s_) { ok = !s->busy.exchange(true); }
    ~BusyGuard() { if (ok) s->busy.store(false); }
};

// call plumbing (runtime.cu)
int settle(snap_set_s *s, double deadline);   // wait for a timed-out earlier call
int quiesce(snap_set_s *s, double deadline);  // drain the caller's stream
int async_ctas(const snap_set_s *s);
int checkpoint_graph(snap_set_s *s, int mode, int cur, uint8_t *dimg, uint64_t cap, bool from_shadow,
                     GraphEntry **out);
int complete_checkpoint(snap_set_s *s, int mode, int cur, uint8_t *host_image, uint64_t *used, snap_stats &st);

// Tensor maps of one buffer for the hash staging (runtime.cu): writes
// kTmapPieces x kTmapBytes to `out`; false if the buffer cannot use them.
bool encode_hash_maps(uint64_t ptr, uint64_t bytes, uint64_t chunk_bytes, void *out);

// two-phase coordination across ranks (coord.cu)
int coordinate(const snap_coord_ops &o, void *ctx);

// asynchronous checkpoint resources (async.cu): the shadow and its table
// (freed with the layout), the background stream and event (freed with the set)
int async_prepare(snap_set_s *s);
void async_free_layout(snap_set_s *s);
void async_free(snap_set_s *s);

// prioritised restore resources (lazy.cu): the pinned order list (freed with
// the layout), the wave cursors and events (freed with the set)
void lazy_free_layout(snap_set_s *s);
void lazy_free(snap_set_s *s);

}  // namespace snapk
