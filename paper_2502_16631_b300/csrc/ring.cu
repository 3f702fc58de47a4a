// Pageable images through the set's pinned ring (snap_opts.ring_bytes).
//
// A checkpoint of device state larger than any pinned image the caller can
// afford (tens of GB) streams through a fixed pinned, device-mapped ring
// split into slots.  The chunk sequence is cut into windows whose bytes fit
// one slot; for each window the persistent tile kernel gathers (and hashes)
// its chunks into the slot in packed order, and host worker threads copy the
// slot into the pageable image while the GPU fills the next slots.  Restore
// runs the other way: workers fill slots from the image, the kernel scatters
// them.  The pipeline is driven from the host only -- no kernel ever waits
// on a host flag -- and slot reuse is ordered by one CUDA event per slot
// and per-window host counters.  Every host wait is bounded by the call's
// deadline.
#include "snap.h"
#include "snap_format.h"
#include "runtime_internal.h"
#include "host_pool.h"
#include "host_copy.h"

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <functional>
#include <mutex>
#include <chrono>
#include <thread>
#include <vector>

namespace snapk {

static inline uint64_t upg(uint64_t x) { return (x + 4095u) & ~uint64_t(4095u); }

struct Ring {
    uint8_t *host = nullptr;  // pinned, mapped
    uint8_t *dev = nullptr;   // its device-visible address
    uint64_t bytes = 0, slot_bytes = 0;
    int slots = 0;
    std::vector<cudaEvent_t> ev;   // one per slot: the end of the last kernel that used it
    std::vector<cudaEvent_t> ev0;  // one per slot: the start of that kernel (device timing)
    Pool *pool = nullptr;       // copy workers: checkpoint drains, file reads
    Pool *fill_pool = nullptr;  // fewer workers for restore fills from memory images
    // one job and one tile cursor per window of the current call, uploaded
    // and zeroed once at its start (grown as calls need, never shrunk)
    Job *d_wjobs = nullptr;
    Job *h_wjobs = nullptr;  // pinned staging
    unsigned long long *d_wcursor = nullptr;
    size_t wcap = 0;
};

void ring_free(snap_set_s *s)
{
    Ring *r = s->ring;
    if (!r) return;
    if (s->st) cudaStreamSynchronize(s->st);
    delete r->pool;
    delete r->fill_pool;
    for (auto e : r->ev) if (e) cudaEventDestroy(e);
    for (auto e : r->ev0) if (e) cudaEventDestroy(e);
    cudaFreeHost(r->host);
    cudaFree(r->d_wjobs);
    cudaFreeHost(r->h_wjobs);
    cudaFree(r->d_wcursor);
    delete r;
    s->ring = nullptr;
}

int ring_get(snap_set_s *s, Ring **out)
{
    if (s->ring) {
        *out = s->ring;
        return SNAP_OK;
    }
    if (fault_injected("pinned_alloc")) return SNAP_ENOMEM;
    auto *r = new (std::nothrow) Ring();
    if (!r) return SNAP_ENOMEM;
    uint64_t bytes = s->opts.ring_bytes;
    int slots = 16;
    while (slots > 2 && bytes / slots < 4 * (uint64_t)s->C) slots /= 2;
    if (bytes / slots < s->C) bytes = (uint64_t)slots * s->C;
    r->slots = slots;
    r->slot_bytes = (bytes / slots) & ~uint64_t(4095u);
    r->bytes = r->slot_bytes * slots;
    cudaError_t e = cudaHostAlloc((void **)&r->host, r->bytes, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) r->dev = mapped_device_ptr(r->host);
    if (e == cudaSuccess && !r->dev) e = cudaErrorInvalidValue;
    r->ev.assign(slots, nullptr);
    r->ev0.assign(slots, nullptr);
    for (int i = 0; i < slots && e == cudaSuccess; ++i) e = cudaEventCreate(&r->ev[i]);
    for (int i = 0; i < slots && e == cudaSuccess; ++i) e = cudaEventCreate(&r->ev0[i]);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->ring = r;
        ring_free(s);
        return SNAP_ENOMEM;
    }
    const int hw = (int)std::thread::hardware_concurrency();
    int nw = std::max(2, std::min(12, hw > 2 ? hw - 2 : 2));
    if (const char *w = std::getenv("SNAP_RING_WORKERS")) nw = std::max(1, std::min(64, std::atoi(w)));
    r->pool = new Pool(nw);
    // A restore's fills write the slots that the scatter kernel is reading
    // over the link from host DRAM: fewer fill workers keep the fills just
    // ahead of the link instead of bursting, and the kernel's reads of pinned
    // memory slow down less (16 GiB through the 4 GiB ring on B300: scatter
    // 49.4 GB/s with 12 fill workers, 51.4 with 8, 46.2 with 16; the
    // checkpoint's drains are best with 12).
    int nf = std::min(nw, 8);
    if (const char *w = std::getenv("SNAP_RING_FILL_WORKERS")) nf = std::max(1, std::min(64, std::atoi(w)));
    r->fill_pool = new Pool(nf);
    s->ring = r;
    *out = r;
    return SNAP_OK;
}

// With `taper`, the first windows grow from kTaperBytes (doubling) and the
// last ones shrink to it (at most half of what is left): the first window's
// transfer and the last window's host copy are the two steps of a ring call
// that nothing overlaps, so they are kept short.
constexpr uint64_t kTaperBytes = 16ull << 20;

std::vector<Window> make_windows(const snap_set_s *s, uint64_t slot_bytes, bool taper)
{
    std::vector<Window> w;
    Window cur{0, 0, 0, 0};
    const uint64_t end = s->desc.empty() ? 0 : s->desc.back().state_off + s->desc.back().bytes;
    uint64_t target = slot_bytes;
    for (size_t k = 0; k < s->desc.size(); ++k) {
        const AllocDesc &a = s->desc[k];
        const uint64_t nk = (a.bytes + s->C - 1) / s->C;
        for (uint64_t i = 0; i < nk; ++i) {
            const uint64_t L = std::min<uint64_t>(s->C, a.bytes - i * s->C);
            const uint64_t b = a.state_off + i * s->C;
            if (cur.c1 > cur.c0 && (b + L) - cur.b0 > target) {
                w.push_back(cur);
                cur = Window{cur.c1, cur.c1, b, b};
            }
            if (cur.c1 == cur.c0) {
                cur.b0 = b;
                target = slot_bytes;
                if (taper) {
                    const uint64_t head = w.size() < 16 ? kTaperBytes << w.size() : slot_bytes;
                    const uint64_t tail = std::max<uint64_t>(kTaperBytes, (end - b) / 2);
                    target = std::min(slot_bytes, std::min(head, tail));
                }
            }
            cur.c1 = a.chunk0 + i + 1;
            cur.b1 = b + L;
        }
    }
    if (cur.c1 > cur.c0) w.push_back(cur);
    return w;
}

// Per-window completion counter shared by the host workers and the launcher.
struct Progress {
    std::mutex mu;
    std::condition_variable cv;
    std::vector<int> left;         // parts still running per window
    std::vector<char> launched;    // launcher recorded the window's event
    std::atomic<int> err{0};
    int outstanding = 0;           // parts queued or running

    void done(size_t w)
    {
        std::lock_guard<std::mutex> lk(mu);
        --left[w];
        --outstanding;
        cv.notify_all();
    }
    // wait until pred() with the deadline; false on timeout
    template <class F>
    bool wait(double deadline, F pred)
    {
        std::unique_lock<std::mutex> lk(mu);
        while (!pred()) {
            if (now_ms() > deadline) return false;
            cv.wait_for(lk, std::chrono::milliseconds(2));
        }
        return true;
    }
};

// Copy between the packed window [b0, b1) of the slot and the image's data
// regions, restricted to the part [p0, p1) of the window.
void copy_window_part(const snap_set_s *s, const Window &w, uint8_t *slot, uint8_t *image, uint64_t p0,
                             uint64_t p1, bool to_image)
{
    // allocations overlapping [w.b0 + p0, w.b0 + p1)
    const uint64_t lo = w.b0 + p0, hi = w.b0 + p1;
    size_t k = 0;
    {
        size_t a = 0, b = s->desc.size();
        while (b - a > 1) {  // last allocation with state_off <= lo
            const size_t m = (a + b) / 2;
            if (s->desc[m].state_off <= lo) a = m; else b = m;
        }
        k = a;
    }
    for (; k < s->desc.size() && s->desc[k].state_off < hi; ++k) {
        const AllocDesc &a = s->desc[k];
        const uint64_t x0 = std::max(lo, a.state_off), x1 = std::min(hi, a.state_off + a.bytes);
        if (x1 <= x0) continue;
        uint8_t *img = image + a.data_off + (x0 - a.state_off);
        uint8_t *sl = slot + (x0 - w.b0);
        if (to_image) stream_copy(img, sl, x1 - x0);
        else stream_copy(sl, img, x1 - x0);
    }
}

// copy_window_part for an ImageIO end (memory or file); false after an I/O error.
static bool copy_window_io(const snap_set_s *s, const Window &w, uint8_t *slot, ImageIO &io, uint64_t p0, uint64_t p1,
                           bool to_image)
{
    if (io.mem) {
        copy_window_part(s, w, slot, io.mem, p0, p1, to_image);
        return true;
    }
    const uint64_t lo = w.b0 + p0, hi = w.b0 + p1;
    size_t k = 0;
    {
        size_t a = 0, b = s->desc.size();
        while (b - a > 1) {
            const size_t m = (a + b) / 2;
            if (s->desc[m].state_off <= lo) a = m; else b = m;
        }
        k = a;
    }
    for (; k < s->desc.size() && s->desc[k].state_off < hi; ++k) {
        const AllocDesc &a = s->desc[k];
        const uint64_t x0 = std::max(lo, a.state_off), x1 = std::min(hi, a.state_off + a.bytes);
        if (x1 <= x0) continue;
        if (to_image) io.put(a.data_off + (x0 - a.state_off), slot + (x0 - w.b0), x1 - x0);
        else io.get(a.data_off + (x0 - a.state_off), slot + (x0 - w.b0), x1 - x0);
    }
    return io.err.load() == 0;
}

static Job window_job(const snap_set_s *s, Ring *r, int slot, uint32_t op, const Window &w, uint32_t *hash_out)
{
    Job j{};
    j.allocs = s->d_allocs;
    j.n_allocs = s->desc.size();
    j.chunk_bytes = s->C;
    j.tile_begin = w.c0;
    j.n_tiles = w.c1 - w.c0;
    j.host = r->dev + (uint64_t)slot * r->slot_bytes;
    j.window_off = w.b0;
    j.op = op;
    j.layout = LAYOUT_PACKED;
    j.hash_out = hash_out;
    j.res = &s->d_cb->res;
    return j;
}

// Room for n window jobs in the ring's per-call table.  A call starts with
// no earlier work of the set still running (settle), so the old table can go.
static int window_table(snap_set_s *s, Ring *r, size_t n)
{
    if (n <= r->wcap) return SNAP_OK;
    cudaStreamSynchronize(s->st);
    cudaFree(r->d_wjobs);
    cudaFreeHost(r->h_wjobs);
    cudaFree(r->d_wcursor);
    r->d_wjobs = r->h_wjobs = nullptr;
    r->d_wcursor = nullptr;
    r->wcap = 0;
    const size_t cap = std::max<size_t>(n, 64);
    cudaError_t e = cudaMalloc((void **)&r->d_wjobs, sizeof(Job) * cap);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&r->h_wjobs, sizeof(Job) * cap, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc((void **)&r->d_wcursor, sizeof(unsigned long long) * cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(r->d_wjobs);
        cudaFreeHost(r->h_wjobs);
        cudaFree(r->d_wcursor);
        r->d_wjobs = r->h_wjobs = nullptr;
        r->d_wcursor = nullptr;
        return SNAP_ENOMEM;
    }
    r->wcap = cap;
    return SNAP_OK;
}

// One copy of the call's window jobs (h_wjobs[0..n)) and one clear of their
// cursors, ahead of every window's launch on the library stream.
static cudaError_t upload_windows(snap_set_s *s, Ring *r, size_t n)
{
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(r->d_wjobs, r->h_wjobs, sizeof(Job) * n, cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->d_wcursor, 0, sizeof(unsigned long long) * n, s->st);
    return e;
}

// Launch window w's tile kernel into its slot between the slot's two events
// (start, end).
static cudaError_t launch_window(snap_set_s *s, Ring *r, size_t w, int slot, const TileShape &sh,
                                 const CombineConsts &cc)
{
    cudaError_t e = cudaEventRecord(r->ev0[slot], s->st);
    if (e == cudaSuccess) e = launch_tiles(r->d_wjobs + w, 1, r->d_wcursor + w, cc, sh, &s->d_cb->res, s->st);
    if (e == cudaSuccess) e = cudaEventRecord(r->ev[slot], s->st);
    return e;
}

// Device time (ms) of the kernel last launched into `slot`, once its end
// event has completed; the sum over a call's windows is its copy_ms.
static double slot_kernel_ms(Ring *r, int slot)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r->ev0[slot], r->ev[slot]) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
    }
    return ms;
}

// The kernels of the last min(W, slots) windows, after the stream is drained.
static double tail_kernel_ms(Ring *r, size_t W)
{
    double ms = 0.0;
    for (size_t w = W > (size_t)r->slots ? W - r->slots : 0; w < W; ++w) ms += slot_kernel_ms(r, (int)(w % r->slots));
    return ms;
}

uint64_t parts_for(uint64_t bytes, int threads)
{
    const uint64_t p = std::max<uint64_t>(1, bytes / (8ull << 20));  // about 8 MiB per part
    return std::min<uint64_t>(p, (uint64_t)threads * 2);
}

// Window size of a ring transfer: at most a slot, and about 1/32 of the
// state (at least 16 MiB), so that the first window's gather (or fill) and
// the last window's host copy, which nothing overlaps, stay short.
static uint64_t ring_window_bytes(const snap_set_s *s, const Ring *r)
{
    const uint64_t target = std::max<uint64_t>(16ull << 20, (s->total_bytes / 32 + 4095u) & ~uint64_t(4095u));
    return std::max<uint64_t>(s->C, std::min<uint64_t>(r->slot_bytes, target));
}

// Kernels this call launched may still be running after an error: the next
// call on the set waits for them (bounded) before it reuses the ring.
static void mark_in_flight(snap_set_s *s)
{
    if (cudaEventRecord(s->ev[EV_END], s->st) == cudaSuccess) s->in_flight = true;
    else cudaGetLastError();
}

// Fault injection (SNAP_FAULT=ring_stall, tests only): a checkpoint's
// copy-out task stalls until just past the call's deadline, as a consumer
// that stops draining the ring would, so the launcher's wait for a free
// slot runs out (SNAP_ETIMEDOUT); the task then finishes, so nothing
// outlives the call.
static void stall_past(double deadline)
{
    while (now_ms() < deadline + 20.0) std::this_thread::sleep_for(std::chrono::milliseconds(1));
}

// Wait for every queued worker task (bounded); used on every exit path so
// that no task outlives the caller's buffers.
static void drain(Progress &pg)
{
    std::unique_lock<std::mutex> lk(pg.mu);
    while (pg.outstanding > 0) pg.cv.wait_for(lk, std::chrono::milliseconds(2));
}

// --------------------------------------------------------------- checkpoint
static int ring_full(snap_set_s *s, Ring *r, ImageIO &io, uint64_t cap, double deadline, int cur, snap_stats &st)
{
    if (cap < s->full_bytes) return SNAP_EINVAL;
    const std::vector<Window> win = make_windows(s, ring_window_bytes(s, r), true);
    const size_t W = win.size();
    Progress pg;
    pg.left.assign(W, 0);
    pg.launched.assign(W, 0);
    int rc = window_table(s, r, W);
    if (rc) return rc;
    for (size_t w = 0; w < W; ++w)
        r->h_wjobs[w] = window_job(s, r, (int)(w % r->slots), OP_GATHER, win[w], s->d_hash[cur]);
    std::memset(s->h_cb, 0, offsetof(CallBlock, jobs));
    s->h_cb->res.first_bad = ~0ull;
    cudaError_t e = cudaMemcpyAsync(s->d_cb, s->h_cb, offsetof(CallBlock, jobs), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = upload_windows(s, r, W);
    const TileShape sh = s->shape[SHAPE_GATHER];
    const CombineConsts cc = make_combine_consts(s->C, sh.piece);
    double kms = 0.0;
    for (size_t w = 0; w < W && e == cudaSuccess && rc == SNAP_OK; ++w) {
        const int slot = (int)(w % r->slots);
        if (w >= (size_t)r->slots) {
            const size_t prev = w - r->slots;  // its copy-out must be finished
            if (!pg.wait(deadline, [&] { return pg.left[prev] == 0; })) rc = SNAP_ETIMEDOUT;
            if (pg.err) rc = pg.err;
            if (rc) break;
            kms += slot_kernel_ms(r, slot);  // its copy-out waited for the kernel
        }
        e = launch_window(s, r, w, slot, sh, cc);
        if (e != cudaSuccess) break;
        const uint64_t nbytes = win[w].b1 - win[w].b0;
        const uint64_t np = parts_for(nbytes, r->pool->size());
        {
            std::lock_guard<std::mutex> lk(pg.mu);
            pg.left[w] = (int)np;
            pg.outstanding += (int)np;
        }
        for (uint64_t p = 0; p < np; ++p) {
            const uint64_t p0 = nbytes * p / np, p1 = nbytes * (p + 1) / np;
            r->pool->push([&, w, slot, p0, p1] {
                if (fault_injected("ring_stall")) stall_past(deadline);
                if (!pg.err) {
                    const int q = wait_event(r->ev[slot], deadline);  // ETIMEDOUT or ECUDA
                    if (q) pg.err = q;
                }
                if (!pg.err && !copy_window_io(s, win[w], r->host + (uint64_t)slot * r->slot_bytes, io, p0, p1, true))
                    pg.err = SNAP_EIO;
                pg.done(w);
            });
        }
    }
    if (e != cudaSuccess && rc == SNAP_OK) rc = cuda_status(e);
    drain(pg);
    if (rc == SNAP_OK && pg.err) rc = pg.err;
    if (rc) {
        mark_in_flight(s);
        return rc;
    }
    // hashes and kernel flags
    if (s->n_chunks)
        e = cudaMemcpyAsync(s->h_hash_stage, s->d_hash[cur], s->n_chunks * 4, cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_res, &s->d_cb->res, sizeof(Result), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda_status(e);
    if (s->h_res->err) return SNAP_ECUDA;
    st.copy_ms = kms + tail_kernel_ms(r, W);
    // metadata: records, hashes and padding (the data regions are written)
    for (size_t k = 0; k < s->desc.size(); ++k) {
        const AllocDesc &a = s->desc[k];
        const uint64_t nk = (a.bytes + s->C - 1) / s->C;
        const uint64_t rec[4] = {a.bytes, nk, a.data_off, 0};
        io.put(a.rec_off, rec, 32);
        io.put(a.rec_off + 32, s->h_hash_stage + a.chunk0, 4 * nk);
        io.zero(a.rec_off + 32 + 4 * nk, a.data_off - (a.rec_off + 32 + 4 * nk));
        io.zero(a.data_off + a.bytes, upg(a.data_off + a.bytes) - (a.data_off + a.bytes));
    }
    if (io.err) return io.err;
    st.image_bytes = s->full_bytes;
    st.dirty_chunks = s->n_chunks;
    st.kernel_launches = W;
    return SNAP_OK;
}

// Incremental into a pageable patch: device hash + diff + layout as in the
// direct path, metadata written by the host from the copied-back tables, and
// the dirty chunks streamed through the ring one C-byte slot each.
static int ring_incremental(snap_set_s *s, Ring *r, ImageIO &io, uint64_t cap, double deadline, int cur,
                            uint64_t *used, snap_stats &st)
{
    std::memset(s->h_cb, 0, offsetof(CallBlock, jobs));
    s->h_cb->res.first_bad = ~0ull;
    s->h_cb->cp.image = nullptr;
    s->h_cb->cp.cap = cap;
    Job jh{};
    jh.allocs = s->d_allocs;
    jh.n_allocs = s->desc.size();
    jh.chunk_bytes = s->C;
    jh.n_tiles = s->n_chunks;
    jh.op = OP_HASH;
    jh.hash_out = s->d_hash[cur];
    jh.res = &s->d_cb->res;
    s->h_cb->jobs[0] = jh;
    const TileShape shh = s->shape[SHAPE_HASH];
    const CombineConsts cch = make_combine_consts(s->C, shh.piece);
    const uint32_t *curp = s->d_hash[cur], *prevp = s->d_hash[1 - cur];
    const double th0 = now_ms();
    cudaError_t e = cudaMemcpyAsync(s->d_cb, s->h_cb, offsetof(CallBlock, jobs) + sizeof(Job), cudaMemcpyHostToDevice,
                                    s->st);
    if (e == cudaSuccess && s->n_chunks)
        e = launch_tiles(s->d_cb->jobs, 1, &s->d_cb->cursor[0], cch, shh, &s->d_cb->res, s->st);
    if (e == cudaSuccess)
        e = launch_diff(curp, prevp, s->n_chunks, s->d_blockcnt, s->d_blockoff, s->d_dlist, &s->d_cb->res, s->st);
    if (e == cudaSuccess)
        e = launch_patch_layout(s->d_allocs, s->desc.size(), s->C, s->d_dlist, s->d_patch_rec, s->d_patch_data,
                                s->d_dstart, &s->d_cb->cp, &s->d_cb->res, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_res, &s->d_cb->res, sizeof(Result), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda_status(e);
    if (s->h_res->err) return SNAP_ECUDA;
    if (s->h_res->cap_exceeded) return SNAP_EINVAL;
    st.hash_ms = now_ms() - th0;
    const uint64_t nd = s->h_res->n_dirty, na = s->desc.size();
    std::vector<uint32_t> dl(nd ? nd : 1);
    std::vector<uint64_t> prec(na ? na : 1), pdat(na ? na : 1), dst(na + 1);
    if (nd) e = cudaMemcpy(dl.data(), s->d_dlist, nd * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && na) e = cudaMemcpy(prec.data(), s->d_patch_rec, na * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && na) e = cudaMemcpy(pdat.data(), s->d_patch_data, na * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(dst.data(), s->d_dstart, (na + 1) * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && s->n_chunks)
        e = cudaMemcpy(s->h_hash_stage, curp, s->n_chunks * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    // metadata: record, all hashes, dirty count and index list per allocation
    std::vector<uint32_t> meta;
    for (size_t k = 0; k < na; ++k) {
        const AllocDesc &a = s->desc[k];
        const uint64_t nk = (a.bytes + s->C - 1) / s->C;
        const uint64_t ndk = dst[k + 1] - dst[k];
        const uint64_t rec[4] = {a.bytes, nk, pdat[k], 0};
        meta.resize(8 + nk + 1 + ndk);
        std::memcpy(meta.data(), rec, 32);
        std::memcpy(meta.data() + 8, s->h_hash_stage + a.chunk0, 4 * nk);
        meta[8 + nk] = (uint32_t)ndk;
        for (uint64_t j = 0; j < ndk; ++j) meta[9 + nk + j] = dl[dst[k] + j] - (uint32_t)a.chunk0;
        io.put(prec[k], meta.data(), 4 * meta.size());
        const uint64_t z = prec[k] + 36 + 4 * nk + 4 * ndk;
        io.zero(z, pdat[k] - z);
    }
    if (io.err) return io.err;
    // dirty data: windows of whole C-byte slots over the dirty ranks; into
    // memory about as many windows as the ring has slots (at least 2 MiB
    // each) so that the host copies of one window overlap the gathers of the
    // next, into a file whole slots (one sequential writer per window)
    const uint64_t per_slot = r->slot_bytes / s->C;
    const uint64_t per = io.mem ? std::max<uint64_t>(1, std::min<uint64_t>(per_slot,
                                      std::max<uint64_t>((nd + r->slots - 1) / (uint64_t)r->slots,
                                                         (2ull << 20) / s->C)))
                                : per_slot;
    const size_t W = (size_t)((nd + per - 1) / per);
    Progress pg;
    pg.left.assign(W, 0);
    const TileShape shg = s->shape[SHAPE_GATHER];
    const CombineConsts ccg = make_combine_consts(s->C, shg.piece);
    double kms = 0.0;
    int rc = window_table(s, r, W);
    if (rc) return rc;
    for (size_t w = 0; w < W; ++w) {
        const uint64_t r0 = w * per, r1 = std::min<uint64_t>(nd, r0 + per);
        Job j{};
        j.allocs = s->d_allocs;
        j.n_allocs = na;
        j.chunk_bytes = s->C;
        j.tile_list = s->d_dlist + r0;
        j.n_tiles = r1 - r0;
        j.host = r->dev + (uint64_t)(w % r->slots) * r->slot_bytes;
        j.op = OP_GATHER_DIRTY;
        j.layout = LAYOUT_PACKED;
        j.res = &s->d_cb->res;
        r->h_wjobs[w] = j;
    }
    e = upload_windows(s, r, W);
    if (e != cudaSuccess) return cuda_status(e);
    for (size_t w = 0; w < W && rc == SNAP_OK; ++w) {
        const int slot = (int)(w % r->slots);
        if (w >= (size_t)r->slots) {
            const size_t prev = w - r->slots;
            if (!pg.wait(deadline, [&] { return pg.left[prev] == 0; })) rc = SNAP_ETIMEDOUT;
            if (pg.err) rc = pg.err;
            if (rc) break;
            kms += slot_kernel_ms(r, slot);
        }
        const uint64_t r0 = w * per, r1 = std::min<uint64_t>(nd, r0 + per);
        e = launch_window(s, r, w, slot, shg, ccg);
        if (e != cudaSuccess) {
            rc = cuda_status(e);
            break;
        }
        // into memory the window's chunks are copied out by up to 2 x threads
        // parts of at least 1 MiB each, so the last window's copy is short
        // too; into a file one writer per window
        const uint64_t np = io.mem ? std::min<uint64_t>({r1 - r0, (uint64_t)r->pool->size() * 2,
                                                         std::max<uint64_t>(1, (r1 - r0) * s->C >> 20)})
                                   : 1;
        {
            std::lock_guard<std::mutex> lk(pg.mu);
            pg.left[w] = (int)np;
            pg.outstanding += (int)np;
        }
        for (uint64_t p = 0; p < np; ++p) {
            const uint64_t q0 = r0 + (r1 - r0) * p / np, q1 = r0 + (r1 - r0) * (p + 1) / np;
            r->pool->push([&, w, slot, r0, q0, q1] {
                if (!pg.err) {
                    const int q = wait_event(r->ev[slot], deadline);
                    if (q) pg.err = q;
                }
                if (!pg.err) {
                    const uint8_t *sl = r->host + (uint64_t)slot * r->slot_bytes;
                    // allocation of the part's first dirty chunk, then forward
                    size_t k = (size_t)(std::upper_bound(dst.begin(), dst.begin() + na, q0) - dst.begin()) - 1;
                    for (uint64_t q = q0; q < q1; ++q) {
                        while (k + 1 < na && dst[k + 1] <= q) ++k;
                        const AllocDesc &a = s->desc[k];
                        const uint64_t i = dl[q] - a.chunk0;
                        const uint64_t L = std::min<uint64_t>(s->C, a.bytes - i * s->C);
                        io.put(pdat[k] + (q - dst[k]) * s->C, sl + (q - r0) * s->C, upg(L));
                    }
                    if (io.err) pg.err = SNAP_EIO;
                }
                pg.done(w);
            });
        }
    }
    drain(pg);
    if (rc == SNAP_OK && pg.err) rc = pg.err;
    if (rc) {
        mark_in_flight(s);
        return rc;
    }
    e = cudaMemcpyAsync(s->h_res, &s->d_cb->res, sizeof(Result), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda_status(e);
    if (s->h_res->err) return SNAP_ECUDA;
    st.copy_ms = kms + tail_kernel_ms(r, W);
    *used = s->h_res->patch_bytes;
    st.image_bytes = *used;
    st.dirty_chunks = nd;
    st.kernel_launches = 5 + W;
    return SNAP_OK;
}

int ring_checkpoint(snap_set_s *s, ImageIO &io, uint64_t cap, int mode, uint64_t *used, double t0, double tq,
                    double deadline)
{
    Ring *r = nullptr;
    int rc = ring_get(s, &r);
    if (rc) return rc;
    const int cur = 1 - s->prev_idx;
    const uint64_t gen = s->next_gen;
    snap_stats st{};
    uint8_t hdr[SNAP_IMG_HEADER_BYTES];
    if (mode == SNAP_FULL) {
        rc = ring_full(s, r, io, cap, deadline, cur, st);
        if (rc) return rc;
        write_header(hdr, SNAP_IMG_FLAG_DEVICE_STATE, s->C, s->desc.size(), s->total_bytes, gen, 0);
        *used = s->full_bytes;
    } else {
        rc = ring_incremental(s, r, io, cap, deadline, cur, used, st);
        if (rc) return rc;
        write_header(hdr, SNAP_IMG_FLAG_DEVICE_STATE | SNAP_IMG_FLAG_INCREMENTAL, s->C, s->desc.size(),
                     s->total_bytes, gen, s->base_gen);
    }
    io.put(0, hdr, sizeof hdr);
    if (io.err) return io.err;
    s->prev_idx = cur;
    s->has_base = true;
    s->base_gen = gen;
    s->next_gen = gen + 1;
    st.state_bytes = s->total_bytes;
    st.total_chunks = s->n_chunks;
    st.generation = gen;
    st.quiesce_ms = tq - t0;
    st.total_ms = now_ms() - t0;
    st.frozen_ms = st.total_ms;
    s->last = st;
    return SNAP_OK;
}

// ------------------------------------------------------------------ restore
int ring_restore(snap_set_s *s, ImageIO &io, const ImageHeader &h, double t0, double tq, double deadline)
{
    Ring *r = nullptr;
    int rc = ring_get(s, &r);
    if (rc) return rc;
    const int cur = 1 - s->prev_idx;
    const std::vector<Window> win = make_windows(s, ring_window_bytes(s, r), true);
    const size_t W = win.size();
    Progress pg;
    pg.left.assign(W, 0);
    pg.launched.assign(W, 0);
    rc = window_table(s, r, W);
    if (rc) return rc;
    for (size_t w = 0; w < W; ++w) r->h_wjobs[w] = window_job(s, r, (int)(w % r->slots), OP_SCATTER, win[w], nullptr);
    std::memset(s->h_cb, 0, offsetof(CallBlock, jobs));
    cudaError_t e = cudaMemcpyAsync(s->d_cb, s->h_cb, offsetof(CallBlock, jobs), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess && s->n_chunks)
        e = cudaMemcpyAsync(s->d_hash[cur], s->h_hash_stage, s->n_chunks * 4, cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = upload_windows(s, r, W);
    if (e != cudaSuccess) return cuda_status(e);
    const TileShape sh = s->shape[SHAPE_SCATTER];
    const CombineConsts cc = make_combine_consts(s->C, sh.piece);
    double kms = 0.0;

    // queue the fill of window w: it waits for the kernel of window w - slots
    Pool *fills = io.mem ? r->fill_pool : r->pool;  // a file is read by the full pool
    auto queue_fill = [&](size_t w) {
        const int slot = (int)(w % r->slots);
        const uint64_t nbytes = win[w].b1 - win[w].b0;
        const uint64_t np = parts_for(nbytes, fills->size());
        {
            std::lock_guard<std::mutex> lk(pg.mu);
            pg.left[w] = (int)np;
            pg.outstanding += (int)np;
        }
        for (uint64_t p = 0; p < np; ++p) {
            const uint64_t p0 = nbytes * p / np, p1 = nbytes * (p + 1) / np;
            fills->push([&, w, slot, p0, p1] {
                if (w >= (size_t)r->slots && !pg.err) {
                    const size_t prev = w - r->slots;
                    if (!pg.wait(deadline, [&] { return pg.launched[prev] != 0; })) pg.err = SNAP_ETIMEDOUT;
                    if (!pg.err) {
                        const int q = wait_event(r->ev[slot], deadline);
                        if (q) pg.err = q;
                    }
                }
                if (!pg.err && !copy_window_io(s, win[w], r->host + (uint64_t)slot * r->slot_bytes, io, p0, p1, false))
                    pg.err = SNAP_EIO;
                pg.done(w);
            });
        }
    };
    for (size_t w = 0; w < std::min<size_t>(W, r->slots); ++w) queue_fill(w);
    for (size_t w = 0; w < W && rc == SNAP_OK; ++w) {
        const int slot = (int)(w % r->slots);
        if (!pg.wait(deadline, [&] { return pg.left[w] == 0; })) rc = SNAP_ETIMEDOUT;
        if (pg.err) rc = pg.err;
        if (rc) break;
        if (w >= (size_t)r->slots) kms += slot_kernel_ms(r, slot);  // its fill waited for that kernel
        e = launch_window(s, r, w, slot, sh, cc);
        if (e != cudaSuccess) {
            rc = cuda_status(e);
            break;
        }
        {
            std::lock_guard<std::mutex> lk(pg.mu);
            pg.launched[w] = 1;
            pg.cv.notify_all();
        }
        if (w + r->slots < W) queue_fill(w + r->slots);
    }
    if (rc) {
        pg.err = rc;  // release fills waiting on windows that will not launch
        {
            std::lock_guard<std::mutex> lk(pg.mu);
            std::fill(pg.launched.begin(), pg.launched.end(), 1);
            pg.cv.notify_all();
        }
    }
    drain(pg);
    if (rc) {
        mark_in_flight(s);
        return rc;
    }
    e = cudaMemcpyAsync(s->h_res, &s->d_cb->res, sizeof(Result), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda_status(e);
    if (s->h_res->err) return SNAP_ECUDA;
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
    st.copy_ms = kms + tail_kernel_ms(r, W);
    st.kernel_launches = W;
    st.total_ms = now_ms() - t0;
    st.frozen_ms = st.total_ms;
    s->last = st;
    return SNAP_OK;
}

}  // namespace snapk
