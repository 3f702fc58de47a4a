// Prioritised restore: what the application needs first is in place first.
//
// Sec. 7 cites on-demand restore (Yang et al.), where a restored process
// resumes before all of its memory is back.  Device memory has no demand
// faults to hook, so here the caller names the allocations it needs first;
// the scatter runs in waves (wave 0 = those allocations, then the rest in
// waves of doubling size), each wave one launch of the persistent tile
// kernel over a chunk list, followed by an event.  snap_restore_ready turns
// an allocation's wave event into a stream dependency of the caller, so its
// kernels start the moment their inputs are back while the later waves are
// still crossing the link.  The image and commit rules are snap_restore's.
#include "snap.h"
#include "snap_format.h"
#include "snap_internal.h"
#include "runtime_internal.h"

#include <algorithm>
#include <cstring>
#include <vector>

using namespace snapk;

namespace snapk {

static constexpr uint64_t kFirstWaveBytes = 64ull << 20;

void lazy_free_layout(snap_set_s *s)
{
    cudaFreeHost(s->h_order);
    s->h_order = nullptr;
}

void lazy_free(snap_set_s *s)
{
    lazy_free_layout(s);
    cudaFree(s->d_wave_cursor);
    s->d_wave_cursor = nullptr;
    for (auto &e : s->ev_wave) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    if (s->ev_rstart) cudaEventDestroy(s->ev_rstart);
    s->ev_rstart = nullptr;
}

static int lazy_prepare(snap_set_s *s)
{
    cudaError_t e = cudaSuccess;
    if (!s->d_wave_cursor) e = cudaMalloc((void **)&s->d_wave_cursor, SNAP_RESTORE_MAX_WAVES * sizeof(unsigned long long));
    for (auto &ev : s->ev_wave)
        if (e == cudaSuccess && !ev) e = cudaEventCreate(&ev);
    if (e == cudaSuccess && !s->ev_rstart) e = cudaEventCreate(&s->ev_rstart);
    if (e == cudaSuccess && !s->h_order) {
        if (fault_injected("order_alloc")) return SNAP_ENOMEM;
        e = cudaHostAlloc((void **)&s->h_order, std::max<uint64_t>(1, s->n_chunks) * 4, cudaHostAllocDefault);
        if (e != cudaSuccess) s->h_order = nullptr;
    }
    return cuda_status(e);
}

// Allocation order and waves: `first` (validated) then the rest by index.
// Fills s->h_order with chunk indices, s->wave_of, and the wave boundaries
// (in chunks) in `ends`.
static int plan_waves(snap_set_s *s, const uint32_t *first, uint32_t n_first, std::vector<uint64_t> &ends)
{
    const size_t n = s->desc.size();
    std::vector<char> seen(n, 0);
    std::vector<uint32_t> order;
    order.reserve(n);
    for (uint32_t i = 0; i < n_first; ++i) {
        const uint32_t k = first[i];
        if (k >= n || seen[k]) return SNAP_EINVAL;
        seen[k] = 1;
        order.push_back(k);
    }
    for (uint32_t k = 0; k < n; ++k)
        if (!seen[k]) order.push_back(k);
    s->wave_of.assign(n, 0);
    ends.clear();
    uint64_t pos = 0, wave_bytes = 0, target = kFirstWaveBytes;
    for (size_t r = 0; r < order.size(); ++r) {
        const uint32_t k = order[r];
        const AllocDesc &a = s->desc[k];
        const uint64_t nk = (a.bytes + s->C - 1) / s->C;
        s->wave_of[k] = (int)ends.size();
        for (uint64_t i = 0; i < nk; ++i) s->h_order[pos + i] = (uint32_t)(a.chunk0 + i);
        pos += nk;
        wave_bytes += a.bytes;
        // wave 0 is exactly the priority list when one is given; every other
        // wave closes once it reaches its target size
        const bool priority_wave = n_first && ends.empty();
        const bool close = priority_wave ? r + 1 == n_first : wave_bytes >= target;
        if (close && ends.size() + 1 < SNAP_RESTORE_MAX_WAVES && r + 1 < order.size()) {
            ends.push_back(pos);
            target = std::max(kFirstWaveBytes, priority_wave ? wave_bytes : 2 * wave_bytes);
            wave_bytes = 0;
        }
    }
    ends.push_back(pos);
    return SNAP_OK;
}

}  // namespace snapk

extern "C" {

int snap_restore_async(const void *host_image, uint64_t bytes, snap_set s, const uint32_t *first, uint32_t n_first)
{
    const double t0 = now_ms();
    if (!s || !host_image || ((uintptr_t)host_image & 15u)) return SNAP_EINVAL;
    if (n_first && !first) return SNAP_EINVAL;
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
    if (h.flags & SNAP_IMG_FLAG_INCREMENTAL) return SNAP_EFORMAT;  // merge patches first
    rc = walk_records(s, img, bytes, h, s->h_hash_stage);
    if (rc) return rc;
    uint8_t *dimg = mapped_image_ptr(host_image, bytes);
    if (!dimg) return SNAP_EINVAL;  // the waves read through the mapping
    rc = lazy_prepare(s);
    if (rc) return rc;
    std::vector<uint64_t> ends;
    rc = plan_waves(s, first, n_first, ends);
    if (rc) return rc;
    rc = quiesce(s, deadline);
    if (rc) return rc;
    const double tq = now_ms();

    // the call block: one scatter job per wave over its slice of the order
    CallBlock &cb = *s->h_cb;
    std::memset(&cb, 0, offsetof(CallBlock, jobs));
    cb.res.first_bad = ~0ull;
    cb.cp.image = dimg;
    cb.cp.cap = bytes;
    uint32_t *d_order = s->d_dlist;  // chunk-list scratch, unused by restores otherwise
    for (size_t w = 0; w < ends.size(); ++w) {
        const uint64_t b = w ? ends[w - 1] : 0;
        Job j{};
        j.allocs = s->d_allocs;
        j.n_allocs = s->desc.size();
        j.chunk_bytes = s->C;
        j.tile_list = d_order + b;
        j.n_tiles = ends[w] - b;
        j.host = dimg;
        j.op = OP_SCATTER;
        j.layout = LAYOUT_IMAGE;
        j.res = &s->d_cb->res;
        cb.jobs[w] = j;
    }
    const int cur = 1 - s->prev_idx;
    const TileShape sh = s->shape[SHAPE_SCATTER];
    const CombineConsts cc = make_combine_consts(s->C, sh.piece);
    cudaStream_t q = s->st;
    cudaError_t e = cudaMemcpyAsync(s->d_cb, s->h_cb, sizeof(CallBlock), cudaMemcpyHostToDevice, q);
    if (e == cudaSuccess && s->n_chunks)
        e = cudaMemcpyAsync(d_order, s->h_order, s->n_chunks * 4, cudaMemcpyHostToDevice, q);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->d_wave_cursor, 0, SNAP_RESTORE_MAX_WAVES * sizeof(unsigned long long), q);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_rstart, q);
    uint64_t kernels = 0;
    for (size_t w = 0; w < ends.size() && e == cudaSuccess; ++w) {
        if (s->h_cb->jobs[w].n_tiles) {
            e = launch_tiles(s->d_cb->jobs + w, 1, s->d_wave_cursor + w, cc, sh, &s->d_cb->res, q);
            ++kernels;
        }
        if (e == cudaSuccess) e = cudaEventRecord(s->ev_wave[w], q);
    }
    if (e == cudaSuccess && s->n_chunks)
        e = cudaMemcpyAsync(s->d_hash[cur], s->h_hash_stage, s->n_chunks * 4, cudaMemcpyHostToDevice, q);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_res, &s->d_cb->res, sizeof(Result), cudaMemcpyDeviceToHost, q);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev[EV_END], q);
    if (e != cudaSuccess) {
        // whatever was queued may still run: the next call waits for it
        if (cudaEventRecord(s->ev[EV_END], q) == cudaSuccess) s->in_flight = true;
        return cuda_status(e);
    }
    s->n_waves = (int)ends.size();
    s->call_kernels = kernels;
    s->restore_cur = cur;
    s->restore_gen = h.generation;
    s->restore_t0 = t0;
    s->restore_tq = tq;
    s->restore_tlaunch = now_ms();
    s->restore_pending.store(true);
    g.ok = false;  // busy until snap_restore_wait
    return SNAP_OK;
}

int snap_restore_ready(snap_set s, uint32_t index, void *stream)
{
    if (!s) return SNAP_EINVAL;
    if (!s->restore_pending.load()) return index < s->allocs.size() ? SNAP_OK : SNAP_EINVAL;
    if (index >= s->wave_of.size()) return SNAP_EINVAL;
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : s->user_stream;
    return cuda_status(cudaStreamWaitEvent(st, s->ev_wave[s->wave_of[index]], 0));
}

int snap_restore_wait(snap_set s, uint32_t timeout_ms)
{
    if (!s) return SNAP_EINVAL;
    if (s->restore_waiting.exchange(true)) return SNAP_EBUSY;
    struct Release {
        snap_set_s *s;
        ~Release() { s->restore_waiting.store(false); }
    } rel{s};
    if (!s->restore_pending.load()) return SNAP_EINVAL;
    cudaSetDevice(s->device);
    int rc = wait_event(s->ev[EV_END], now_ms() + timeout_ms);
    if (rc == SNAP_ETIMEDOUT) return rc;  // still pending
    if (rc == SNAP_OK && s->h_res->err) rc = SNAP_ECUDA;
    if (rc == SNAP_OK) {
        s->prev_idx = s->restore_cur;
        s->has_base = true;
        s->base_gen = s->restore_gen;
        s->next_gen = s->restore_gen + 1;
        snap_stats st{};
        st.state_bytes = s->total_bytes;
        st.image_bytes = s->full_bytes;
        st.total_chunks = s->n_chunks;
        st.generation = s->restore_gen;
        st.quiesce_ms = s->restore_tq - s->restore_t0;
        float w0 = 0.f, all = 0.f;
        if (cudaEventElapsedTime(&w0, s->ev_rstart, s->ev_wave[0]) != cudaSuccess) w0 = 0.f;
        if (cudaEventElapsedTime(&all, s->ev_rstart, s->ev_wave[s->n_waves - 1]) != cudaSuccess) all = 0.f;
        cudaGetLastError();
        st.copy_ms = all;
        st.frozen_ms = (s->restore_tlaunch - s->restore_t0) + w0;
        st.kernel_launches = s->call_kernels;
        st.total_ms = now_ms() - s->restore_t0;
        s->last = st;
    }
    s->restore_pending.store(false);
    s->busy.store(false);
    return rc;
}

}  // extern "C"
