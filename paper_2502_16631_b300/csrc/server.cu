// Serving loop: checkpoint, incremental and restore requests from many
// tenant sets, continuously batched into shared persistent launches.
//
// A scheduler thread owns the GPU side.  Requests wait in arrival order and
// are admitted while the pinned-host and HBM budgets allow (a request with a
// pageable image charges min(its bytes, 2 GiB) of pinned staging; every
// request charges its tenant's resident state plus scratch of HBM).  Each
// admitted request is cut into windows of chunk tiles; every round the
// scheduler packs up to 64 windows from all admitted requests -- one window
// per request per pass, shortest remaining work first, at most 8 of one
// request -- into ONE launch of the persistent tile kernel (one job per
// window), so tiles of requests that arrived at different times share the
// GPU.  Two rounds are kept in flight.
// Host workers move window data between the server's pinned slots and the
// tenants' pageable images: slots are filled before a restore window
// launches and drained after a checkpoint window completes.  A pinned,
// mapped image needs neither: its windows read and write it directly.  When a
// request's last window is drained its metadata is written, the tenant set
// commits (exactly as the synchronous calls do) and its waiter is woken;
// latency is measured from submit to that moment.
//
// No kernel waits on the host; every host wait is bounded.
#include "snap.h"
#include "snap_format.h"
#include "runtime_internal.h"
#include "host_pool.h"
#include "host_copy.h"

#include <algorithm>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

namespace snapk {
namespace {

constexpr int kRounds = 2;
constexpr size_t kMinBatch = 8;  // windows a round waits for while another runs
constexpr int kRoundWindowsPerRequest = 8;  // windows of one request per round (each at most one slot)
constexpr uint64_t kStagingCap = 2ull << 30;  // pinned staging charged per request

static inline uint64_t upg(uint64_t x) { return (x + 4095u) & ~uint64_t(4095u); }

enum WinState { W_WAIT = 0, W_FILLING, W_READY, W_LAUNCHED, W_DRAINING, W_DONE };

struct SWin {
    uint32_t op;
    uint64_t c0, c1;  // chunk range, or dirty-rank range for OP_GATHER_DIRTY
    uint64_t b0, b1;  // packed bytes (staged windows)
    int slot = -1;
    int state = W_WAIT;
    int parts = 0;    // host tasks still running on this window
};

enum ReqPhase { P_QUEUED = 0, P_QUIESCE, P_HASH, P_WINDOWS, P_DONE };

struct SReq {
    uint64_t ticket = 0;
    snap_set_s *set = nullptr;
    int kind = 0;
    uint8_t *image = nullptr;
    uint8_t *dimg = nullptr;  // device address of a pinned, mapped image: its
                              // windows read and write it directly (no slot,
                              // no host copy); null for a pageable image
    uint64_t cap = 0;
    double t_arrive = 0, t_admit = 0, t_done = 0;
    int status = 1;  // 1 while running
    int phase = P_QUEUED;
    std::vector<SWin> wins;
    size_t done_w = 0;
    int cur = 0;
    uint64_t gen = 0;
    ImageHeader h{};
    std::vector<uint32_t> dl;
    std::vector<uint64_t> prec, pdat, dst;
    uint64_t pinned_charge = 0, hbm_charge = 0;
    uint64_t used = 0;  // image bytes written
    snap_stats st{};
    cudaEvent_t ev_q = nullptr;
    bool failed = false;
};

struct Round {
    Job *d_jobs = nullptr, *h_jobs = nullptr;
    unsigned long long *d_cursor = nullptr;
    Result *d_res = nullptr, *h_res = nullptr;
    cudaEvent_t ev = nullptr;
    std::vector<std::pair<SReq *, size_t>> wins;
    bool busy = false;
    double t_launch = 0;
};

}  // namespace
}  // namespace snapk

using namespace snapk;

struct snap_server_s {
    int device = 0;
    int sms = 148;
    uint64_t C = 65536;
    uint32_t timeout_ms = 10000;
    cudaStream_t st = nullptr, ctl = nullptr;
    uint64_t pinned_budget = 0, hbm_budget = 0, pinned_used = 0, hbm_used = 0;
    uint64_t slot_bytes = 64ull << 20;
    int nslots = 0;
    uint8_t *pool_host = nullptr, *pool_dev = nullptr;
    std::vector<int> free_slots;
    Pool *workers = nullptr;
    TileShape shape{10, 2, 128, 148, 1};
    CombineConsts cc{};
    Round rounds[kRounds];
    std::mutex mu;
    std::condition_variable cv;
    std::deque<SReq *> pending;
    std::vector<SReq *> active;
    std::map<uint64_t, SReq *> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread sched;
    // counters, printed at destroy when SNAP_LOG is set
    uint64_t n_rounds = 0, n_windows = 0, host_bytes = 0;
    double gpu_busy_ms = 0, host_copy_ms = 0, t_first = 0, t_last = 0;
    std::mutex stat_mu;
};

namespace snapk {
namespace {

// ------------------------------------------------------------- helpers
Job base(const snap_server_s *sv, const SReq *r, uint32_t op, Round &rd)
{
    const snap_set_s *s = r->set;
    Job j{};
    j.allocs = s->d_allocs;
    j.n_allocs = s->desc.size();
    j.chunk_bytes = s->C;
    j.op = op;
    j.layout = LAYOUT_PACKED;
    j.res = rd.d_res;
    (void)sv;
    return j;
}

void fail(snap_server_s *sv, SReq *r, int rc)
{
    r->failed = true;
    if (r->status == 1) r->status = rc;
    (void)sv;
}

// Build the windows of a request once its tenant is quiesced.
int prepare(snap_server_s *sv, SReq *r)
{
    snap_set_s *s = r->set;
    cudaSetDevice(s->device);
    int rc = build_layout(s);
    if (rc) return rc;
    if (r->kind == SNAP_REQ_INCREMENTAL && !s->has_base) return SNAP_ENOBASE;
    if (r->kind == SNAP_REQ_FULL && r->cap < s->full_bytes) return SNAP_EINVAL;
    if (r->kind == SNAP_REQ_RESTORE) {
        if (r->cap < s->full_bytes) return SNAP_EFORMAT;
        rc = walk_records(s, r->image, r->cap, r->h, s->h_hash_stage);  // validates, collects hashes
        if (rc) return rc;
    }
    r->cur = 1 - s->prev_idx;
    r->gen = s->next_gen;
    if (r->kind == SNAP_REQ_INCREMENTAL) {
        SWin w{};
        w.op = OP_HASH;
        w.c0 = 0;
        w.c1 = s->n_chunks;
        w.state = W_READY;
        r->wins.push_back(w);
        r->phase = P_HASH;
        return SNAP_OK;
    }
    const uint32_t op = r->kind == SNAP_REQ_RESTORE ? OP_SCATTER : OP_GATHER;
    for (const Window &x : make_windows(s, sv->slot_bytes)) {
        SWin w{};
        w.op = op;
        w.c0 = x.c0;
        w.c1 = x.c1;
        w.b0 = x.b0;
        w.b1 = x.b1;
        if (r->dimg) w.state = W_READY;  // direct: nothing to stage
        r->wins.push_back(w);
    }
    if (r->kind == SNAP_REQ_RESTORE && s->n_chunks) {
        // the image's hashes become the tenant's table (walk_records filled the stage)
        cudaError_t e = cudaMemcpyAsync(s->d_hash[r->cur], s->h_hash_stage, s->n_chunks * 4, cudaMemcpyHostToDevice,
                                        sv->ctl);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sv->ctl);
        if (e != cudaSuccess) return cuda_status(e);
    }
    r->phase = P_WINDOWS;
    return SNAP_OK;
}

// After the hash pass of an incremental request: diff, layout, metadata,
// then the dirty-chunk windows.
int after_hash(snap_server_s *sv, SReq *r)
{
    snap_set_s *s = r->set;
    const uint64_t na = s->desc.size();
    std::memset(s->h_cb, 0, offsetof(CallBlock, jobs));
    s->h_cb->cp.cap = r->cap;
    const uint32_t *curp = s->d_hash[r->cur], *prevp = s->d_hash[1 - r->cur];
    cudaError_t e = cudaMemcpyAsync(s->d_cb, s->h_cb, offsetof(CallBlock, jobs), cudaMemcpyHostToDevice, sv->ctl);
    if (e == cudaSuccess)
        e = launch_diff(curp, prevp, s->n_chunks, s->d_blockcnt, s->d_blockoff, s->d_dlist, &s->d_cb->res, sv->ctl);
    if (e == cudaSuccess)
        e = launch_patch_layout(s->d_allocs, na, s->C, s->d_dlist, s->d_patch_rec, s->d_patch_data, s->d_dstart,
                                &s->d_cb->cp, &s->d_cb->res, sv->ctl);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_res, &s->d_cb->res, sizeof(Result), cudaMemcpyDeviceToHost, sv->ctl);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sv->ctl);
    if (e != cudaSuccess) return cuda_status(e);
    if (s->h_res->cap_exceeded) return SNAP_EINVAL;
    const uint64_t nd = s->h_res->n_dirty;
    r->st.dirty_chunks = nd;
    r->st.image_bytes = s->h_res->patch_bytes;
    r->dl.assign(nd ? nd : 1, 0);
    r->prec.assign(na ? na : 1, 0);
    r->pdat.assign(na ? na : 1, 0);
    r->dst.assign(na + 1, 0);
    if (nd) e = cudaMemcpy(r->dl.data(), s->d_dlist, nd * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && na) e = cudaMemcpy(r->prec.data(), s->d_patch_rec, na * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && na) e = cudaMemcpy(r->pdat.data(), s->d_patch_data, na * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(r->dst.data(), s->d_dstart, (na + 1) * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && s->n_chunks) e = cudaMemcpy(s->h_hash_stage, curp, s->n_chunks * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    // metadata of the patch
    for (size_t k = 0; k < na; ++k) {
        const AllocDesc &a = s->desc[k];
        const uint64_t nk = (a.bytes + s->C - 1) / s->C;
        const uint64_t ndk = r->dst[k + 1] - r->dst[k];
        const uint64_t rec[4] = {a.bytes, nk, r->pdat[k], 0};
        uint8_t *p = r->image + r->prec[k];
        std::memcpy(p, rec, 32);
        std::memcpy(p + 32, s->h_hash_stage + a.chunk0, 4 * nk);
        const uint32_t n32 = (uint32_t)ndk;
        std::memcpy(p + 32 + 4 * nk, &n32, 4);
        for (uint64_t j = 0; j < ndk; ++j) {
            const uint32_t idx = r->dl[r->dst[k] + j] - (uint32_t)a.chunk0;
            std::memcpy(p + 36 + 4 * nk + 4 * j, &idx, 4);
        }
        const uint64_t z = r->prec[k] + 36 + 4 * nk + 4 * ndk;
        std::memset(r->image + z, 0, r->pdat[k] - z);
    }
    r->used = s->h_res->patch_bytes;
    // dirty windows: whole C-byte slots
    const uint64_t per = sv->slot_bytes / s->C;
    for (uint64_t r0 = 0; r0 < nd; r0 += per) {
        SWin w{};
        w.op = OP_GATHER_DIRTY;
        w.c0 = r0;
        w.c1 = std::min(nd, r0 + per);
        if (r->dimg) w.state = W_READY;
        r->wins.push_back(w);
    }
    r->phase = P_WINDOWS;
    return SNAP_OK;
}

// Copy a drained dirty window's chunks from the slot into the patch.
void drain_dirty(const SReq *r, const SWin &w, const uint8_t *slot)
{
    const snap_set_s *s = r->set;
    const size_t na = s->desc.size();
    size_t k = 0;
    for (uint64_t q = w.c0; q < w.c1; ++q) {
        const uint64_t c = r->dl[q];
        while (k + 1 < na && s->desc[k + 1].chunk0 <= c) ++k;
        const AllocDesc &a = s->desc[k];
        const uint64_t i = c - a.chunk0;
        const uint64_t L = std::min<uint64_t>(s->C, a.bytes - i * s->C);
        stream_copy(r->image + r->pdat[k] + (q - r->dst[k]) * s->C, slot + (q - w.c0) * s->C, upg(L));
    }
}

// Last window done: metadata (full checkpoints), header, commit.
void finish(snap_server_s *sv, SReq *r)
{
    snap_set_s *s = r->set;
    int rc = r->failed ? r->status : SNAP_OK;
    if (rc == SNAP_OK && r->kind == SNAP_REQ_FULL) {
        cudaError_t e = cudaSuccess;
        if (s->n_chunks) e = cudaMemcpy(s->h_hash_stage, s->d_hash[r->cur], s->n_chunks * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_status(e);
        for (size_t k = 0; rc == SNAP_OK && k < s->desc.size(); ++k) {
            const AllocDesc &a = s->desc[k];
            const uint64_t nk = (a.bytes + s->C - 1) / s->C;
            const uint64_t rec[4] = {a.bytes, nk, a.data_off, 0};
            std::memcpy(r->image + a.rec_off, rec, 32);
            std::memcpy(r->image + a.rec_off + 32, s->h_hash_stage + a.chunk0, 4 * nk);
            std::memset(r->image + a.rec_off + 32 + 4 * nk, 0, a.data_off - (a.rec_off + 32 + 4 * nk));
            std::memset(r->image + a.data_off + a.bytes, 0, upg(a.data_off + a.bytes) - (a.data_off + a.bytes));
        }
        if (rc == SNAP_OK)
            write_header(r->image, SNAP_IMG_FLAG_DEVICE_STATE, s->C, s->desc.size(), s->total_bytes, r->gen, 0);
        r->used = s->full_bytes;
        r->st.image_bytes = s->full_bytes;
        r->st.dirty_chunks = s->n_chunks;
    } else if (rc == SNAP_OK && r->kind == SNAP_REQ_INCREMENTAL) {
        write_header(r->image, SNAP_IMG_FLAG_DEVICE_STATE | SNAP_IMG_FLAG_INCREMENTAL, s->C, s->desc.size(),
                     s->total_bytes, r->gen, s->base_gen);
    }
    if (rc == SNAP_OK) {
        s->prev_idx = r->cur;
        s->has_base = true;
        if (r->kind == SNAP_REQ_RESTORE) {
            s->base_gen = r->h.generation;
            s->next_gen = r->h.generation + 1;
            r->st.image_bytes = s->full_bytes;
        } else {
            s->base_gen = r->gen;
            s->next_gen = r->gen + 1;
        }
    }
    r->t_done = now_ms();
    r->st.state_bytes = s->total_bytes;
    r->st.total_chunks = s->n_chunks;
    r->st.generation = r->kind == SNAP_REQ_RESTORE ? r->h.generation : r->gen;
    r->st.total_ms = r->t_done - r->t_arrive;
    r->st.frozen_ms = r->st.total_ms;
    r->st.quiesce_ms = r->t_admit - r->t_arrive;  // time queued before admission
    s->busy.store(false);
    sv->pinned_used -= r->pinned_charge;
    sv->hbm_used -= r->hbm_charge;
    std::vector<uint32_t>().swap(r->dl);
    std::vector<uint64_t>().swap(r->prec);
    std::vector<uint64_t>().swap(r->pdat);
    std::vector<uint64_t>().swap(r->dst);
    std::vector<SWin>().swap(r->wins);
    r->status = rc;
    r->phase = P_DONE;
}

bool tenant_active(const snap_server_s *sv, const snap_set_s *s)
{
    for (const SReq *r : sv->active)
        if (r->set == s) return true;
    return false;
}

uint64_t req_bytes(const SReq *r) { return r->set->total_bytes; }

void admit(snap_server_s *sv)
{
    for (auto it = sv->pending.begin(); it != sv->pending.end();) {
        SReq *r = *it;
        if (tenant_active(sv, r->set)) {
            ++it;
            continue;
        }
        // staging is charged to pageable images only (a pinned image is the
        // caller's own, counted when it was pinned)
        const uint64_t pin = r->dimg ? 0 : std::min<uint64_t>(req_bytes(r), kStagingCap);
        const uint64_t hbm = req_bytes(r) + 12 * r->set->n_chunks;
        if (sv->pinned_used + pin > sv->pinned_budget || sv->hbm_used + hbm > sv->hbm_budget) {
            ++it;
            continue;
        }
        if (r->set->busy.exchange(true)) {  // a direct call is running on this tenant
            ++it;
            continue;
        }
        r->pinned_charge = pin;
        r->hbm_charge = hbm;
        sv->pinned_used += pin;
        sv->hbm_used += hbm;
        r->t_admit = now_ms();
        r->phase = P_QUIESCE;
        cudaEventRecord(r->ev_q, r->set->user_stream);
        sv->active.push_back(r);
        it = sv->pending.erase(it);
    }
}

// Queue the host fills of a restore window (image -> slot).
void start_fill(snap_server_s *sv, SReq *r, size_t wi)
{
    SWin &w = r->wins[wi];
    const uint64_t nbytes = w.b1 - w.b0;
    const uint64_t np = parts_for(nbytes, sv->workers->size());
    w.parts = (int)np;
    w.state = W_FILLING;
    const Window x{w.c0, w.c1, w.b0, w.b1};
    uint8_t *slot = sv->pool_host + (uint64_t)w.slot * sv->slot_bytes;
    for (uint64_t p = 0; p < np; ++p) {
        const uint64_t p0 = nbytes * p / np, p1 = nbytes * (p + 1) / np;
        sv->workers->push([sv, r, wi, x, slot, p0, p1] {
            const double c0 = now_ms();
            copy_window_part(r->set, x, slot, r->image, p0, p1, false);
            {
                std::lock_guard<std::mutex> g(sv->stat_mu);
                sv->host_copy_ms += now_ms() - c0;
                sv->host_bytes += p1 - p0;
            }
            std::lock_guard<std::mutex> lk(sv->mu);
            SWin &ww = r->wins[wi];
            if (--ww.parts == 0) ww.state = W_READY;
            sv->cv.notify_all();
        });
    }
}

// Queue the host drain of a checkpoint window (slot -> image).
void start_drain(snap_server_s *sv, SReq *r, size_t wi)
{
    SWin &w = r->wins[wi];
    w.state = W_DRAINING;
    uint8_t *slot = sv->pool_host + (uint64_t)w.slot * sv->slot_bytes;
    if (w.op == OP_GATHER_DIRTY) {
        w.parts = 1;
        const SWin copy = w;
        sv->workers->push([sv, r, wi, copy, slot] {
            drain_dirty(r, copy, slot);
            std::lock_guard<std::mutex> lk(sv->mu);
            SWin &ww = r->wins[wi];
            if (--ww.parts == 0) {
                ww.state = W_DONE;
                sv->free_slots.push_back(ww.slot);
                ++r->done_w;
            }
            sv->cv.notify_all();
        });
        return;
    }
    const uint64_t nbytes = w.b1 - w.b0;
    const uint64_t np = parts_for(nbytes, sv->workers->size());
    w.parts = (int)np;
    const Window x{w.c0, w.c1, w.b0, w.b1};
    for (uint64_t p = 0; p < np; ++p) {
        const uint64_t p0 = nbytes * p / np, p1 = nbytes * (p + 1) / np;
        sv->workers->push([sv, r, wi, x, slot, p0, p1] {
            const double c0 = now_ms();
            copy_window_part(r->set, x, slot, r->image, p0, p1, true);
            {
                std::lock_guard<std::mutex> g(sv->stat_mu);
                sv->host_copy_ms += now_ms() - c0;
                sv->host_bytes += p1 - p0;
            }
            std::lock_guard<std::mutex> lk(sv->mu);
            SWin &ww = r->wins[wi];
            if (--ww.parts == 0) {
                ww.state = W_DONE;
                sv->free_slots.push_back(ww.slot);
                ++r->done_w;
            }
            sv->cv.notify_all();
        });
    }
}

// Windows that could join a round now.
size_t count_ready(const snap_server_s *sv)
{
    size_t n = 0, need_slot = 0;
    for (const SReq *r : sv->active) {
        if (r->phase != P_WINDOWS && r->phase != P_HASH) continue;
        for (const SWin &w : r->wins) {
            if (w.state == W_READY) ++n;
            else if (w.state == W_WAIT && w.op != OP_SCATTER) ++need_slot;
        }
    }
    return n + std::min<size_t>(need_slot, sv->free_slots.size());
}

// Fill one round with ready windows: one window per request per pass over
// the active requests, which the scheduler keeps shortest-remaining first.
bool build_round(snap_server_s *sv, Round &rd)
{
    rd.wins.clear();
    // at most kRoundWindowsPerRequest windows of one request per round: a
    // request whose windows are all ready at once (a pinned image) would
    // otherwise fill a round alone, one link direction for its whole length
    std::vector<int> taken(sv->active.size(), 0);
    bool progress = true;
    while ((int)rd.wins.size() < kMaxJobs && progress) {
        progress = false;
        for (size_t a = 0; a < sv->active.size(); ++a) {
            SReq *r = sv->active[a];
            if ((int)rd.wins.size() >= kMaxJobs) break;
            if (r->phase != P_WINDOWS && r->phase != P_HASH) continue;
            if (taken[a] >= kRoundWindowsPerRequest) continue;
            for (size_t i = 0; i < r->wins.size(); ++i) {
                SWin &w = r->wins[i];
                bool take = false;
                if (w.state == W_READY) take = true;  // hash windows, filled restore windows
                else if (w.state == W_WAIT && w.op != OP_SCATTER && !sv->free_slots.empty()) {
                    w.slot = sv->free_slots.back();
                    sv->free_slots.pop_back();
                    take = true;
                }
                if (take) {
                    w.state = W_LAUNCHED;
                    rd.wins.emplace_back(r, i);
                    ++taken[a];
                    progress = true;
                    break;  // one window per request per pass: fair interleaving
                }
            }
        }
    }
    return !rd.wins.empty();
}

cudaError_t launch_round(snap_server_s *sv, Round &rd)
{
    // device -> host (and hash) windows first, restores last: the kernel
    // works on the two groups with separate cursors, both link directions
    auto is_a = [](const std::pair<SReq *, size_t> &p) { return p.first->wins[p.second].op != OP_SCATTER; };
    const auto mid = std::stable_partition(rd.wins.begin(), rd.wins.end(), is_a);
    const int n_a = (int)(mid - rd.wins.begin());
    for (size_t q = 0; q < rd.wins.size(); ++q) {
        SReq *r = rd.wins[q].first;
        const SWin &w = r->wins[rd.wins[q].second];
        Job j = base(sv, r, w.op, rd);
        if (w.op == OP_HASH) {
            j.tile_begin = w.c0;
            j.n_tiles = w.c1 - w.c0;
            j.hash_out = r->set->d_hash[r->cur];
        } else if (w.op == OP_GATHER_DIRTY) {
            j.tile_list = r->set->d_dlist + w.c0;
            j.n_tiles = w.c1 - w.c0;
            if (r->dimg) {
                // straight into the patch: dirty rank c0 + tile, at the slot
                // the patch layout gave it
                j.layout = LAYOUT_IMAGE;
                j.host = r->dimg;
                j.window_off = w.c0;
                j.patch_data = r->set->d_patch_data;
                j.dstart = r->set->d_dstart;
            } else {
                j.host = sv->pool_dev + (uint64_t)w.slot * sv->slot_bytes;
            }
        } else {
            j.tile_begin = w.c0;
            j.n_tiles = w.c1 - w.c0;
            if (r->dimg) {
                j.layout = LAYOUT_IMAGE;
                j.host = r->dimg;
            } else {
                j.host = sv->pool_dev + (uint64_t)w.slot * sv->slot_bytes;
                j.window_off = w.b0;
            }
            if (w.op == OP_GATHER) j.hash_out = r->set->d_hash[r->cur];
        }
        rd.h_jobs[q] = j;
    }
    std::memset(rd.h_res, 0, sizeof(Result));
    cudaError_t e = cudaMemcpyAsync(rd.d_jobs, rd.h_jobs, sizeof(Job) * rd.wins.size(), cudaMemcpyHostToDevice, sv->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(rd.d_cursor, 0, 2 * sizeof(unsigned long long), sv->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(rd.d_res, 0, sizeof(Result), sv->st);
    if (e == cudaSuccess)
        e = launch_tiles2(rd.d_jobs, (int)rd.wins.size(), n_a, rd.d_cursor, rd.d_cursor + 1, sv->cc, sv->shape,
                          rd.d_res, sv->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rd.h_res, rd.d_res, sizeof(Result), cudaMemcpyDeviceToHost, sv->st);
    if (e == cudaSuccess) e = cudaEventRecord(rd.ev, sv->st);
    rd.busy = e == cudaSuccess;
    if (rd.busy) {
        const double t = now_ms();
        rd.t_launch = t;
        if (sv->t_first == 0) sv->t_first = t;
        ++sv->n_rounds;
        sv->n_windows += rd.wins.size();
    }
    return e;
}

void complete_round(snap_server_s *sv, Round &rd)
{
    const bool kerr = rd.h_res->err != 0;
    for (auto &p : rd.wins) {
        SReq *r = p.first;
        SWin &w = r->wins[p.second];
        if (kerr) fail(sv, r, SNAP_ECUDA);
        if ((w.op == OP_GATHER || w.op == OP_GATHER_DIRTY) && !r->dimg) {
            if (r->failed) {
                w.state = W_DONE;
                sv->free_slots.push_back(w.slot);
                ++r->done_w;
            } else {
                start_drain(sv, r, p.second);
            }
        } else {
            if (w.slot >= 0) sv->free_slots.push_back(w.slot);
            w.state = W_DONE;
            ++r->done_w;
        }
    }
    rd.wins.clear();
    rd.busy = false;
}

void scheduler(snap_server_s *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        if (sv->stop && sv->pending.empty() && sv->active.empty()) break;
        admit(sv);
        for (SReq *r : sv->active) {
            if (r->phase == P_QUIESCE) {
                const cudaError_t q = cudaEventQuery(r->ev_q);
                if (q == cudaErrorNotReady) {
                    if (now_ms() > r->t_admit + r->set->timeout_ms) {
                        fail(sv, r, SNAP_ETIMEDOUT);
                        finish(sv, r);
                    }
                    continue;
                }
                const int rc = q == cudaSuccess ? prepare(sv, r) : cuda_status(q);
                if (rc) {
                    fail(sv, r, rc);
                    finish(sv, r);
                }
            }
        }
        // Shortest remaining work first: requests nearer completion get the
        // staging slots and the round places first, so they leave sooner and
        // fewer requests share the link at any time.  Requests still hashing
        // or quiescing are ranked by their size in 64 MiB windows.
        std::stable_sort(sv->active.begin(), sv->active.end(), [](const SReq *x, const SReq *y) {
            const uint64_t rx = x->wins.size() - std::min<uint64_t>(x->wins.size(), x->done_w);
            const uint64_t ry = y->wins.size() - std::min<uint64_t>(y->wins.size(), y->done_w);
            const uint64_t kx = x->phase == P_WINDOWS ? 2 * rx + 1 : x->set->total_bytes >> 26;
            const uint64_t ky = y->phase == P_WINDOWS ? 2 * ry + 1 : y->set->total_bytes >> 26;
            return kx < ky;
        });
        // restore fills need slots before their windows can launch
        for (SReq *r : sv->active) {
            if (r->phase != P_WINDOWS || r->kind != SNAP_REQ_RESTORE) continue;
            for (size_t i = 0; i < r->wins.size() && !sv->free_slots.empty(); ++i) {
                SWin &w = r->wins[i];
                if (w.state != W_WAIT) continue;
                w.slot = sv->free_slots.back();
                sv->free_slots.pop_back();
                start_fill(sv, r, i);
                break;  // one new fill per request per pass
            }
        }
        // completed rounds
        for (Round &rd : sv->rounds) {
            if (!rd.busy) continue;
            const cudaError_t q = cudaEventQuery(rd.ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) rd.h_res->err |= 1;
            {
                // rounds finish in stream order: busy time is the union of
                // [launch, completion] intervals
                const double t = now_ms();
                sv->gpu_busy_ms += t - std::max(rd.t_launch, sv->t_last);
                sv->t_last = t;
            }
            complete_round(sv, rd);
        }
        // hash passes done -> diff and dirty windows
        for (SReq *r : sv->active) {
            if (r->phase == P_HASH && r->done_w == 1 && !r->failed) {
                r->wins.clear();
                r->done_w = 0;
                lk.unlock();
                const int rc = after_hash(sv, r);
                lk.lock();
                if (rc) {
                    fail(sv, r, rc);
                    finish(sv, r);
                }
            } else if (r->phase == P_HASH && r->failed) {
                finish(sv, r);
            }
        }
        // finished requests
        for (SReq *r : sv->active) {
            if (r->phase != P_WINDOWS) continue;
            bool busy = false;
            for (const SWin &w : r->wins) busy |= (w.state == W_FILLING || w.state == W_DRAINING || w.state == W_LAUNCHED);
            if (r->done_w == r->wins.size() && !busy) finish(sv, r);
        }
        for (auto it = sv->active.begin(); it != sv->active.end();) {
            if ((*it)->phase == P_DONE) it = sv->active.erase(it);
            else ++it;
        }
        sv->cv.notify_all();  // waiters
        // launch into free round buffers
        for (Round &rd : sv->rounds) {
            if (rd.busy) continue;
            // while the GPU is busy, let windows accumulate so that a round
            // batches several requests (and both link directions)
            bool gpu_busy = false;
            for (const Round &o : sv->rounds) gpu_busy |= o.busy;
            if (gpu_busy && count_ready(sv) < kMinBatch) break;
            if (!build_round(sv, rd)) break;
            const cudaError_t e = launch_round(sv, rd);
            if (e != cudaSuccess) {
                for (auto &p : rd.wins) {
                    fail(sv, p.first, cuda_status(e));
                    SWin &w = p.first->wins[p.second];
                    if (w.slot >= 0) sv->free_slots.push_back(w.slot);
                    w.state = W_DONE;
                    ++p.first->done_w;
                }
                rd.wins.clear();
            }
        }
        sv->cv.wait_for(lk, std::chrono::microseconds(200));
    }
}

}  // namespace
}  // namespace snapk

extern "C" {

int snap_server_create(snap_server *out, uint64_t pinned_budget, uint64_t hbm_budget, const snap_opts *o)
{
    if (!out || pinned_budget == 0 || hbm_budget == 0) return SNAP_EINVAL;
    *out = nullptr;
    auto *sv = new (std::nothrow) snap_server_s();
    if (!sv) return SNAP_ENOMEM;
    int dev = o ? o->device : -1;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        delete sv;
        return SNAP_ECUDA;
    }
    sv->device = dev;
    sv->C = (o && o->chunk_bytes) ? o->chunk_bytes : 65536;
    if (sv->C < 4096 || sv->C % 4096 || sv->C > (16u << 20)) {
        delete sv;
        return SNAP_EINVAL;
    }
    sv->timeout_ms = (o && o->timeout_ms) ? o->timeout_ms : 10000;
    sv->pinned_budget = pinned_budget;
    sv->hbm_budget = hbm_budget;
    cudaSetDevice(dev);
    // physical staging pool: the pinned budget, at most $SNAP_SERVER_POOL_BYTES (default 8 GiB)
    uint64_t pool = 8ull << 30;
    if (const char *e = std::getenv("SNAP_SERVER_POOL_BYTES")) pool = std::strtoull(e, nullptr, 10);
    if (o && o->ring_bytes) pool = o->ring_bytes;
    pool = std::min(pool, pinned_budget);
    sv->slot_bytes = std::max<uint64_t>(sv->C, std::min<uint64_t>(64ull << 20, pool / 4)) & ~uint64_t(4095u);
    sv->nslots = (int)std::max<uint64_t>(2, pool / sv->slot_bytes);
    cudaDeviceProp prop{};
    cudaError_t e = cudaGetDeviceProperties(&prop, dev);
    sv->sms = prop.multiProcessorCount;
    sv->shape = TileShape{10, 2, 128, sv->sms, 1};
    sv->cc = make_combine_consts(sv->C, sv->shape.piece);
    if (e == cudaSuccess) e = init_tile_kernel();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->ctl, cudaStreamNonBlocking);
    if (e == cudaSuccess && fault_injected("pinned_alloc")) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess)
        e = cudaHostAlloc((void **)&sv->pool_host, sv->slot_bytes * sv->nslots, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) {
        sv->pool_dev = mapped_device_ptr(sv->pool_host);
        if (!sv->pool_dev) e = cudaErrorInvalidValue;
    }
    for (int i = 0; i < kRounds && e == cudaSuccess; ++i) {
        Round &rd = sv->rounds[i];
        e = cudaMalloc((void **)&rd.d_jobs, sizeof(Job) * kMaxJobs);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&rd.h_jobs, sizeof(Job) * kMaxJobs, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc((void **)&rd.d_cursor, 2 * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMalloc((void **)&rd.d_res, sizeof(Result));
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&rd.h_res, sizeof(Result), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&rd.ev, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        snap_server_destroy(sv);
        return e == cudaErrorMemoryAllocation ? SNAP_ENOMEM : SNAP_ECUDA;
    }
    for (int i = 0; i < sv->nslots; ++i) sv->free_slots.push_back(i);
    // copy workers: 5 per 4 host threads (the copies are memory-bound and a
    // worker waits on its window now and then; on a 16-thread host, 32
    // tenants at 20 requests/s: 20 workers moved 54.3-54.7 GB/s of link
    // traffic with p50 2.2-2.5 s over four runs, 16 workers 46.8-53.5 GB/s
    // with p50 2.8-10.6 s, 24 workers 53.5-53.9 GB/s; earlier 16 workers had
    // moved 7 % more than 12)
    const int hw = (int)std::thread::hardware_concurrency();
    int nw = std::max(2, std::min(40, (hw * 5 + 3) / 4));
    if (const char *w = std::getenv("SNAP_WORKERS")) nw = std::max(1, std::min(64, std::atoi(w)));
    sv->workers = new Pool(nw);
    sv->sched = std::thread(scheduler, sv);
    *out = sv;
    return SNAP_OK;
}

int snap_server_destroy(snap_server sv)
{
    if (!sv) return SNAP_EINVAL;
    if (sv->sched.joinable()) {
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->stop = true;
        }
        sv->cv.notify_all();
        sv->sched.join();  // the scheduler finishes admitted and queued requests first
    }
    if (std::getenv("SNAP_LOG") && sv->n_rounds)
        std::fprintf(stderr,
                     "snap_server: %llu rounds, %.1f windows/round, GPU busy %.1f %% of %.1f s, host copies %.1f GB "
                     "at %.1f GB/s per worker (%d workers), pool %d x %llu MiB\n",
                     (unsigned long long)sv->n_rounds, (double)sv->n_windows / sv->n_rounds,
                     100.0 * sv->gpu_busy_ms / std::max(1.0, sv->t_last - sv->t_first),
                     (sv->t_last - sv->t_first) * 1e-3, sv->host_bytes * 1e-9,
                     sv->host_bytes / std::max(1e-9, sv->host_copy_ms * 1e-3) * 1e-9, sv->workers->size(),
                     sv->nslots, (unsigned long long)(sv->slot_bytes >> 20));
    delete sv->workers;
    cudaSetDevice(sv->device);
    if (sv->st) cudaStreamSynchronize(sv->st);
    for (Round &rd : sv->rounds) {
        cudaFree(rd.d_jobs);
        cudaFreeHost(rd.h_jobs);
        cudaFree(rd.d_cursor);
        cudaFree(rd.d_res);
        cudaFreeHost(rd.h_res);
        if (rd.ev) cudaEventDestroy(rd.ev);
    }
    cudaFreeHost(sv->pool_host);
    if (sv->st) cudaStreamDestroy(sv->st);
    if (sv->ctl) cudaStreamDestroy(sv->ctl);
    for (auto &kv : sv->all) {
        if (kv.second->ev_q) cudaEventDestroy(kv.second->ev_q);
        delete kv.second;
    }
    delete sv;
    return SNAP_OK;
}

int snap_server_submit(snap_server sv, snap_set tenant, int kind, void *image, uint64_t cap, uint64_t *ticket)
{
    if (!sv || !tenant || !image || !ticket) return SNAP_EINVAL;
    if (kind != SNAP_REQ_FULL && kind != SNAP_REQ_INCREMENTAL && kind != SNAP_REQ_RESTORE) return SNAP_EINVAL;
    if (tenant->device != sv->device || tenant->C != sv->C) return SNAP_EINVAL;
    const double t = now_ms();
    auto *r = new (std::nothrow) SReq();
    if (!r) return SNAP_ENOMEM;
    r->set = tenant;
    r->kind = kind;
    r->image = static_cast<uint8_t *>(image);
    r->cap = cap;
    r->t_arrive = t;
    // an image whose whole capacity lies in one pinned, mapped region
    // (snap_host_alloc / snap_host_register) is used directly
    if (cap) r->dimg = mapped_image_ptr(image, cap);
    // size the request against the tenant's layout (built here when the
    // tenant is idle; a busy tenant's layout cannot change under it)
    if (!tenant->busy.exchange(true)) {
        cudaSetDevice(tenant->device);
        const int rc = build_layout(tenant);
        tenant->busy.store(false);
        if (rc) {
            delete r;
            return rc;
        }
    }
    if (tenant->total_bytes + 12 * tenant->n_chunks > sv->hbm_budget) {
        delete r;
        return SNAP_EBUDGET;
    }
    if (kind == SNAP_REQ_FULL && cap < tenant->full_bytes) {
        delete r;
        return SNAP_EINVAL;
    }
    if (kind == SNAP_REQ_RESTORE) {
        int rc = parse_header(r->image, cap, &r->h);
        if (rc == SNAP_OK && (r->h.flags & SNAP_IMG_FLAG_INCREMENTAL)) rc = SNAP_EFORMAT;
        if (rc) {
            delete r;
            return rc;
        }
    }
    if (cudaEventCreateWithFlags(&r->ev_q, cudaEventDisableTiming) != cudaSuccess) {
        delete r;
        return SNAP_ECUDA;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) {
        cudaEventDestroy(r->ev_q);
        delete r;
        return SNAP_EINVAL;
    }
    r->ticket = sv->next_ticket++;
    sv->all[r->ticket] = r;
    sv->pending.push_back(r);
    *ticket = r->ticket;
    sv->cv.notify_all();
    return SNAP_OK;
}

int snap_server_wait(snap_server sv, uint64_t ticket, uint32_t timeout_ms, int *status, snap_stats *st)
{
    if (!sv) return SNAP_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return SNAP_EINVAL;
    SReq *r = it->second;
    const double deadline = now_ms() + timeout_ms;
    while (r->phase != P_DONE) {
        if (now_ms() > deadline) return SNAP_ETIMEDOUT;
        sv->cv.wait_for(lk, std::chrono::milliseconds(1));
    }
    if (status) *status = r->status;
    if (st) *st = r->st;
    return SNAP_OK;
}

}  // extern "C"
