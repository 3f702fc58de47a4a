// Asynchronous checkpoint: the caller is held only for the cut.
//
// CRIUgpu freezes the application for the whole snapshot (Sec. 3.1.1 lock,
// then checkpoint); Sec. 7 cites CheckFreq, Nebula and Gemini, which
// overlap snapshotting with training.  Here the freeze shrinks to a quiesce
// plus one device-to-device copy of the registered allocations into a
// library-owned shadow at HBM bandwidth.  The hash, diff and transfer of
// the image then run from the shadow, on a background stream of the least
// priority with a reduced grid, while the caller's stream resumes; the
// image is exactly what a synchronous checkpoint at the cut produces, and
// it is committed (Sec. 3.1: only a completed checkpoint replaces the base)
// when snap_checkpoint_wait sees it finish.
#include "snap.h"
#include "snap_format.h"
#include "snap_internal.h"
#include "runtime_internal.h"

#include <algorithm>
#include <cstring>
#include <vector>

using namespace snapk;

namespace snapk {

int async_prepare(snap_set_s *s)
{
    cudaError_t e = cudaSuccess;
    if (!s->st_bg) {
        int least = 0, greatest = 0;
        e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->st_bg, cudaStreamNonBlocking, least);
        if (e != cudaSuccess) {
            s->st_bg = nullptr;
            return cuda_status(e);
        }
    }
    if (!s->ev_bg) {
        e = cudaEventCreateWithFlags(&s->ev_bg, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            s->ev_bg = nullptr;
            return cuda_status(e);
        }
    }
    if (s->d_shadow) return SNAP_OK;
    // packed size: the last allocation's offset plus its bytes
    uint64_t bytes = 0;
    for (const AllocDesc &a : s->desc) bytes = std::max<uint64_t>(bytes, a.state_off + a.bytes);
    if (fault_injected("shadow_alloc")) return SNAP_ENOMEM;
    const size_t na = std::max<size_t>(1, s->desc.size());
    e = cudaMalloc((void **)&s->d_shadow, std::max<uint64_t>(bytes, 256));
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_allocs_shadow, na * sizeof(AllocDesc));
    if (e == cudaSuccess && !s->desc.empty()) {
        std::vector<AllocDesc> sh(s->desc);
        for (AllocDesc &a : sh) {
            a.ptr = (uint64_t)(uintptr_t)(s->d_shadow + a.state_off);
            a.tmap = 0;  // the tensor maps describe the registered buffers, not the shadow
        }
        e = cudaMemcpy(s->d_allocs_shadow, sh.data(), sh.size() * sizeof(AllocDesc), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        async_free_layout(s);
        return cuda_status(e);
    }
    s->shadow_bytes = bytes;
    return SNAP_OK;
}

void async_free_layout(snap_set_s *s)
{
    if (s->st_bg) cudaStreamSynchronize(s->st_bg);
    cudaFree(s->d_shadow);
    cudaFree(s->d_allocs_shadow);
    s->d_shadow = nullptr;
    s->d_allocs_shadow = nullptr;
    s->shadow_bytes = 0;
}

void async_free(snap_set_s *s)
{
    async_free_layout(s);
    if (s->ev_bg) cudaEventDestroy(s->ev_bg);
    if (s->st_bg) cudaStreamDestroy(s->st_bg);
    s->ev_bg = nullptr;
    s->st_bg = nullptr;
}

}  // namespace snapk

extern "C" {

int snap_checkpoint_async(snap_set s, void *host_image, uint64_t cap, int mode)
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
    if (!dimg) return SNAP_EINVAL;  // the background part writes through the mapping
    rc = async_prepare(s);
    if (rc) return rc;
    const int cur = 1 - s->prev_idx;
    GraphEntry *ge = nullptr;
    rc = checkpoint_graph(s, mode, cur, dimg, cap, true, &ge);
    if (rc) return rc;

    // the freeze: drain the caller's stream, copy the state into the shadow
    rc = quiesce(s, deadline);
    if (rc) return rc;
    const double tq = now_ms();
    cudaError_t e = launch_shadow_copy(s->d_allocs, s->desc.size(), s->C, s->n_chunks, s->d_shadow, s->sms, s->st);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev[EV_END], s->st);
    if (e != cudaSuccess) return cuda_status(e);
    rc = wait_event(s->ev[EV_END], deadline);
    if (rc == SNAP_ETIMEDOUT) s->in_flight = true;
    if (rc) return rc;
    const double tcut = now_ms();

    // the background part, from the shadow
    e = cudaGraphLaunch(ge->exec, s->st_bg);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_bg, s->st_bg);
    if (e != cudaSuccess) return cuda_status(e);
    s->call_kernels = ge->kernels + 1;  // + the shadow copy
    s->async_mode = mode;
    s->async_cur = cur;
    s->async_image = static_cast<uint8_t *>(host_image);
    s->async_t0 = t0;
    s->async_tq = tq;
    s->async_tcut = tcut;
    s->async_pending.store(true);
    g.ok = false;  // the set stays busy until snap_checkpoint_wait
    return SNAP_OK;
}

int snap_checkpoint_wait(snap_set s, uint32_t timeout_ms, uint64_t *used)
{
    if (!s) return SNAP_EINVAL;
    if (s->async_waiting.exchange(true)) return SNAP_EBUSY;
    struct Release {
        snap_set_s *s;
        ~Release() { s->async_waiting.store(false); }
    } rel{s};
    if (!s->async_pending.load()) return SNAP_EINVAL;
    cudaSetDevice(s->device);
    int rc = wait_event(s->ev_bg, now_ms() + timeout_ms);
    if (rc == SNAP_ETIMEDOUT) return rc;  // still pending
    snap_stats st{};
    if (rc == SNAP_OK && s->h_res->err) rc = SNAP_ECUDA;
    if (rc == SNAP_OK) rc = complete_checkpoint(s, s->async_mode, s->async_cur, s->async_image, used, st);
    if (rc == SNAP_OK) {
        st.quiesce_ms = s->async_tq - s->async_t0;
        st.kernel_launches = s->call_kernels;
        st.total_ms = now_ms() - s->async_t0;
        st.frozen_ms = s->async_tcut - s->async_t0;
        s->last = st;
    }
    s->async_pending.store(false);
    s->busy.store(false);
    return rc;
}

}  // extern "C"
