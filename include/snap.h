/*
 * snap.h -- C ABI of libsnap: GPU device-memory snapshot and restore.
 *
 * The library implements the data path of transparent GPU checkpointing as
 * CRIUgpu (arXiv 2502.16631) frames it: a process's device allocations are
 * copied into a host-memory checkpoint image and later put back byte for byte
 * (Sec. 3.1.1, the checkpoint and restore actions; Sec. 6, deterministic
 * restore).  On top of that it adds what Sec. 7 names as optimisations that
 * could be incorporated: per-chunk CRC-32C hashes and incremental
 * (dirty-chunk) checkpoints, a batched persistent launch, and a serving loop.
 *
 * Conventions for every call:
 *  - The return value is a status (snap_status); SNAP_OK is 0, errors are
 *    negative.  snap_strerror() names them.
 *  - Pointers marked "device" are CUDA device addresses on the set's device;
 *    "host" pointers are CPU addresses.  No call takes ownership of caller
 *    memory; the library owns what it allocates (hash tables, descriptors,
 *    graphs, the pinned ring) and frees it in the matching destroy call.
 *  - Calls are synchronous: when a call returns SNAP_OK the image (checkpoint)
 *    or the device buffers (restore) are complete.  The exceptions are
 *    snap_checkpoint_async and snap_restore_async, completed by their _wait
 *    calls (the set stays busy in between), and the serving API.
 *  - One call at a time per set: a call that finds another in progress on the
 *    same set returns SNAP_EBUSY.  Different sets may be used concurrently.
 *  - Failure atomicity (the plugin exit callback rolls back on error,
 *    Sec. 3.1): on any error the set's committed hash table, generation and
 *    base are unchanged, and no image other than the call's own output
 *    buffer is modified.
 */
#ifndef SNAP_H
#define SNAP_H

#include <stdint.h>

#if defined(__GNUC__)
#define SNAP_API __attribute__((visibility("default")))
#else
#define SNAP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
typedef enum {
    SNAP_OK = 0,
    SNAP_EINVAL = -1,     /* bad argument: null pointer, misaligned pointer,
                             capacity too small, bad option value          */
    SNAP_ENOMEM = -2,     /* a device, pinned-host or host allocation failed */
    SNAP_ECUDA = -3,      /* a CUDA runtime call failed, or a kernel reported
                             an internal error (a bounded wait expired)    */
    SNAP_ETIMEDOUT = -4,  /* quiesce or completion did not finish before the
                             deadline (Sec. 3.1.1: the lock action uses a
                             10 s timeout, then rolls back)               */
    SNAP_ENOBASE = -5,    /* incremental checkpoint without a committed base */
    SNAP_EFORMAT = -6,    /* image header/record malformed or truncated     */
    SNAP_EMISMATCH = -7,  /* image does not fit the set: allocation count or
                             sizes differ, or patch/base generations differ
                             (restore needs a compatible target, Sec. 4.4)  */
    SNAP_EBUSY = -8,      /* another call is in progress on this set        */
    SNAP_EBUDGET = -9,    /* request can never fit the server's budgets     */
    SNAP_EIO = -10,       /* opening, reading, writing or renaming an image
                             file failed                                    */
    SNAP_EPEER = -11      /* a coordinated call failed on another rank       */
} snap_status;

typedef enum { SNAP_FULL = 0, SNAP_INCREMENTAL = 1 } snap_mode;

/* Serving request kinds. */
typedef enum { SNAP_REQ_FULL = 0, SNAP_REQ_INCREMENTAL = 1, SNAP_REQ_RESTORE = 2 } snap_req_kind;

typedef struct snap_set_s *snap_set;
typedef struct snap_server_s *snap_server;

/* Options; a zero field takes the default shown. */
typedef struct {
    uint64_t chunk_bytes;  /* hash chunk C: multiple of 4096 in [4 KiB, 16 MiB]; default 65536 */
    uint32_t timeout_ms;   /* quiesce/completion deadline; default 10000 (Sec. 3.1.1) */
    int32_t device;        /* CUDA device ordinal; -1 = the current device */
    void *stream;          /* caller's cudaStream_t whose queued work must finish
                              before a snapshot starts (the "lock"); NULL = the
                              legacy default stream */
    uint32_t ctas_per_sm;  /* persistent CTAs per SM; 0 = tuned default */
    uint32_t stages;       /* staging buffers per warp; 0 = tuned default */
    uint64_t ring_bytes;   /* pinned ring for pageable images; default 4 GiB
                              (its host copy workers: min(12, host threads
                              - 2), or $SNAP_RING_WORKERS; a restore from a
                              memory image fills slots with at most 8 of
                              them, or $SNAP_RING_FILL_WORKERS) */
    uint32_t async_ctas;   /* CTAs of the background part of snap_checkpoint_async;
                              default 8 (enough to saturate the host link) */
    uint32_t hash_tma;     /* 1: stage the hash pass with 2D TMA tensor copies
                              (else per-lane cp.async; snap_autotune may
                              change it) */
    uint32_t incr_copy;    /* how a pipelined incremental checkpoint into a
                              pinned image moves its dirty chunks while the
                              hash pass runs: SNAP_INCR_COPY_DMA (the launch
                              lists each group's runs of consecutive dirty
                              chunks in mapped host memory and the calling
                              thread hands each run to the copy engines, so
                              every SM but one hashes) or SNAP_INCR_COPY_SM
                              (gather CTAs of the same launch, SM loads and
                              stores); 0 = $SNAP_INCR_COPY ("sm" / "dma") when
                              set, else DMA.  The DMA form allocates, on its
                              first use, a pinned and mapped run table of 32
                              bytes per chunk of the set and one copy stream */
} snap_opts;
enum { SNAP_INCR_COPY_DEFAULT = 0, SNAP_INCR_COPY_SM = 1, SNAP_INCR_COPY_DMA = 2 };

/* Per-call statistics (times in milliseconds; quiesce_ms and total_ms are
 * host wall time, the others come from CUDA events on the library stream). */
typedef struct {
    uint64_t state_bytes;    /* device bytes covered by the call          */
    uint64_t image_bytes;    /* bytes of image written or read            */
    uint64_t total_chunks;
    uint64_t dirty_chunks;   /* incremental: chunks copied                */
    uint64_t mismatches;     /* verify: chunks whose hash differs         */
    uint64_t generation;     /* generation of the image written/restored  */
    double quiesce_ms;
    double hash_ms;          /* hash pass (incremental / verify)          */
    double diff_ms;          /* dirty diff + compaction + patch layout    */
    double copy_ms;          /* gather (checkpoint) or scatter (restore)  */
    double total_ms;         /* call entry to return                      */
    uint64_t kernel_launches; /* libsnap kernels the call ran on the GPU  */
    double frozen_ms;        /* how long the caller was held: the whole call
                                for synchronous calls; quiesce + cut for
                                snap_checkpoint_async                     */
    uint64_t device_errors;  /* error bits the kernels of the set's most
                                recent call reported (that call returned
                                SNAP_ECUDA), 0 if none: 1 = a bounded wait
                                ran out, 2 = a tile outside its allocation
                                table or misaligned, 4 = shared memory not
                                where the CRC lookups expect it.  Unlike the
                                other fields it is not the last successful
                                call's. */
    uint64_t dma_copies;     /* copy-engine copies of dirty runs the call
                                issued (incremental, SNAP_INCR_COPY_DMA) */
} snap_stats;

/* ------------------------------------------------------------------ sets */
/* Create an empty set of device allocations on o->device.  o may be NULL.
 * *out receives the handle (owned by the library; free with
 * snap_set_destroy).  Errors: EINVAL (bad option), ENOMEM, ECUDA. */
SNAP_API int snap_set_create(snap_set *out, const snap_opts *o);

/* Release everything the set owns.  Caller memory is untouched. */
SNAP_API int snap_set_destroy(snap_set s);

/* Register a device allocation [dptr, dptr+bytes) (Sec. 3.1.1: the device
 * memory a checkpoint captures).  dptr must be a device pointer of the set's
 * device, 16-byte aligned (cudaMalloc and torch allocations are); bytes may
 * be anything, including 0.  Allocations keep registration order in the
 * image.  The caller keeps ownership and must keep the memory alive while
 * registered.  Registering after a checkpoint drops the committed base (the
 * next incremental returns ENOBASE).  Returns the allocation index (>= 0) or
 * an error (EINVAL, EBUSY). */
SNAP_API int snap_register(snap_set s, void *dptr, uint64_t bytes);

/* Do the set's one-time setup now instead of inside the first call: build
 * its device tables (what & SNAP_PREPARE_LAYOUT) and allocate its pinned
 * ring for pageable images (what & SNAP_PREPARE_RING).  Call it outside
 * stream capture and outside latency-critical regions.  Errors: EINVAL,
 * EBUSY, ENOMEM, ECUDA. */
#define SNAP_PREPARE_LAYOUT 1
#define SNAP_PREPARE_RING 2
#define SNAP_PREPARE_SHADOW 4  /* device shadow for snap_checkpoint_async */
SNAP_API int snap_set_prepare(snap_set s, int what);

/* Bytes a host image needs: exact for SNAP_FULL; an upper bound for
 * SNAP_INCREMENTAL (the patch size depends on how many chunks are dirty). */
SNAP_API int snap_image_bytes(snap_set s, int mode, uint64_t *out);

/* Pinned, device-mapped host memory for images (cudaHostAlloc, mapped and
 * portable).  An image whose bytes all lie in one such region (or one
 * snap_host_register region) is written/read by the kernels directly over
 * the host link; any other image -- pageable, pinned by other means, or only
 * partly inside a region -- goes through the set's pinned ring.  Free with
 * snap_host_free.  Errors: EINVAL, ENOMEM. */
SNAP_API int snap_host_alloc(uint64_t bytes, void **out);
SNAP_API int snap_host_free(void *p);

/* Pin and map existing host memory [p, p+bytes) -- a caller's own image
 * buffer -- so that checkpoints, restores and server requests read and
 * write it directly over the link, as they do snap_host_alloc memory,
 * instead of staging it through pinned slots and host copies.  The memory
 * stays the caller's; undo with snap_host_unregister(p) before freeing it.
 * Pinning costs time in proportion to bytes and counts against the host's
 * locked memory.  Errors: EINVAL (null, zero bytes, already registered /
 * not registered), ENOMEM, ECUDA. */
SNAP_API int snap_host_register(void *p, uint64_t bytes);
SNAP_API int snap_host_unregister(void *p);

/* --------------------------------------------------------- checkpoint path */
/* Checkpoint the set into host_image[0..cap) (16-byte aligned).
 *  SNAP_FULL: writes the full image: 64-byte header, then per allocation a
 *    32-byte record {bytes, n_chunks, data_offset, 0}, the CRC-32C of every
 *    chunk, padding to 4 KiB, the bytes, padding to 4 KiB (layout in
 *    snap_format.h).  Sec. 3.1.1 "checkpoint".
 *  SNAP_INCREMENTAL: hashes every chunk, diffs against the committed hash
 *    table, and writes a patch holding all new hashes, the ascending list of
 *    dirty chunks and only their bytes.  Needs a committed base (ENOBASE).
 * Steps: quiesce the caller's stream with the deadline (the "lock",
 * Sec. 3.1.1), run the graph-captured persistent kernels, wait with the
 * deadline, then commit the new hash table and generation.  An incremental
 * checkpoint of a state large enough to pipeline, into a pinned image whose
 * capacity covers the largest patch, moves its dirty chunks as
 * opts.incr_copy says: by default the calling thread hands each run of
 * dirty chunks the launch lists to the copy engines while the launch is
 * still hashing (the patch bytes are the same either way).  *used receives
 * the image size.  Errors: EINVAL (cap too small: nothing committed),
 * ENOBASE, ETIMEDOUT, EBUSY, ENOMEM, ECUDA. */
SNAP_API int snap_checkpoint(snap_set s, void *host_image, uint64_t cap, int mode, uint64_t *used);

/* Asynchronous checkpoint (the overlapped snapshotting Sec. 7 cites from
 * CheckFreq/Nebula/Gemini): quiesce the caller's stream, copy every
 * registered allocation device to device into a library-owned shadow
 * buffer (the cut), and return; the caller may then modify its allocations
 * freely.  Hashing, diffing and the transfer into host_image (pinned and
 * mapped: snap_host_alloc memory) run from the shadow on a least-priority
 * stream with opts.async_ctas CTAs, leaving the other SMs to the caller.
 * snap_last_stats after the wait: frozen_ms = entry to return of this call,
 * total_ms = entry to the commit in snap_checkpoint_wait.
 * The result is exactly what snap_checkpoint would have produced at the
 * cut.  The set stays busy (EBUSY for other calls) until
 * snap_checkpoint_wait.  The shadow (the packed size of the state) is
 * allocated on first use, or by snap_set_prepare(SNAP_PREPARE_SHADOW).
 * Errors as snap_checkpoint, plus EINVAL for a pageable image. */
SNAP_API int snap_checkpoint_async(snap_set s, void *host_image, uint64_t cap, int mode);

/* Wait up to timeout_ms for the pending asynchronous checkpoint; on
 * completion write its header, commit and return its status (*used = image
 * bytes).  ETIMEDOUT leaves it pending; EINVAL if none is pending. */
SNAP_API int snap_checkpoint_wait(snap_set s, uint32_t timeout_ms, uint64_t *used);

/* Restore a full image into the set's registered buffers (Sec. 3.1.1
 * "restore"; Sec. 6).  The image must describe the same allocation count and
 * sizes (EMISMATCH otherwise) and be well formed (EFORMAT; a patch must first
 * be merged with snap_apply_patch).  The image's hashes become the committed
 * base.  Errors: EINVAL, EFORMAT, EMISMATCH, ETIMEDOUT, EBUSY, ECUDA. */
SNAP_API int snap_restore(const void *host_image, uint64_t bytes, snap_set s);

/* Persist a checkpoint straight to storage (the "memory write" stage of the
 * paper's checkpoint, Table 2), overlapped with the gather: windows of the
 * state stream through the set's pinned ring and host workers write each
 * window to the file as soon as the GPU has filled it, so the device-to-host
 * link and the storage work at the same time.  The image (full or patch,
 * byte-identical to what snap_checkpoint writes into memory) goes to
 * "<path>.tmp", which is renamed to `path` only after the whole image is
 * written (and, with SNAP_FILE_SYNC, flushed to the device with fsync), so
 * `path` never holds a partial image; on any failure the temporary file is
 * removed and nothing is committed.  *used = image bytes.  The completion
 * deadline is timeout_ms plus the image size at 64 MB/s.  Errors as
 * snap_checkpoint, plus EIO. */
#define SNAP_FILE_SYNC 1
SNAP_API int snap_checkpoint_file(snap_set s, const char *path, int mode, int flags, uint64_t *used);

/* Restore a full image file written by snap_checkpoint_file (or any full
 * image saved to a file), overlapping the reads with the scatter through the
 * pinned ring.  The header and every record are read and validated before
 * any device byte changes.  Errors as snap_restore, plus EIO. */
SNAP_API int snap_restore_file(const char *path, snap_set s);

/* Prioritised restore (the on-demand restore Sec. 7 cites from Yang et al.:
 * what the application needs first is restored first).  Validates the image
 * as snap_restore does, quiesces the caller's stream and queues the scatter
 * in priority order: the n_first allocations listed in `first` (indices as
 * snap_register returned them, no repeats; may be empty) form wave 0, the
 * other allocations follow in index order in waves of doubling size (the
 * first at least 64 MiB; at most SNAP_RESTORE_MAX_WAVES waves).  Returns
 * once the waves are queued.  snap_restore_ready makes a stream wait for one
 * allocation; snap_restore_wait finishes the restore.  Until then the set
 * answers SNAP_EBUSY to other calls, and the image (pinned and mapped:
 * snap_host_alloc memory) must stay untouched.  Errors as snap_restore, plus
 * EINVAL for a pageable image or a bad `first` list. */
#define SNAP_RESTORE_MAX_WAVES 16u
SNAP_API int snap_restore_async(const void *host_image, uint64_t bytes, snap_set s, const uint32_t *first,
                                uint32_t n_first);

/* Make `stream` (a cudaStream_t; NULL: the set's stream) wait, without
 * blocking the host, until allocation `index` of the pending prioritised
 * restore is in place.  With no restore pending the allocation is already
 * in place and it returns SNAP_OK.  EINVAL for an index out of range.  Not
 * to be called concurrently with snap_restore_wait on the same set. */
SNAP_API int snap_restore_ready(snap_set s, uint32_t index, void *stream);

/* Wait up to timeout_ms for the pending prioritised restore; on completion
 * adopt the image's hashes and generation as the committed base (as
 * snap_restore does) and return its status.  ETIMEDOUT leaves it pending;
 * EINVAL if none is pending.  snap_last_stats afterwards: frozen_ms = call
 * entry until wave 0 was in place, total_ms = call entry until the commit,
 * copy_ms = device time of all waves. */
SNAP_API int snap_restore_wait(snap_set s, uint32_t timeout_ms);

/* Re-hash the device state and compare every chunk with the hashes stored in
 * host_image (a full image or a patch).  *n_mismatch = number of differing
 * chunks.  Sec. 6 (a restore must reproduce the snapshotted state). */
SNAP_API int snap_verify(const void *host_image, uint64_t bytes, snap_set s, uint64_t *n_mismatch);

/* Merge a patch into its base full image in place (host only): dirty chunks
 * are copied into their slots, all hashes replaced, the generation advanced.
 * base.generation must equal patch.parent_generation (EMISMATCH); both are
 * validated completely before the base is modified (EFORMAT leaves it
 * intact; so does ENOMEM, when the host cannot hold the per-allocation
 * tables of a base whose header claims very many allocations). */
SNAP_API int snap_apply_patch(void *base_image, uint64_t base_bytes, const void *patch, uint64_t patch_bytes);

/* Copy the committed hash table (all chunks, registration order) to host
 * out[0..n) and its generation; EINVAL if n is smaller than the chunk count,
 * ENOBASE if nothing is committed. */
SNAP_API int snap_committed_hashes(snap_set s, uint32_t *out, uint64_t n, uint64_t *generation);

/* Statistics of the set's last successful call. */
SNAP_API int snap_last_stats(snap_set s, snap_stats *out);

/* Static message for a status code. */
SNAP_API const char *snap_strerror(int status);

/* ------------------------------------------------------------- plain form */
/* The comparison baseline, not a fallback: one cudaMemcpyAsync per
 * allocation between the device buffers and the data regions of a full
 * image (no hashes, no header), full copy every time. */
SNAP_API int snap_plain_checkpoint(snap_set s, void *host_image, uint64_t cap);
SNAP_API int snap_plain_restore(const void *host_image, uint64_t bytes, snap_set s);

/* ------------------------------------------------------------- hashing */
/* Standalone chunk hasher: hashes[i] = CRC-32C of bytes [i*C, min((i+1)*C,
 * bytes)) of the device buffer dptr (16-byte aligned); hashes is a device
 * array of ceil(bytes/C) entries; C = chunk_bytes as for snap_opts.  Runs on
 * `stream` (cudaStream_t, NULL = legacy default) and waits for it.  Uses
 * library-owned device scratch (allocated on the first call per device). */
SNAP_API int snap_hash_chunks(const void *dptr, uint64_t bytes, uint64_t chunk_bytes,
                     uint32_t *hashes, void *stream);

/* Allocation-free chunk hasher (the paper has no counterpart: this serves
 * callers that cannot allocate GPU memory -- a checkpoint or crash handler
 * that must not touch the allocator whose state it is saving, a process
 * whose memory pool is exhausted or owned by another framework).  Hashes
 * n_buffers device buffers (each 16-byte aligned) in one launch: hashes (a
 * device array) receives the chunk hashes of buffer 0, then buffer 1, ...,
 * ceil(bytes[k]/chunk_bytes) entries each, as snap_hash_chunks would
 * produce buffer by buffer.  It calls no cudaMalloc/cudaFree/cudaHostAlloc:
 * its scratch is a fixed device array inside libsnap that every GPU using
 * the library keeps until the process exits.  Limits: n_buffers <=
 * SNAP_NOALLOC_MAX_BUFFERS, else SNAP_EINVAL with nothing launched.  The
 * first call on each device looks up that array (cudaGetSymbolAddress).
 * Calls share the array: two calls whose GPU work overlaps (other streams
 * or threads on the same device) race; this process's host calls are
 * serialised.  Every call copies its descriptor block from pageable host
 * memory onto `stream`, runs there, and synchronises `stream` before it
 * returns, so it must never be made while `stream` is being captured. */
#define SNAP_NOALLOC_MAX_BUFFERS 1024u
SNAP_API int snap_hash_chunks_noalloc(const void *const *dptrs, const uint64_t *bytes, uint32_t n_buffers,
                                      uint64_t chunk_bytes, uint32_t *hashes, void *stream);

/* Measure the rate at which SM loads and stores move bytes between device
 * memory and pinned, mapped host memory (direction 0: device to host, 1:
 * host to device, 2: both at once, half the warps each way; *gbs is then the
 * two directions' bytes together), best of `reps` launches over `bytes` per
 * direction (a multiple of 8 KiB is used).  This is the ceiling of the
 * gather and scatter kernels, which move the image with SM accesses, and
 * (direction 2) of a launch mixing them; on the measured B300 machines every SM
 * store form (16-byte stores, TMA bulk stores, plain load/store) reaches the
 * same rate, below the copy engines'.  Allocates and frees `bytes` (twice
 * that for direction 2) of device and pinned host memory.  device -1 = the
 * current device.  Errors: EINVAL, ENOMEM, ECUDA. */
SNAP_API int snap_link_ceiling(int device, int direction, uint64_t bytes, int reps, double *gbs);

/* Measure the host-memory side of staged transfers: `threads` host threads
 * copy `bytes` (rounded down to 4 KiB) between a pinned, mapped buffer and a
 * pageable one with the copy routine the ring and the server's workers use
 * (streaming stores) -- direction 0: pinned to pageable (a checkpoint
 * draining its slots), 1: pageable to pinned (a restore filling them), 2:
 * half the threads each way at once, *gbs counting both directions' bytes.
 * With with_link != 0 the GPU meanwhile moves bytes over the host link in
 * both directions with SM loads and stores (the host DRAM traffic the copies
 * share in the serving loop).  Best of `reps` rounds after a warm-up round.
 * Every byte staged through a slot costs host DRAM a read and a write for the
 * copy plus one access for the link transfer, so this bounds what staged
 * (pageable-image) checkpoints and restores can sustain.  Allocates and frees
 * `bytes` (twice that for direction 2) of pinned and of pageable memory, and
 * 2 GiB of each more with with_link, on the current device.  Errors: EINVAL,
 * ENOMEM, ECUDA. */
SNAP_API int snap_host_copy_ceiling(int threads, int direction, uint64_t bytes, int reps, int with_link,
                                    double *gbs);

/* ----------------------------------------------------------- autotuning */
typedef struct {
    uint32_t warps;        /* warps per CTA of the persistent kernel */
    uint32_t stages;       /* staging buffers per warp               */
    uint32_t piece_bytes;  /* bytes each lane stages per step        */
    uint32_t ctas_per_sm;
    double gbs;            /* measured throughput of the winner      */
    uint32_t chains;       /* hashing: CRC chains per lane (1 or 2)  */
    uint32_t tma;          /* hashing: 1 = stages loaded by 2D TMA tensor
                              copies, 0 = by per-lane cp.async       */
} snap_tuning;

/* Time the set's hash pass (mode SNAP_INCREMENTAL) or full gather (SNAP_FULL)
 * over a grid of launch shapes, adopt the fastest for this set, and record it
 * in the tuning cache keyed by (GPU name, operation, chunk size, state size
 * class = floor(log2(state bytes))); the cache file is $SNAP_TUNE_CACHE if
 * set (one JSON object per line, appended).  Every set reads that file when
 * its layout is built (the first call after registering) and starts with the
 * last shapes stored for its key, unless snap_opts.stages or hash_tma chose
 * the shape.  The device state is read, never modified.  host_image
 * (SNAP_FULL only) is a scratch image of snap_image_bytes(FULL) bytes in
 * snap_host_alloc memory. */
SNAP_API int snap_autotune(snap_set s, int mode, void *host_image, uint64_t cap, snap_tuning *out);

/* The launch shape the set uses for mode (SNAP_FULL: the gather;
 * SNAP_INCREMENTAL: the hash pass, which verify shares), after building its
 * layout; *out->gbs is 0.  Errors: EINVAL, EBUSY, ENOMEM, ECUDA. */
SNAP_API int snap_get_tuning(snap_set s, int mode, snap_tuning *out);

/* ------------------------------------------------------------- serving */
/* A request loop over many tenant sets: requests are admitted as pinned-host
 * and HBM budget frees up, and the chunk tiles of all admitted requests are
 * batched into shared persistent launches (continuous batching), so requests
 * that arrive while others run overlap on the device.  The server pins a
 * staging pool of o->ring_bytes (else $SNAP_SERVER_POOL_BYTES, else 8 GiB;
 * at most pinned_budget) in slots of up to 64 MiB, and runs 5 host copy
 * workers per 4 host threads ($SNAP_WORKERS overrides) to move window data
 * between the pool and the tenants' images.  o may be NULL (chunk_bytes,
 * timeout_ms and device as for snap_set_create).  Errors: EINVAL (zero
 * budget, bad chunk size), ENOMEM (pool), ECUDA. */
SNAP_API int snap_server_create(snap_server *out, uint64_t pinned_budget, uint64_t hbm_budget,
                       const snap_opts *o);
SNAP_API int snap_server_destroy(snap_server sv);
/* Queue a request on tenant set `tenant` (created on the server's device).
 * kind: SNAP_REQ_FULL / SNAP_REQ_INCREMENTAL write `image` (cap bytes);
 * SNAP_REQ_RESTORE reads it.  An image whose cap bytes lie in one pinned,
 * mapped region (snap_host_alloc, snap_host_register) is read and written
 * directly by the kernels and charges no staging; any other image is staged
 * through the server's pool by its copy workers.  *ticket identifies it.
 * EBUDGET if it can never be admitted under the budgets. */
SNAP_API int snap_server_submit(snap_server sv, snap_set tenant, int kind, void *image, uint64_t cap,
                       uint64_t *ticket);
/* Wait up to timeout_ms for a ticket; *status gets the request's own status,
 * st (may be NULL) its statistics with total_ms = arrival-to-completion
 * latency.  Returns ETIMEDOUT if it is still running. */
SNAP_API int snap_server_wait(snap_server sv, uint64_t ticket, uint32_t timeout_ms, int *status,
                     snap_stats *st);

/* ----------------------------------------------------------- coordination */
/* Several processes (one per GPU, each with its own set) take one consistent
 * checkpoint: every task is locked before any is checkpointed, and the
 * checkpoint counts only if every task completed it (Sec. 3.1: the lock and
 * checkpoint actions run for all tasks, and each plugin learns at exit
 * whether the whole operation succeeded; Sec. 4.4 / Table 3: data-parallel
 * replicas each store their own copy).  The transport between the ranks is
 * the caller's: `agree` combines the ranks' statuses (for example an
 * all-reduce taking the minimum) and returns the global one.
 *
 * snap_coordinate runs that two-phase protocol over caller-supplied local
 * steps (host code only; no GPU needed):
 *   st = lock();  g = agree(0, st);  if g != OK: return st ? st : EPEER
 *   st = run();   g = agree(1, st);  if g != OK: abort(); return st ? st : EPEER
 *   commit();     return OK
 * lock and run return a status; commit and abort cannot fail.  agree gets
 * the phase (0 or 1) and the local status and must return the same value on
 * every rank (a transport failure should be returned as a negative status,
 * for example ETIMEDOUT).  Any step but agree may be NULL (a no-op). */
typedef struct {
    int (*lock)(void *ctx);
    int (*run)(void *ctx);
    void (*commit)(void *ctx);
    void (*abort)(void *ctx);
    int (*agree)(void *ctx, int phase, int status);
} snap_coord_ops;
SNAP_API int snap_coordinate(const snap_coord_ops *ops, void *ctx);

/* snap_checkpoint as one rank of a coordinated checkpoint: lock = quiesce
 * (plus the argument checks), run = the checkpoint into host_image (pinned or
 * pageable) without committing, commit = the new hashes and generation become
 * the base, abort = they are discarded (the image buffer holds a checkpoint
 * no rank will use).  `agree` and `agree_ctx` as for snap_coordinate.
 * Returns OK only if every rank completed; EPEER if this rank did and another
 * did not. */
typedef int (*snap_agree_fn)(void *ctx, int phase, int status);
SNAP_API int snap_checkpoint_coordinated(snap_set s, void *host_image, uint64_t cap, int mode, uint64_t *used,
                                         snap_agree_fn agree, void *agree_ctx);

/* snap_restore as one rank of a coordinated restore: lock = validate the
 * image against the set (header, every record) and quiesce, so that a bad
 * image or a busy set on any rank stops every rank before any device byte
 * changes; run = the restore; commit = the image's hashes and generation
 * become the base; abort (another rank failed in its run) = the previous
 * base stays.  After a successful run the device holds the image's bytes
 * either way, and an incremental checkpoint against the previous base is
 * still exact.  Returns OK only if every rank completed; EPEER if this rank
 * did and another did not. */
SNAP_API int snap_restore_coordinated(const void *host_image, uint64_t bytes, snap_set s, snap_agree_fn agree,
                                      void *agree_ctx);

#ifdef __cplusplus
}
#endif
#endif /* SNAP_H */
