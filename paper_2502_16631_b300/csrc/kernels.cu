// Device kernels of libsnap (sm_103a): the persistent tile kernel.
//
// The hot path of a GPU checkpoint (CRIUgpu, Sec. 3.1.1: device memory is
// copied into host memory; restore copies it back) plus the chunk hashing
// that incremental checkpointing adds (Sec. 7).
//
// One persistent kernel (snap_tiles) serves every operation: each warp pulls
// (allocation, chunk) tiles from a device-side cursor across a list of jobs
// and runs the job's operation on its chunk:
//   OP_GATHER        TMA bulk copy HBM -> shared memory in 32*P-byte stages,
//                    CRC-32C from shared memory, 128-bit stores to the mapped
//                    host image (the device -> host link is the bound);
//   OP_HASH/VERIFY   staging of lane-contiguous segments in an XOR-swizzled,
//                    bank-conflict-free layout (128-bit cp.async by every
//                    lane, or one 2D TMA tensor copy per stage whose hardware
//                    swizzle is the same layout), CRC-32C per lane,
//                    warp-shuffle combine through GF(2) shift constants (HBM
//                    read is the bound);
//   OP_GATHER_DIRTY  the gather path without hashing, into patch slots;
//   OP_SCATTER       128-bit loads from the mapped host image, stores to HBM
//                    (host -> device link is the bound).
// CRC-32C lookups use slicing-by-4 tables replicated once per lane so that
// every lane reads its own shared-memory bank (lookups never conflict).
//
// Every wait is bounded: an mbarrier wait gives up after kWaitNs, records
// ERR_WAIT_TIMEOUT, drains the warp's outstanding copies (again bounded) and
// the warp leaves.  No wait depends on the host or on another kernel.
#include "snap_internal.h"
#include "crc32c_gf2.h"

namespace snapk {

__device__ const SliceTables g_slice = make_slice_tables();
__constant__ Pow8Table c_pow8 = make_pow8_table();

constexpr uint32_t kTableBytes = 4 * 256 * 32 * 4;     // 4 tables x 256 x 32 lanes
// Shared-window address of the first dynamic shared-memory byte, where the
// CRC tables start: the 1 KiB below it is reserved per CTA on sm_100-class
// GPUs.  Folding it into the lookups' immediate offsets saves an add per
// lookup; the kernel checks it at entry and refuses to run (ERR_SMEM_BASE)
// if a platform ever places dynamic shared memory elsewhere.
constexpr uint32_t kTableBase = 1024;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

size_t tile_smem_bytes(const TileShape &sh)
{
    return kTableBytes + (size_t)sh.warps * sh.stages * 32 * sh.chains * sh.piece +
           (size_t)sh.warps * sh.stages * 8 + (kMaxJobs + 1) * 8;
}

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t a, uint32_t tx)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(tx) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the completion of phase `parity` of the mbarrier at a.
__device__ __noinline__ bool mbar_wait_lane(uint32_t a, uint32_t parity)
{
    if (mbar_try(a, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try(a, parity)) return true;
        if (global_ns() - t0 > kWaitNs) return false;
        __nanosleep(128);
    }
}
// Warp-wide: every lane waits, and the warp agrees on the outcome so that
// control flow never diverges around the full-mask shuffles that follow.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity)
{
    const bool ok = mbar_wait_lane(a, parity);
    return __all_sync(0xFFFFFFFFu, ok);
}
__device__ __forceinline__ void tma_load_1d(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, uint64_t tmap, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}
// The tensor maps live in global memory and are rewritten between launches
// (the standalone hasher reuses one slot): make the tensor-map proxy see the
// latest contents before using one.
__device__ __forceinline__ void tmap_acquire(uint64_t tmap)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint32_t mbar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// ------------------------------------------------------------- CRC pieces
// Table layout (128 KiB): tables t = 2p + h (p = pair 0/1, h = half 0/1);
// entry (t, v) of lane l is the 32-bit word at byte offset
//     p * 65536 + v * 256 + h * 128 + l * 4,
// i.e. each 256-byte row holds one value of two tables for all 32 lanes, so
// a lane always reads its own bank, and the row offset v * 256 is a single
// byte-permute of the CRC register.  `lb` is the lane's 32-bit shared
// address of entry (0, 0); the pair/half part is an immediate offset.  In
// crc_word one byte-permute builds (v << 8) | (lane * 4) from the CRC
// register and `l4` = lane * 4, and the table base is part of the immediate,
// so a lookup is a permute and a load.
template <int OFF>
__device__ __forceinline__ uint32_t lds_tab(uint32_t addr)
{
    uint32_t v;
    asm("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(addr), "n"(OFF));
    return v;
}
__device__ __forceinline__ uint32_t crc_word(uint32_t crc, uint32_t w, uint32_t l4)
{
    const uint32_t x = crc ^ w;
    // byte 1 of each index = byte i of x (the row), byte 0 = lane * 4 (the
    // column), bytes 2-3 zero (byte 1 of l4)
    const uint32_t a3 = lds_tab<kTableBase + 65536 + 128>(__byte_perm(x, l4, 0x5504u));  // byte 0 -> table 3
    const uint32_t a2 = lds_tab<kTableBase + 65536>(__byte_perm(x, l4, 0x5514u));        // byte 1 -> table 2
    const uint32_t a1 = lds_tab<kTableBase + 128>(__byte_perm(x, l4, 0x5524u));          // byte 2 -> table 1
    const uint32_t a0 = lds_tab<kTableBase>(__byte_perm(x, l4, 0x5534u));                // byte 3 -> table 0
    return a0 ^ a1 ^ a2 ^ a3;
}
__device__ __forceinline__ uint32_t crc_byte(uint32_t crc, uint32_t b, uint32_t lb)
{
    return lds_tab<0>(lb + (((crc ^ b) & 0xFFu) << 8)) ^ (crc >> 8);
}
__device__ __forceinline__ uint32_t crc_block(uint32_t crc, const uint4 v, uint32_t l4)
{
    crc = crc_word(crc, v.x, l4);
    crc = crc_word(crc, v.y, l4);
    crc = crc_word(crc, v.z, l4);
    return crc_word(crc, v.w, l4);
}
__device__ __forceinline__ uint4 lds128(uint32_t addr)
{
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr)
                 : "memory");
    return v;
}
__device__ __forceinline__ uint32_t warp_xor(uint32_t v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v ^= __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ uint64_t up_page(uint64_t x) { return (x + 4095u) & ~uint64_t(4095u); }

// Warp-cooperative zero fill of host memory [p, p+n).
__device__ void warp_zero(uint8_t *p, uint64_t n, int lane)
{
    uint64_t head = (16u - ((uintptr_t)p & 15u)) & 15u;
    if (head > n) head = n;
    if ((uint64_t)lane < head) p[lane] = 0;
    p += head;
    n -= head;
    const uint64_t n16 = n >> 4;
    for (uint64_t q = lane; q < n16; q += 32) reinterpret_cast<uint4 *>(p)[q] = make_uint4(0, 0, 0, 0);
    const uint64_t rem = n & 15u;
    if ((uint64_t)lane < rem) p[(n16 << 4) + lane] = 0;
}

// ------------------------------------------------------------ warp state
struct WarpCtx {
    uint8_t *stage;        // this warp's stage buffers
    uint32_t mbar;         // shared address of its first mbarrier
    uint32_t issued;       // stages issued so far (per warp, across chunks)
    uint32_t consumed;     // stages consumed so far
    uint32_t ib, cb, cpar; // next buffer to issue / to consume, its phase parity
    int stages, piece, lane, chains;
    uint32_t lb;           // shared address of this lane's table column
    uint32_t l4;           // lane * 4 (the column offset inside a table row)
    bool tma;              // stage full chunks with TMA tensor copies where possible
    uint64_t tmap_seen;    // the tensor map this warp last acquired
    uint32_t stage_bytes;  // 32 * chains * piece
};

// The stage ring is walked with incremental counters (no division by the
// runtime stage count): issue takes buffer ib; the next stage to consume is
// buffer cb, whose mbarrier phase parity is cpar.
__device__ __forceinline__ uint32_t issue_advance(WarpCtx &w)
{
    const uint32_t b = w.ib;
    w.ib = (b + 1u == (uint32_t)w.stages) ? 0u : b + 1u;
    ++w.issued;
    return b;
}
__device__ __forceinline__ void cons_advance(WarpCtx &w)
{
    if (++w.cb == (uint32_t)w.stages) {
        w.cb = 0u;
        w.cpar ^= 1u;
    }
    ++w.consumed;
}

// Wait (bounded) for every issued, unconsumed stage: used when giving up.
__device__ void drain(WarpCtx &w)
{
    while (w.consumed < w.issued) {
        (void)mbar_wait(w.mbar + 8 * w.cb, w.cpar);
        cons_advance(w);
    }
}

// Test hook (Job.test_stall): take a stage and expect 16 bytes on its
// mbarrier that no copy will deliver, then wait for it.  Nothing is in flight
// for this warp at a tile's start (every chunk routine consumes the stages it
// issues), so the barrier is the next one to consume; its bounded wait runs
// out and the caller's error path (ERR_WAIT_TIMEOUT, drain, leave) runs with
// no copy outstanding.
__device__ bool stall_stage(WarpCtx &w)
{
    const uint32_t buf = issue_advance(w);
    const uint32_t mb = w.mbar + 8 * buf;
    if (w.lane == 0) mbar_arrive_tx(mb, 16u);
    else mbar_arrive(mb);
    return mbar_wait(w.mbar + 8 * w.cb, w.cpar);
}

// ------------------------------------------- segmented hash (HBM-bound path)
// Lane l owns bytes [l*s, min((l+1)*s, L)) of the chunk; stage k holds the
// next P bytes of every lane's segment in slot l (slot j at j*P).  Inside a
// slot, 16-byte unit u is stored at unit u ^ swz(j): the 8 lanes of a
// quarter-warp reading unit u of 8 consecutive slots then hit 8 different
// 16-byte bank groups, and so do the copies that fill them, with no padding.
// Each cp.async instruction of the warp moves four whole 128-byte lines.
template <uint32_t BPP>
__device__ __forceinline__ uint32_t swz(uint32_t j)
{
    if constexpr (BPP == 1) return 0u;
    else if constexpr (BPP == 2) return (j >> 2) & 1u;
    else if constexpr (BPP == 4) return (j >> 1) & 3u;
    else return j & 7u;
}
__device__ __forceinline__ uint32_t swz_rt(uint32_t j, uint32_t bpp)
{
    return bpp >= 8u ? (j & 7u) : bpp == 4u ? ((j >> 1) & 3u) : bpp == 2u ? ((j >> 2) & 1u) : 0u;
}

__device__ __forceinline__ void seg_issue(WarpCtx &w, const uint8_t *src, uint32_t L, uint32_t s, uint32_t k)
{
    const uint32_t buf = issue_advance(w);
    const uint32_t P = (uint32_t)w.piece;
    uint8_t *sb = w.stage + buf * w.stage_bytes;
    const uint32_t sbs = smem_addr(sb);
    const uint32_t bpp = P >> 4;  // 16-byte blocks per piece
    for (uint32_t m = 0; m < bpp; ++m) {
        const uint32_t q = m * 32u + (uint32_t)w.lane;
        const uint32_t j = q / bpp, b = q - j * bpp;
        const uint32_t plo = j * s + k * P;
        uint32_t phi = plo + P;
        const uint32_t seg_hi = j * s + s;
        if (phi > seg_hi) phi = seg_hi;
        if (phi > L) phi = L;
        if (plo + 16u * b + 16u <= phi) cp_async16(sbs + j * P + 16u * (b ^ swz_rt(j, bpp)), src + plo + 16u * b);
    }
    cp_async_arrive(w.mbar + 8 * buf);
}

// Full chunk (L == C, C/32 a multiple of P): the copy plan of every stage is
// the same up to a k*P offset, so each lane keeps one source and one
// destination base; the CRC loop over the piece is fully unrolled.
template <int P>
__device__ bool hash_full_chunk(WarpCtx &w, const uint8_t *src, uint32_t C, const CombineConsts &cc, uint32_t &out,
                                uint64_t tmap, uint32_t row0)
{
    constexpr uint32_t BPP = P / 16;    // 16-byte blocks per piece
    constexpr uint32_t PPI = 32 / BPP;  // pieces covered by one warp instruction
    const uint32_t lane = (uint32_t)w.lane;
    const uint32_t s = C >> 5;
    const uint32_t nst = s / P;
    const uint32_t jl = lane / BPP, bl = lane % BPP;
    const uint8_t *sp0 = src + jl * s + 16u * bl;
    const uint32_t stage0 = smem_addr(w.stage);
    const uint32_t S = (uint32_t)w.stages;
    const uint32_t rsw = swz<BPP>(lane);
    uint32_t crc = lane == 0 ? 0xFFFFFFFFu : 0u;

    // stage k: one TMA box (P bytes of each of the 32 segment rows, placed
    // with the hardware swizzle) when the allocation has a tensor map, else
    // cp.async copies by every lane into the same swizzled layout
    auto issue = [&](uint32_t k) {
        const uint32_t buf = issue_advance(w);
        const uint32_t sbs = stage0 + buf * w.stage_bytes;
        const uint32_t mb = w.mbar + 8 * buf;
        if (tmap) {
            if (lane == 0) {
                mbar_arrive_tx(mb, 32u * P);
                tma_load_2d(sbs, tmap, (int)(k * P), (int)row0, mb);
            } else {
                mbar_arrive(mb);
            }
            return;
        }
#pragma unroll
        for (uint32_t m = 0; m < BPP; ++m) {
            const uint32_t j = jl + m * PPI;
            cp_async16(sbs + j * P + 16u * (bl ^ swz<BPP>(j)), sp0 + m * PPI * s + k * P);
        }
        cp_async_arrive(mb);
    };
    // the stages were last touched through the generic proxy: order that
    // before the TMA writes into them
    if (tmap) {
        fence_proxy_async();
        if (tmap != w.tmap_seen) {  // once per map per warp and launch
            if (lane == 0) tmap_acquire(tmap);
            w.tmap_seen = tmap;
        }
    }
    const uint32_t pre = nst < S ? nst : S;
    for (uint32_t k = 0; k < pre; ++k) issue(k);
    for (uint32_t k = 0; k < nst; ++k) {
        const uint32_t buf = w.cb;
        if (!mbar_wait(w.mbar + 8 * buf, w.cpar)) return false;
        cons_advance(w);
        const uint32_t rd = stage0 + buf * w.stage_bytes + lane * P;
#pragma unroll
        for (uint32_t b = 0; b < BPP; ++b) crc = crc_block(crc, lds128(rd + 16u * (b ^ rsw)), w.l4);
        __syncwarp();
        if (k + S < nst) {
            if (tmap) fence_proxy_async();
            issue(k + S);
        }
    }
    out = warp_xor(gf2_mulmod(crc, cc.kseg[lane])) ^ 0xFFFFFFFFu;
    return true;
}

// Full chunk with two independent CRC chains per lane: the chunk is cut
// into 64 segments of C/64 bytes; lane l hashes segments l and l+32, so
// every lane has two lookup chains in flight.  A stage holds the next P
// bytes of all 64 segments (slot v at v*(P+16), conflict-free reads).
template <int P>
__device__ bool hash_full_chunk2(WarpCtx &w, const uint8_t *src, uint32_t C, const CombineConsts &cc, uint32_t &out)
{
    constexpr uint32_t BPP = P / 16;    // 16-byte blocks per piece
    constexpr uint32_t PPI = 32 / BPP;  // pieces covered by one warp instruction
    constexpr uint32_t NI = 64 / PPI;   // copy instructions per stage
    const uint32_t lane = (uint32_t)w.lane;
    const uint32_t s = C >> 6;
    const uint32_t nst = s / P;
    const uint32_t jl = lane / BPP, bl = lane % BPP;
    const uint8_t *sp0 = src + jl * s + 16u * bl;
    const uint32_t stage0 = smem_addr(w.stage);
    const uint32_t S = (uint32_t)w.stages;
    const uint32_t rsw = swz<BPP>(lane);  // = swz(lane + 32)
    uint32_t ca = lane == 0 ? 0xFFFFFFFFu : 0u, cb = 0u;

    auto issue = [&](uint32_t k) {
        const uint32_t buf = issue_advance(w);
        const uint32_t sbs = stage0 + buf * w.stage_bytes;
#pragma unroll
        for (uint32_t m = 0; m < NI; ++m) {
            const uint32_t j = jl + m * PPI;
            cp_async16(sbs + j * P + 16u * (bl ^ swz<BPP>(j)), sp0 + m * PPI * s + k * P);
        }
        cp_async_arrive(w.mbar + 8 * buf);
    };
    const uint32_t pre = nst < S ? nst : S;
    for (uint32_t k = 0; k < pre; ++k) issue(k);
    for (uint32_t k = 0; k < nst; ++k) {
        const uint32_t buf = w.cb;
        if (!mbar_wait(w.mbar + 8 * buf, w.cpar)) return false;
        cons_advance(w);
        const uint32_t ra = stage0 + buf * w.stage_bytes + lane * P;
        const uint32_t rb = ra + 32u * P;
#pragma unroll
        for (uint32_t b = 0; b < BPP; ++b) {
            const uint4 va = lds128(ra + 16u * (b ^ rsw));
            const uint4 vb = lds128(rb + 16u * (b ^ rsw));
            ca = crc_block(ca, va, w.l4);
            cb = crc_block(cb, vb, w.l4);
        }
        __syncwarp();
        if (k + S < nst) issue(k + S);
    }
    const uint32_t v = gf2_mulmod(ca, cc.kseg2[lane]) ^ gf2_mulmod(cb, cc.kseg2[lane + 32]);
    out = warp_xor(v) ^ 0xFFFFFFFFu;
    return true;
}

// The chunk's CRC-32C lands in `out` in every lane; false if a wait gave up.
// tmap_base: the allocation's tensor maps (0: none); row0 = 32 x the
// chunk's index in its allocation (its first segment row).
__device__ bool hash_chunk_seg(WarpCtx &w, const uint8_t *src, uint32_t L, uint32_t C, const CombineConsts &cc,
                               uint32_t &out, uint64_t tmap_base, uint32_t row0)
{
    if (w.chains == 2 && L == C && ((C >> 6) % (uint32_t)w.piece) == 0u) {
        switch (w.piece) {
        case 32: return hash_full_chunk2<32>(w, src, C, cc, out);
        case 64: return hash_full_chunk2<64>(w, src, C, cc, out);
        case 128: return hash_full_chunk2<128>(w, src, C, cc, out);
        default: break;
        }
    }
    if (L == C && ((C >> 5) % (uint32_t)w.piece) == 0u) {
        const uint64_t tb = tmap_base;
        switch (w.piece) {
        case 32: return hash_full_chunk<32>(w, src, C, cc, out, tb ? tb : 0, row0);
        case 64: return hash_full_chunk<64>(w, src, C, cc, out, tb ? tb + kTmapBytes : 0, row0);
        case 128: return hash_full_chunk<128>(w, src, C, cc, out, tb ? tb + 2 * kTmapBytes : 0, row0);
        case 256: return hash_full_chunk<256>(w, src, C, cc, out, 0, row0);
        default: break;
        }
    }
    const int lane = w.lane;
    const uint32_t P = (uint32_t)w.piece;
    const uint32_t s = (L == C) ? (C >> 5) : ((((L + 31u) >> 5) + 15u) & ~15u);
    const uint32_t nst = (s + P - 1) / P;
    uint32_t lo = (uint32_t)lane * s;
    if (lo > L) lo = L;
    uint32_t hi = lo + s;
    if (hi > L) hi = L;
    uint32_t crc = lane == 0 ? 0xFFFFFFFFu : 0u;

    const uint32_t pre = nst < (uint32_t)w.stages ? nst : (uint32_t)w.stages;
    for (uint32_t k = 0; k < pre; ++k) seg_issue(w, src, L, s, k);
    for (uint32_t k = 0; k < nst; ++k) {
        const uint32_t buf = w.cb;
        if (!mbar_wait(w.mbar + 8 * buf, w.cpar)) return false;
        cons_advance(w);
        const uint32_t plo = lo + k * P;
        if (plo < hi) {
            const uint32_t phi = plo + P < hi ? plo + P : hi;
            const uint32_t rd = smem_addr(w.stage + buf * w.stage_bytes) + (uint32_t)lane * P;
            const uint32_t rsw = swz_rt((uint32_t)lane, P >> 4);
            const uint32_t nfull = (phi - plo) >> 4;
            if (nfull == (P >> 4)) {
#pragma unroll 4
                for (uint32_t b = 0; b < (P >> 4); ++b) crc = crc_block(crc, lds128(rd + 16u * (b ^ rsw)), w.l4);
            } else {
                for (uint32_t b = 0; b < nfull; ++b) crc = crc_block(crc, lds128(rd + 16u * (b ^ rsw)), w.l4);
            }
            const uint32_t rem = (phi - plo) & 15u;
            if (rem) {
                const uint8_t *tp = src + plo + (nfull << 4);
                for (uint32_t r = 0; r < rem; ++r) crc = crc_byte(crc, __ldg(tp + r), w.lb);
            }
        }
        __syncwarp();
        if (k + (uint32_t)w.stages < nst) seg_issue(w, src, L, s, k + (uint32_t)w.stages);
    }
    uint32_t v = 0;
    if (lo < L) {
        const uint32_t K = (L == C) ? cc.kseg[lane] : gf2_x8n(L - hi, c_pow8);
        v = gf2_mulmod(crc, K);
    }
    out = warp_xor(v) ^ 0xFFFFFFFFu;
    return true;
}

// ------------------------------------ interleaved gather (link-bound path)
// Stage k is the contiguous range [k*32P, (k+1)*32P) of the chunk, moved by
// one TMA bulk copy; lane l hashes its piece [k*32P + l*P, +P), so its pieces
// are 31*P bytes apart (the gap is shifted in with the constant kgap), and
// the warp stores the stage to the host as contiguous 512-byte rows.
__device__ __forceinline__ void int_issue(WarpCtx &w, const uint8_t *src, uint32_t L, uint32_t k)
{
    const uint32_t buf = issue_advance(w);
    const uint32_t SB = 32u * (uint32_t)w.piece;
    const uint32_t mb = w.mbar + 8 * buf;
    if (w.lane == 0) {
        const uint32_t lo = k * SB;
        const uint32_t slen = (L - lo) < SB ? (L - lo) : SB;
        const uint32_t n16 = slen & ~15u;
        mbar_arrive_tx(mb, n16);
        if (n16) tma_load_1d(smem_addr(w.stage + buf * w.stage_bytes), src + lo, n16, mb);
    } else {
        mbar_arrive(mb);
    }
}

__device__ bool gather_chunk_int(WarpCtx &w, const uint8_t *src, uint32_t L, uint32_t C, bool do_hash,
                                 uint8_t *dst, const CombineConsts &cc, uint32_t &out)
{
    const int lane = w.lane;
    const uint32_t P = (uint32_t)w.piece;
    const uint32_t SB = 32u * P;
    const uint32_t nst = (L + SB - 1) / SB;
    uint32_t crc = lane == 0 ? 0xFFFFFFFFu : 0u;
    uint32_t e = 0;  // end of this lane's last hashed piece

    const uint32_t pre = nst < (uint32_t)w.stages ? nst : (uint32_t)w.stages;
    // the buffers were last touched through the generic proxy (reads, or
    // cp.async writes of a hashed chunk): order that before the TMA writes
    fence_proxy_async();
    for (uint32_t k = 0; k < pre; ++k) int_issue(w, src, L, k);
    for (uint32_t k = 0; k < nst; ++k) {
        const uint32_t buf = w.cb;
        if (!mbar_wait(w.mbar + 8 * buf, w.cpar)) return false;
        cons_advance(w);
        const uint8_t *sb = w.stage + buf * w.stage_bytes;
        const uint32_t slo = k * SB;
        const uint32_t slen = (L - slo) < SB ? (L - slo) : SB;
        const uint32_t n16 = slen & ~15u;
        if (do_hash) {
            const uint32_t plo = slo + (uint32_t)lane * P;
            if (plo < L) {
                const uint32_t phi = plo + P < L ? plo + P : L;
                const uint32_t gap = plo - e;
                if (crc != 0u && gap != 0u) crc = gf2_mulmod(crc, gap == 31u * P ? cc.kgap : gf2_x8n(gap, c_pow8));
                const uint4 *sp = reinterpret_cast<const uint4 *>(sb + (uint32_t)lane * P);
                const uint32_t nfull = (phi - plo) >> 4;
                for (uint32_t b = 0; b < nfull; ++b) crc = crc_block(crc, sp[b], w.l4);
                const uint32_t rem = (phi - plo) & 15u;
                if (rem) {
                    const uint8_t *tp = src + plo + (nfull << 4);
                    for (uint32_t r = 0; r < rem; ++r) crc = crc_byte(crc, __ldg(tp + r), w.lb);
                }
                e = phi;
            }
        }
        // stage -> host as contiguous 16-byte columns of the warp
        const uint4 *s4 = reinterpret_cast<const uint4 *>(sb);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst + slo);
        const uint32_t nb = n16 >> 4;
        for (uint32_t q = (uint32_t)lane; q < nb; q += 32u) d4[q] = s4[q];
        if (slen != n16 && lane == 0)
            for (uint32_t r = n16; r < slen; ++r) dst[slo + r] = __ldg(src + slo + r);
        __syncwarp();
        if (k + (uint32_t)w.stages < nst) {
            fence_proxy_async();
            int_issue(w, src, L, k + (uint32_t)w.stages);
        }
    }
    if (do_hash) {
        uint32_t v = 0;
        if (e != 0u) {
            const uint32_t K = (L == C && C % SB == 0u) ? cc.kint[lane] : gf2_x8n(L - e, c_pow8);
            v = gf2_mulmod(crc, K);
        }
        out = warp_xor(v) ^ 0xFFFFFFFFu;
    }
    return true;
}

// ------------------------------------------------- scatter (host -> device)
__device__ void scatter_chunk(const uint8_t *src, uint8_t *dst, uint32_t L, int lane)
{
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    const uint32_t nb = L >> 4;
    constexpr uint32_t U = 8;
    uint32_t q = (uint32_t)lane;
    for (; q + 32u * (U - 1) < nb; q += 32u * U) {
        uint4 v[U];
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) v[u] = s4[q + 32u * u];
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) d4[q + 32u * u] = v[u];
    }
    for (; q < nb; q += 32u) d4[q] = s4[q];
    const uint32_t rem = L & 15u;
    if ((uint32_t)lane < rem) dst[(nb << 4) + lane] = src[(nb << 4) + lane];
}

// Largest k with a[k].chunk0 <= chunk (ties: the largest index, so that
// zero-byte allocations, which own no chunk, are never chosen).
__device__ __forceinline__ uint64_t find_alloc(const AllocDesc *a, uint64_t n, uint64_t chunk)
{
    uint64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a[mid].chunk0 <= chunk) lo = mid; else hi = mid;
    }
    return lo;
}

// ------------------------------------------ fused incremental: the roles
// Wait (one thread) until *p >= v, bounded by kWaitNs; false if the wait
// ran out (ERR_WAIT_TIMEOUT recorded) or another CTA recorded an error.
__device__ bool fused_wait(const unsigned long long *p, unsigned long long v, Result *kres)
{
    const volatile unsigned long long *vp = p;
    const volatile unsigned long long *verr = &kres->err;
    if (*vp >= v) {
        __threadfence();
        return true;
    }
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (*vp >= v) break;
        if (*verr) return false;
        if (global_ns() - t0 > kWaitNs) {
            atomicOr(&kres->err, (unsigned long long)ERR_WAIT_TIMEOUT);
            return false;
        }
        __nanosleep(200);
    }
    __threadfence();  // what the producer wrote before its release is visible
    return true;
}

// Exclusive scan of one value per thread over the CTA (any multiple of 32
// threads up to 1024); *total = the sum.  ws: 33 words of shared memory.
__device__ unsigned long long cta_exscan(unsigned long long v, unsigned long long *total, unsigned long long *ws)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long t = lane < nw ? ws[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) ws[lane] = t;  // inclusive over warps
        if (lane == nw - 1) ws[32] = t;
    }
    __syncthreads();
    const unsigned long long r = (warp ? ws[warp - 1] : 0ull) + x - v;
    *total = ws[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ uint64_t lower_bound_list(const uint32_t *a, uint64_t n, uint64_t key)
{
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if ((uint64_t)a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// The group of a chunk: the last g with gch[g] <= chunk (an empty group
// shares its start with the next one, which then owns the chunk).
__device__ __forceinline__ int fused_group(const FusedIncr &f, uint64_t chunk)
{
    int lo = 0, hi = f.n_groups;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (f.gch[mid] <= chunk) lo = mid; else hi = mid;
    }
    return lo;
}

// Copy-engine form, metadata CTA: list group g's dirty runs (dirty entries
// [beg, end) of the ascending list, laid out already) after the *nruns runs
// of earlier groups, then publish the group to the host: entries first,
// then its begin and count, then, after a system-scope fence, ready = 1.
// A run is a maximal range of consecutive dirty chunks of one allocation;
// its patch slots are contiguous (a full chunk fills its C-byte slot), so
// one copy moves it.  With `use` false (the patch would pass the image
// capacity) the group is published with no runs.
__device__ void fused_list_runs(const Job &jb, FusedIncr &f, int g, unsigned long long beg,
                                unsigned long long end, bool use, unsigned long long *nruns,
                                unsigned long long *ws)
{
    const uint64_t C = jb.chunk_bytes;
    const unsigned long long first = *nruns;
    // starts and ends listed so far: a run may start in one pass of the loop
    // and end in a later one, so each side keeps its own count
    unsigned long long n = first, ne = first;
    for (unsigned long long base = beg; use && base < end; base += blockDim.x) {
        const unsigned long long r = base + threadIdx.x;
        bool st = false, en = false;
        uint64_t k = 0, i = 0, slot = 0, L = 0;
        if (r < end) {
            const uint64_t c = f.dlist[r];
            k = find_alloc(jb.allocs, jb.n_allocs, c);
            const AllocDesc a = jb.allocs[k];
            const uint64_t nk = (a.bytes + C - 1) / C;
            i = c - a.chunk0;
            st = r == beg || f.dlist[r - 1] + 1 != c || i == 0;
            en = r + 1 == end || f.dlist[r + 1] != c + 1 || i + 1 == nk;
            slot = f.patch_data[k] + (r - f.dstart[k]) * C;
            L = (a.bytes - i * C) < C ? (a.bytes - i * C) : C;
        }
        unsigned long long ts, te;
        const unsigned long long xs = cta_exscan(st ? 1ull : 0ull, &ts, ws);
        const unsigned long long xe = cta_exscan(en ? 1ull : 0ull, &te, ws);
        // the i-th start and the i-th end of the list belong to the same run
        if (st && n + xs < f.runs_cap) {
            DirtyRun *d = f.runs + n + xs;
            d->alloc = k;
            d->chunk = i;
            d->dst0 = slot;
        }
        if (en && ne + xe < f.runs_cap) f.runs[ne + xe].dst1 = slot + L;
        n += ts;
        ne += te;
    }
    __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile RunGroup *p = f.pub + g;
        p->begin = first;
        p->count = n - first;
        __threadfence_system();
        p->ready = 1ull;
    }
    *nruns = n;
}

// The metadata role (one CTA): per group, in order, once its chunks are
// hashed: the dirty list (ascending, continuing the running count), the
// patch layout of its allocations (continuing the running offset; the
// layout snap_format.h states), their records, hashes and dirty indices
// written into the patch, then the group is released to the gather CTAs.
__device__ void fused_meta(const Job &jb, FusedIncr &f, unsigned long long *ws, Result *kres)
{
    const uint64_t C = jb.chunk_bytes;
    const uint32_t *cur = jb.hash_out;
    unsigned long long run = 0;    // dirty entries listed so far
    unsigned long long off = 64;   // patch offset of the next record
    unsigned long long nruns = 0;  // copy-engine form: dirty runs listed so far
    if (threadIdx.x == 0) kres->ts[TS_DIFF_END] = global_ns();  // the whole pipeline is copy time
    for (int g = 0; g < f.n_groups; ++g) {
        const uint64_t c0 = f.gch[g], c1 = f.gch[g + 1];
        if (threadIdx.x == 0) ws[34] = fused_wait(&f.grp_done[g], c1 - c0, kres) ? 1ull : 0ull;
        __syncthreads();
        const bool ok = ws[34] != 0;
        __syncthreads();
        if (!ok) return;
        if (g + 1 == f.n_groups && threadIdx.x == 0) kres->ts[TS_HASH_END] = global_ns();
        // the group's dirty chunks, ascending
        const unsigned long long beg = run;
        for (uint64_t base = c0; base < c1; base += blockDim.x) {
            const uint64_t c = base + threadIdx.x;
            // other SMs wrote these hashes during this launch: read them at L2, never from a stale L1 line
            const bool d = c < c1 && __ldcg(cur + c) != f.prev[c];
            unsigned long long tot;
            const unsigned long long ex = cta_exscan(d ? 1ull : 0ull, &tot, ws);
            if (d) f.dlist[run + ex] = (uint32_t)c;
            run += tot;
        }
        __syncthreads();  // the list is complete for every thread
        // the layout of the group's allocations
        const uint64_t a0 = f.gal[g], a1 = f.gal[g + 1];
        for (uint64_t base = a0; base < a1; base += blockDim.x) {
            const uint64_t k = base + threadIdx.x;
            unsigned long long R = 0, meta_pad = 0, ds = 0;
            if (k < a1) {
                const AllocDesc a = jb.allocs[k];
                const uint64_t nk = (a.bytes + C - 1) / C;
                ds = lower_bound_list(f.dlist, run, a.chunk0);
                const uint64_t de = lower_bound_list(f.dlist, run, a.chunk0 + nk);
                const uint64_t nd = de - ds;
                uint64_t data = nd * C;
                if (nd && f.dlist[de - 1] == a.chunk0 + nk - 1) data = data - C + up_page(a.bytes - (nk - 1) * C);
                const uint64_t meta = 32 + 4 * nk + 4 + 4 * nd;
                meta_pad = (k == 0) ? up_page(64 + meta) - 64 : up_page(meta);
                R = meta_pad + data;
            }
            unsigned long long tot;
            const unsigned long long ex = cta_exscan(R, &tot, ws);
            if (k < a1) {
                f.patch_rec[k] = off + ex;
                f.patch_data[k] = off + ex + meta_pad;
                f.dstart[k] = ds;
            }
            off += tot;
        }
        if (threadIdx.x == 0) f.dstart[a1] = run;
        __syncthreads();
        // records, hashes, dirty indices and padding of the group's
        // allocations, one warp per allocation
        if (off <= f.cap) {
            const unsigned lane = threadIdx.x & 31u, nwarps = blockDim.x >> 5;
            for (uint64_t k = a0 + (threadIdx.x >> 5); k < a1; k += nwarps) {
                const AllocDesc a = jb.allocs[k];
                const uint64_t nk = (a.bytes + C - 1) / C;
                const uint64_t rec = f.patch_rec[k], data = f.patch_data[k];
                const uint64_t ds = f.dstart[k], nd = f.dstart[k + 1] - ds;
                uint64_t *r64 = reinterpret_cast<uint64_t *>(f.host + rec);
                if (lane < 4) r64[lane] = lane == 0 ? a.bytes : lane == 1 ? nk : lane == 2 ? data : 0ull;
                uint32_t *h = reinterpret_cast<uint32_t *>(f.host + rec + 32);
                for (uint64_t i = lane; i < nk; i += 32) h[i] = __ldcg(cur + a.chunk0 + i);
                if (lane == 0) h[nk] = (uint32_t)nd;
                for (uint64_t j = lane; j < nd; j += 32) h[nk + 1 + j] = f.dlist[ds + j] - (uint32_t)a.chunk0;
                const uint64_t zlo = rec + 36 + 4 * nk + 4 * nd;
                uint32_t *z = reinterpret_cast<uint32_t *>(f.host + zlo);
                const uint64_t nz = (data - zlo) / 4;
                for (uint64_t q = lane; q < nz; q += 32) z[q] = 0u;
                // copy-engine form: the copies carry data bytes only, so the
                // padding after a dirty partial last chunk is zeroed here
                if (f.dma && nd) {
                    const uint64_t Ll = a.bytes - (nk - 1) * C;
                    if ((Ll & 4095u) && f.dlist[ds + nd - 1] == a.chunk0 + nk - 1)
                        warp_zero(f.host + data + (nd - 1) * C + Ll, up_page(Ll) - Ll, lane);
                }
            }
        }
        __syncthreads();
        if (f.dma) {
            fused_list_runs(jb, f, g, beg, run, off <= f.cap, &nruns, ws);
            continue;
        }
        if (threadIdx.x == 0) {
            f.gbeg[g] = beg;
            f.gcnt[g] = off <= f.cap ? run - beg : 0ull;  // over capacity: nothing is gathered
            __threadfence();
            atomicExch(&f.meta_ready[g], 1ull);
        }
    }
    if (threadIdx.x == 0) {
        kres->n_dirty = run;
        kres->patch_bytes = off;
        if (off > f.cap) kres->cap_exceeded = 1ull;
    }
}

// The gather role: per group, in order, once its metadata is written, every
// warp takes dirty chunks from the group's cursor and copies each into its
// patch slot with 16-byte loads and stores (eight in flight per lane), then
// zeroes the slot's padding.  The checks are the tile loop's for a dirty
// gather: the chunk inside its allocation, its rank inside the allocation's
// range of the list, 16-byte aligned addresses (else ERR_BAD_TILE, skipped).
__device__ void fused_gather(const Job &jb, FusedIncr &f, Result *kres)
{
    const int lane = threadIdx.x & 31;
    const uint64_t C = jb.chunk_bytes;
    for (int g = 0; g < f.n_groups; ++g) {
        int ok = 1;
        if (lane == 0) ok = fused_wait(&f.meta_ready[g], 1ull, kres) ? 1 : 0;
        if (!__shfl_sync(0xFFFFFFFFu, ok, 0)) return;
        const unsigned long long n = *reinterpret_cast<volatile unsigned long long *>(&f.gcnt[g]);
        const unsigned long long beg = *reinterpret_cast<volatile unsigned long long *>(&f.gbeg[g]);
        for (;;) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(&f.gcur[g], 1ull);
            t = __shfl_sync(0xFFFFFFFFu, t, 0);
            if (t >= n) break;
            // the list and the layout were written by the metadata CTA during
            // this launch: read them at L2
            const unsigned long long rank = beg + t;
            const uint64_t chunk = __ldcg(f.dlist + rank);
            const uint64_t k = find_alloc(jb.allocs, jb.n_allocs, chunk);
            const AllocDesc a = jb.allocs[k];
            const uint64_t nk = (a.bytes + C - 1) / C;
            const uint64_t i = chunk - a.chunk0;
            const uint64_t ds = __ldcg(reinterpret_cast<const unsigned long long *>(f.dstart) + k);
            const uint64_t de = __ldcg(reinterpret_cast<const unsigned long long *>(f.dstart) + k + 1);
            bool bad = chunk < a.chunk0 || i >= nk || rank < ds || rank >= de;
            const uint64_t off = i * C;
            const uint64_t L = bad ? 0 : ((a.bytes - off) < C ? (a.bytes - off) : C);
            const uint8_t *src = reinterpret_cast<const uint8_t *>(a.ptr) + off;
            uint8_t *dst = f.host + __ldcg(reinterpret_cast<const unsigned long long *>(f.patch_data) + k) + (rank - ds) * C;
            if (!bad) bad = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) != 0;
            if (bad) {  // the same for every lane
                if (lane == 0) atomicOr(&kres->err, (unsigned long long)ERR_BAD_TILE);
                continue;
            }
            const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
            uint4 *d4 = reinterpret_cast<uint4 *>(dst);
            const uint64_t nb = L >> 4;
            constexpr uint32_t U = 8;
            uint64_t q = (uint64_t)lane;
            for (; q + 32u * (U - 1) < nb; q += 32u * U) {
                uint4 v[U];
#pragma unroll
                for (uint32_t u = 0; u < U; ++u) v[u] = s4[q + 32u * u];
#pragma unroll
                for (uint32_t u = 0; u < U; ++u) d4[q + 32u * u] = v[u];
            }
            for (; q < nb; q += 32u) d4[q] = s4[q];
            const uint64_t rem = L & 15u;
            if ((uint64_t)lane < rem) dst[(nb << 4) + lane] = src[(nb << 4) + lane];
            if (L & 4095u) warp_zero(dst + L, up_page(L) - L, lane);
        }
    }
}

// -------------------------------------------------------------- main kernel
// HASH_ONLY instantiation: only OP_HASH / OP_VERIFY jobs, up to 32 warps per
// CTA (1024 threads, so at most 64 registers a thread) to keep more lookup
// chains in flight; the general one serves every op with up to 16 warps.
template <bool HASH_ONLY>
__global__ void __launch_bounds__(HASH_ONLY ? kMaxHashWarps * 32 : kMaxWarps * 32, 1)
snap_tiles(const Job *__restrict__ jobs, int n_jobs, int n_jobs_a, unsigned long long *cursor,
           unsigned long long *cursor_b, const CombineConsts cc, int stages, int piece, int chains, int tma,
           Result *kres)
{
    // Jobs [0, n_jobs_a) form group A (device -> host work), jobs
    // [n_jobs_a, n_jobs) group B (host -> device work); each group has its own
    // tile cursor, even warps start on A and odd warps on B, and a warp
    // whose group runs dry switches to the other, so a launch that mixes
    // checkpoints and restores drives both link directions at once.
    extern __shared__ __align__(1024) uint8_t smem[];
    uint32_t *tables = reinterpret_cast<uint32_t *>(smem);
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t stage_bytes = 32u * (uint32_t)chains * (uint32_t)piece;
    uint8_t *stage_all = smem + kTableBytes;
    uint64_t *mbars = reinterpret_cast<uint64_t *>(stage_all + (size_t)warps * stages * stage_bytes);
    unsigned long long *prefix = reinterpret_cast<unsigned long long *>(mbars + warps * stages);

    // a fused incremental checkpoint's metadata CTA and gather CTAs (the CTA
    // index decides the role of the whole CTA)
    if (n_jobs == 1 && jobs[0].fused && (int)blockIdx.x >= jobs[0].fused->n_hash_ctas) {
        FusedIncr &f = *jobs[0].fused;
        if ((int)blockIdx.x == f.n_hash_ctas)
            fused_meta(jobs[0], f, reinterpret_cast<unsigned long long *>(stage_all), kres);
        else
            fused_gather(jobs[0], f, kres);
        return;
    }

    // the lookups assume the tables at kTableBase; the condition is the same
    // for every thread, so the whole CTA leaves together
    if (smem_addr(tables) != kTableBase) {
        if (threadIdx.x == 0) atomicOr(&kres->err, (unsigned long long)ERR_SMEM_BASE);
        return;
    }
    bool need_tables = false;
    for (int j = 0; j < n_jobs; ++j)
        need_tables |= (jobs[j].op == OP_HASH || jobs[j].op == OP_GATHER || jobs[j].op == OP_VERIFY);
    if (need_tables)
        for (int i = threadIdx.x; i < 32768; i += blockDim.x) {
            // word i: pair i>>14, row (i>>6)&255, half (i>>5)&1, lane i&31
            const int t = ((i >> 14) << 1) | ((i >> 5) & 1);
            tables[i] = g_slice.t[t][(i >> 6) & 255];
        }
    if (lane == 0)
        for (int s = 0; s < stages; ++s) mbar_init(smem_addr(&mbars[warp * stages + s]), 32);
    if (threadIdx.x == 0) {
        prefix[0] = 0;
        for (int j = 0; j < n_jobs; ++j) {
            const Job &jb = jobs[j];
            const unsigned long long n = jb.n_tiles_dev ? *jb.n_tiles_dev : jb.n_tiles;
            prefix[j + 1] = prefix[j] + n;
        }
    }
    fence_mbar_init();
    __syncthreads();
    const unsigned long long total = prefix[n_jobs];
    const unsigned long long tot_a = cursor_b ? prefix[n_jobs_a] : total;
    const unsigned long long tot_b = total - tot_a;
    bool done_a = tot_a == 0, done_b = tot_b == 0;
    int grp = (tot_b != 0 && (warp & 1)) ? 1 : 0;

    WarpCtx w;
    w.stage = stage_all + (size_t)warp * stages * stage_bytes;
    w.mbar = smem_addr(&mbars[warp * stages]);
    w.issued = w.consumed = 0;
    w.ib = w.cb = w.cpar = 0;
    w.stages = stages;
    w.piece = piece;
    w.chains = chains;
    w.tma = tma != 0;
    w.tmap_seen = 0;
    w.lane = lane;
    w.lb = smem_addr(tables) + 4u * (uint32_t)lane;
    w.l4 = 4u * (uint32_t)lane;
    w.stage_bytes = stage_bytes;

    for (;;) {
        if (done_a && done_b) break;
        if (grp == 0 && done_a) grp = 1;
        if (grp == 1 && done_b) grp = 0;
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(grp ? cursor_b : cursor, 1ull);
        v = __shfl_sync(0xFFFFFFFFu, v, 0);
        if (v >= (grp ? tot_b : tot_a)) {
            if (grp) done_b = true; else done_a = true;
            // every tile of this launch is taken: a launch queued behind it
            // with programmatic stream serialization (which reads nothing
            // this one writes) may now take the SMs its CTAs free
            if (done_a && done_b && lane == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
            continue;
        }
        const unsigned long long t = grp ? tot_a + v : v;
        // another warp gave up: stop (lane 0 reads, the warp follows it)
        unsigned long long err = lane == 0 ? *reinterpret_cast<volatile unsigned long long *>(&kres->err) : 0ull;
        if (__shfl_sync(0xFFFFFFFFu, err, 0)) break;
        int j = 0;
        while (j + 1 < n_jobs && prefix[j + 1] <= t) ++j;
        const Job &jb = jobs[j];
        const unsigned long long tt = t - prefix[j];
        // a list job may start at a device-side position of its list
        const unsigned long long toff = jb.tile_off_dev ? *jb.tile_off_dev : 0ull;
        const uint64_t chunk = jb.tile_list ? (uint64_t)jb.tile_list[tt + toff] : jb.tile_begin + tt;
        const uint64_t k = find_alloc(jb.allocs, jb.n_allocs, chunk);
        const AllocDesc ad = jb.allocs[k];
        const uint64_t C = jb.chunk_bytes;
        const uint64_t i = chunk - ad.chunk0;
        const uint64_t nk = (ad.bytes + C - 1) / C;
        if (chunk < ad.chunk0 || i >= nk) {
            if (lane == 0) atomicOr(&kres->err, (unsigned long long)ERR_BAD_TILE);
            break;
        }
        const uint64_t off = i * C;
        const uint32_t L = (uint32_t)((ad.bytes - off) < C ? (ad.bytes - off) : C);
        const uint8_t *dsrc = reinterpret_cast<const uint8_t *>(ad.ptr) + off;
        uint8_t *host_data = jb.layout == LAYOUT_IMAGE ? jb.host + ad.data_off + off
                                                       : jb.host + (ad.state_off + off - jb.window_off);
        // every 16-byte access below needs 16-byte aligned device and host
        // addresses; a misaligned tile is recorded and skipped, never issued
        if ((((uintptr_t)dsrc | (uintptr_t)host_data) & 15u) && jb.op != OP_HASH && jb.op != OP_VERIFY) {
            if (lane == 0) atomicOr(&kres->err, (unsigned long long)ERR_BAD_TILE);
            break;
        }
        if (((uintptr_t)dsrc & 15u) != 0u) {
            if (lane == 0) atomicOr(&kres->err, (unsigned long long)ERR_BAD_TILE);
            break;
        }
        bool ok = true;
        uint32_t h = 0;
        if (jb.test_stall == tt + 1) {
            ok = stall_stage(w);
            if (ok && lane == 0) atomicOr(&kres->err, (unsigned long long)ERR_BAD_TILE);  // cannot happen
            if (!ok) {
                if (lane == 0) atomicOr(&kres->err, (unsigned long long)ERR_WAIT_TIMEOUT);
                drain(w);
            }
            break;
        }
        switch (jb.op) {
        case OP_HASH:
        case OP_VERIFY:
            ok = hash_chunk_seg(w, dsrc, L, (uint32_t)C, cc, h, w.tma ? ad.tmap : 0ull, (uint32_t)(i * 32u));
            if (ok && lane == 0) {
                if (jb.hash_out) jb.hash_out[chunk] = h;
                if (jb.op == OP_VERIFY && jb.hash_cmp[chunk] != h) {
                    atomicAdd(&jb.res->mismatches, 1ull);
                    atomicMin(&jb.res->first_bad, (unsigned long long)chunk);
                }
                if (jb.fused) {  // release the hash to the metadata CTA
                    __threadfence();
                    atomicAdd(&jb.fused->grp_done[fused_group(*jb.fused, chunk)], 1ull);
                }
            }
            break;
        case OP_GATHER:
            if (HASH_ONLY) {
                if (lane == 0) atomicOr(&kres->err, (unsigned long long)ERR_BAD_TILE);
                break;
            }
            ok = gather_chunk_int(w, dsrc, L, (uint32_t)C, true, host_data, cc, h);
            if (ok) {
                if (lane == 0) {
                    if (jb.hash_out) jb.hash_out[chunk] = h;
                    if (jb.layout == LAYOUT_IMAGE) *reinterpret_cast<uint32_t *>(jb.host + ad.rec_off + 32 + 4 * i) = h;
                }
                if (jb.layout == LAYOUT_IMAGE && i + 1 == nk) {
                    const uint64_t end = ad.data_off + ad.bytes;
                    warp_zero(jb.host + end, up_page(end) - end, lane);
                }
            }
            break;
        case OP_GATHER_DIRTY: {
            if (HASH_ONLY) {
                if (lane == 0) atomicOr(&kres->err, (unsigned long long)ERR_BAD_TILE);
                break;
            }
            if (jb.cap_exceeded && *reinterpret_cast<volatile const unsigned long long *>(jb.cap_exceeded)) break;
            // IMAGE: the chunk's slot in the patch (dirty rank window_off +
            // toff + tt, which must fall in its allocation's dirty range);
            // PACKED: slot tt of a ring window of C-byte slots
            const unsigned long long rank = jb.window_off + toff + tt;
            if (jb.layout == LAYOUT_IMAGE && (rank < jb.dstart[k] || rank >= jb.dstart[k + 1])) {
                if (lane == 0) atomicOr(&kres->err, (unsigned long long)ERR_BAD_TILE);
                break;
            }
            uint8_t *dst = jb.layout == LAYOUT_IMAGE ? jb.host + jb.patch_data[k] + (rank - jb.dstart[k]) * C
                                                     : jb.host + tt * C;
            ok = gather_chunk_int(w, dsrc, L, (uint32_t)C, false, dst, cc, h);
            if (ok && (L & 4095u)) warp_zero(dst + L, up_page(L) - L, lane);
            break;
        }
        case OP_SCATTER:
            if (HASH_ONLY) {
                if (lane == 0) atomicOr(&kres->err, (unsigned long long)ERR_BAD_TILE);
                break;
            }
            scatter_chunk(host_data, reinterpret_cast<uint8_t *>(ad.ptr) + off, L, lane);
            break;
        default:
            break;
        }
        if (!ok) {
            if (lane == 0) atomicOr(&kres->err, (unsigned long long)ERR_WAIT_TIMEOUT);
            drain(w);
            break;
        }
    }
}

cudaError_t launch_tiles2(const Job *jobs_dev, int n_jobs, int n_jobs_a, unsigned long long *cursor_a,
                          unsigned long long *cursor_b, const CombineConsts &cc, const TileShape &sh, Result *kres,
                          cudaStream_t st, bool overlap_prev)
{
    const size_t smem = tile_smem_bytes(sh);
    // more than kMaxWarps warps selects the hash/verify-only kernel
    if (smem > kMaxSmem || sh.warps < 1 || sh.warps > kMaxHashWarps || n_jobs < 1 || n_jobs > kMaxJobs)
        return cudaErrorInvalidValue;
    if (n_jobs_a < 0 || n_jobs_a > n_jobs || (n_jobs_a < n_jobs && !cursor_b)) return cudaErrorInvalidValue;
    if (sh.chains < 1 || sh.chains > 2 || sh.stages < 1 || sh.piece < 32 || sh.piece > 256 || (sh.piece & 15))
        return cudaErrorInvalidValue;
    if (overlap_prev) {
        // programmatic stream serialization: this launch's CTAs may start
        // once every CTA of the previous kernel on `st` has run out of
        // tiles, i.e. in that kernel's tail
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)sh.ctas);
        cfg.blockDim = dim3((unsigned)sh.warps * 32u);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at{};
        at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at.val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = &at;
        cfg.numAttrs = 1;
        if (sh.warps > kMaxWarps)
            return cudaLaunchKernelEx(&cfg, snap_tiles<true>, jobs_dev, n_jobs, n_jobs_a, cursor_a, cursor_b, cc,
                                      sh.stages, sh.piece, sh.chains, sh.tma, kres);
        return cudaLaunchKernelEx(&cfg, snap_tiles<false>, jobs_dev, n_jobs, n_jobs_a, cursor_a, cursor_b, cc,
                                  sh.stages, sh.piece, sh.chains, sh.tma, kres);
    }
    if (sh.warps > kMaxWarps)
        snap_tiles<true><<<sh.ctas, sh.warps * 32, smem, st>>>(jobs_dev, n_jobs, n_jobs_a, cursor_a, cursor_b, cc,
                                                               sh.stages, sh.piece, sh.chains, sh.tma, kres);
    else
        snap_tiles<false><<<sh.ctas, sh.warps * 32, smem, st>>>(jobs_dev, n_jobs, n_jobs_a, cursor_a, cursor_b, cc,
                                                                sh.stages, sh.piece, sh.chains, sh.tma, kres);
    return cudaGetLastError();
}

cudaError_t launch_fused_incr(const Job *job_dev, unsigned long long *cursor, const CombineConsts &cc,
                              const TileShape &sh, int grid, Result *kres, cudaStream_t st)
{
    const size_t smem = tile_smem_bytes(sh);
    if (smem > kMaxSmem || sh.warps < 1 || sh.warps > kMaxHashWarps || grid < 3) return cudaErrorInvalidValue;
    if (sh.chains < 1 || sh.chains > 2 || sh.stages < 1 || sh.piece < 32 || sh.piece > 256 || (sh.piece & 15))
        return cudaErrorInvalidValue;
    // the metadata CTA's scan words live in the staging area
    if ((size_t)sh.warps * sh.stages * 32 * sh.chains * sh.piece < 35 * sizeof(unsigned long long))
        return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)sh.warps * 32u);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at{};
    at.id = cudaLaunchAttributeCooperative;  // every CTA resident: the roles wait on one another
    at.val.cooperative = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    unsigned long long *none = nullptr;
    if (sh.warps > kMaxWarps)
        return cudaLaunchKernelEx(&cfg, snap_tiles<true>, job_dev, 1, 1, cursor, none, cc, sh.stages, sh.piece,
                                  sh.chains, sh.tma, kres);
    return cudaLaunchKernelEx(&cfg, snap_tiles<false>, job_dev, 1, 1, cursor, none, cc, sh.stages, sh.piece, sh.chains,
                              sh.tma, kres);
}

bool fused_incr_fits(const TileShape &sh, int grid, int device)
{
    int coop = 0, sms = 0, per = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const size_t smem = tile_smem_bytes(sh);
    const cudaError_t e =
        sh.warps > kMaxWarps
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, snap_tiles<true>, sh.warps * 32, smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, snap_tiles<false>, sh.warps * 32, smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return coop != 0 && (long)per * sms >= grid;
}

cudaError_t launch_tiles(const Job *jobs_dev, int n_jobs, unsigned long long *cursor, const CombineConsts &cc,
                         const TileShape &sh, Result *kres, cudaStream_t st, bool overlap_prev)
{
    return launch_tiles2(jobs_dev, n_jobs, n_jobs, cursor, nullptr, cc, sh, kres, st, overlap_prev);
}

// Opt the kernel into the full shared-memory carve-out; call once per
// device, outside any stream capture.
cudaError_t init_tile_kernel()
{
    cudaError_t e = cudaFuncSetAttribute(snap_tiles<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(snap_tiles<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    return e;
}

CombineConsts make_combine_consts(uint64_t C, int piece)
{
    static constexpr Pow8Table pw = make_pow8_table();
    CombineConsts cc{};
    const uint64_t s = C / 32;
    const uint64_t P = (uint64_t)piece;
    for (int l = 0; l < 32; ++l) {
        cc.kseg[l] = gf2_x8n(C - (uint64_t)(l + 1) * s, pw);
        cc.kint[l] = gf2_x8n((uint64_t)(31 - l) * P, pw);
    }
    for (int v = 0; v < 64; ++v) cc.kseg2[v] = gf2_x8n(C - (uint64_t)(v + 1) * (C / 64), pw);
    cc.kgap = gf2_x8n(31 * P, pw);
    return cc;
}

}  // namespace snapk
