// Host-side merge of an incremental patch into its base full image
// (snap_apply_patch).  The patch records carry every new hash and the
// ascending list of dirty chunks followed by their bytes (snap_format.h);
// the merge copies each dirty chunk into its slot in the base, replaces the
// hash arrays and advances the header to the patch's generation.  Both
// images are validated completely before the base is touched, so a bad
// patch leaves the base as it was (CRIUgpu Sec. 3.1: roll back on failure).
#include "snap.h"
#include "snap_format.h"
#include "runtime_internal.h"

#include <cstring>
#include <new>
#include <vector>

namespace snapk {

static inline uint64_t upg(uint64_t x) { return (x + 4095u) & ~uint64_t(4095u); }

namespace {
struct FullRec {
    uint64_t bytes, n, data_off, hash_off;
};
struct PatchRec {
    uint64_t n, data_off, hash_off, idx_off;
    uint32_t nd;
};
}  // namespace

int apply_patch_host(uint8_t *base, uint64_t base_len, const uint8_t *patch, uint64_t patch_len)
{
    if (!base || !patch) return SNAP_EINVAL;
    ImageHeader hb{}, hp{};
    int rc = parse_header(base, base_len, &hb);
    if (rc) return rc;
    rc = parse_header(patch, patch_len, &hp);
    if (rc) return rc;
    if ((hb.flags & SNAP_IMG_FLAG_INCREMENTAL) || !(hp.flags & SNAP_IMG_FLAG_INCREMENTAL)) return SNAP_EFORMAT;
    if (hp.chunk_bytes != hb.chunk_bytes || hp.n_allocs != hb.n_allocs || hp.total != hb.total)
        return SNAP_EMISMATCH;
    if (hp.parent != hb.generation) return SNAP_EMISMATCH;
    const uint64_t C = hb.chunk_bytes;
    // The allocation count sizes the tables below, so it is bounded first:
    // every record of a full image takes at least its 32-byte header, and a
    // header claiming more allocations than the base can hold is malformed.
    if (hb.n_allocs > (base_len - SNAP_IMG_HEADER_BYTES) / 32) return SNAP_EFORMAT;
    std::vector<FullRec> fr;
    std::vector<PatchRec> pr;
    try {
        fr.resize(hb.n_allocs);
        pr.resize(hb.n_allocs);
    } catch (...) {  // no exception leaves the C ABI
        return SNAP_ENOMEM;
    }

    // validate the base
    uint64_t off = SNAP_IMG_HEADER_BYTES, total = 0;
    for (uint64_t k = 0; k < hb.n_allocs; ++k) {
        if (off + 32 > base_len) return SNAP_EFORMAT;
        uint64_t r[4];
        std::memcpy(r, base + off, 32);
        const uint64_t n = (r[0] + C - 1) / C;
        if (r[1] != n || r[3] != 0 || n > (base_len - off - 32) / 4) return SNAP_EFORMAT;
        if (r[2] != upg(off + 32 + 4 * n) || r[2] > base_len || r[0] > base_len - r[2]) return SNAP_EFORMAT;
        fr[k] = FullRec{r[0], n, r[2], off + 32};
        total += r[0];
        off = upg(r[2] + r[0]);
    }
    if (off > base_len || total != hb.total) return SNAP_EFORMAT;

    // validate the patch against the base
    off = SNAP_IMG_HEADER_BYTES;
    for (uint64_t k = 0; k < hp.n_allocs; ++k) {
        if (off + 36 > patch_len) return SNAP_EFORMAT;
        uint64_t r[4];
        std::memcpy(r, patch + off, 32);
        if (r[0] != fr[k].bytes) return SNAP_EMISMATCH;
        const uint64_t n = fr[k].n;
        if (r[1] != n || r[3] != 0 || n > (patch_len - off - 36) / 4) return SNAP_EFORMAT;
        uint32_t nd;
        std::memcpy(&nd, patch + off + 32 + 4 * n, 4);
        if (nd > n || off + 36 + 4 * n + 4ull * nd > patch_len) return SNAP_EFORMAT;
        if (r[2] != upg(off + 36 + 4 * n + 4ull * nd)) return SNAP_EFORMAT;
        pr[k] = PatchRec{n, r[2], off + 32, off + 36 + 4 * n, nd};
        uint64_t d = r[2];
        int64_t last = -1;
        for (uint32_t j = 0; j < nd; ++j) {
            uint32_t i;
            std::memcpy(&i, patch + pr[k].idx_off + 4ull * j, 4);
            if (i >= n || (int64_t)i <= last) return SNAP_EFORMAT;
            last = i;
            const uint64_t L = std::min<uint64_t>(C, fr[k].bytes - (uint64_t)i * C);
            if (d > patch_len || L > patch_len - d) return SNAP_EFORMAT;
            d += upg(L);
        }
        off = d;
    }
    if (off > patch_len) return SNAP_EFORMAT;

    // merge
    for (uint64_t k = 0; k < hb.n_allocs; ++k) {
        uint64_t d = pr[k].data_off;
        for (uint32_t j = 0; j < pr[k].nd; ++j) {
            uint32_t i;
            std::memcpy(&i, patch + pr[k].idx_off + 4ull * j, 4);
            const uint64_t L = std::min<uint64_t>(C, fr[k].bytes - (uint64_t)i * C);
            std::memcpy(base + fr[k].data_off + (uint64_t)i * C, patch + d, L);
            d += upg(L);
        }
        std::memcpy(base + fr[k].hash_off, patch + pr[k].hash_off, 4 * fr[k].n);
    }
    write_header(base, SNAP_IMG_FLAG_DEVICE_STATE, C, hb.n_allocs, hb.total, hp.generation, 0);
    return SNAP_OK;
}

}  // namespace snapk
