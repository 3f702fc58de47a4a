/*
 * snap oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU restatement of what the GPU
 * snapshot/restore path computes.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file's library; the product
 * library never links, includes or calls it, and it shares no code, header,
 * table or constant generator with the CUDA path.
 *
 * What it restates (paper: CRIUgpu, arXiv 2502.16631):
 *   - checkpoint: device state is copied into a host-memory image
 *     (Sec. 3.1.1, "checkpoint" action); the image carries a flag saying it
 *     holds GPU state so restore can check compatibility (Sec. 3.1.1, last
 *     paragraph);
 *   - restore: device memory is put back byte for byte (Sec. 3.1.1,
 *     "restore" action; Sec. 6 "Deterministic Restore");
 *   - incremental checkpointing is named as an optimisation that could be
 *     incorporated (Sec. 7, Check-N-Run); the hash-diff scheme below is the
 *     one this library defines for it.
 * The checksum is CRC-32C (Castagnoli), reflected, init 0xFFFFFFFF,
 * final xor 0xFFFFFFFF, as defined for iSCSI (RFC 3720, Sec. 12.1 / B.4);
 * check value of "123456789" is 0xE3069283.
 *
 * Everything here is written out in the order the definitions state it:
 * one byte at a time for the CRC, one allocation at a time for the image.
 * The only concurrency is orc_set_threads(): chunks are independent by
 * definition, so hashing them on several threads changes nothing.
 *
 * Parity pins (see tests/): the check value; a bit-at-a-time CRC; the x86
 * SSE4.2 crc32 instruction; GF(2) polynomial division in Python integers;
 * RFC 3720 B.4 vectors; image round trip; patch-apply == full image.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>
#include <pthread.h>

/* ---------------------------------------------------------------- status */
/* Status values of the public C ABI, restated here (not included). */
#define ORC_OK         0
#define ORC_EINVAL    -1
#define ORC_ENOMEM    -2
#define ORC_EFORMAT   -6
#define ORC_EMISMATCH -7

/* ----------------------------------------------------------------- CRC32C */
/* Castagnoli polynomial 0x1EDC6F41; in the reflected (LSB-first) bit order
 * the CRC register uses, its coefficients x^31..x^0 read backwards give
 * 0x82F63B78. */
#define ORC_POLY_REFLECTED 0x82F63B78u

static uint32_t orc_table[256];
static int orc_table_ready = 0;
static pthread_once_t orc_once = PTHREAD_ONCE_INIT;

/* Table entry b = the register after shifting byte b through it eight bits
 * at a time with the reflected polynomial: the classic byte-wise table. */
static void orc_make_table(void)
{
    for (uint32_t b = 0; b < 256; ++b) {
        uint32_t r = b;
        for (int k = 0; k < 8; ++k)
            r = (r & 1u) ? (r >> 1) ^ ORC_POLY_REFLECTED : (r >> 1);
        orc_table[b] = r;
    }
    orc_table_ready = 1;
}

static void orc_init(void) { pthread_once(&orc_once, orc_make_table); }

/* Raw register update: feed n bytes into register value c (no init, no
 * final xor).  c' = T[(c ^ byte) & 0xFF] ^ (c >> 8), byte by byte. */
uint32_t orc_crc32c_update(uint32_t c, const uint8_t *p, uint64_t n)
{
    orc_init();
    for (uint64_t i = 0; i < n; ++i)
        c = orc_table[(c ^ p[i]) & 0xFFu] ^ (c >> 8);
    return c;
}

/* CRC-32C of a message: init all-ones, final xor all-ones. */
uint32_t orc_crc32c(const uint8_t *p, uint64_t n)
{
    return orc_crc32c_update(0xFFFFFFFFu, p, n) ^ 0xFFFFFFFFu;
}

/* ---------------------------------------------------------------- chunking */
/* Allocation of `bytes` bytes has ceil(bytes / C) chunks; chunk i covers
 * [i*C, min((i+1)*C, bytes)).  The last chunk is hashed over its real
 * length (no padding).  A zero-byte allocation has no chunks. */
uint64_t orc_n_chunks(uint64_t bytes, uint64_t C)
{
    return C ? (bytes + C - 1) / C : 0;
}

static int orc_threads = 1;
void orc_set_threads(int n) { orc_threads = n < 1 ? 1 : (n > 256 ? 256 : n); }
int orc_get_threads(void) { return orc_threads; }

typedef struct {
    const uint8_t *p; uint64_t bytes, C; uint32_t *out;
    uint64_t first, last;   /* chunk range [first, last) */
} orc_hash_job;

static void *orc_hash_worker(void *arg)
{
    orc_hash_job *j = (orc_hash_job *)arg;
    for (uint64_t i = j->first; i < j->last; ++i) {
        uint64_t lo = i * j->C;
        uint64_t hi = lo + j->C < j->bytes ? lo + j->C : j->bytes;
        j->out[i] = orc_crc32c(j->p + lo, hi - lo);
    }
    return NULL;
}

/* out[i] = CRC-32C of chunk i of the allocation. */
void orc_chunk_hashes(const uint8_t *p, uint64_t bytes, uint64_t C, uint32_t *out)
{
    orc_init();
    uint64_t n = orc_n_chunks(bytes, C);
    int t = orc_threads;
    if ((uint64_t)t > n) t = (int)(n ? n : 1);
    if (t <= 1) {
        orc_hash_job j = {p, bytes, C, out, 0, n};
        orc_hash_worker(&j);
        return;
    }
    pthread_t th[256];
    orc_hash_job jobs[256];
    for (int k = 0; k < t; ++k) {
        jobs[k] = (orc_hash_job){p, bytes, C, out, n * k / t, n * (k + 1) / t};
        pthread_create(&th[k], NULL, orc_hash_worker, &jobs[k]);
    }
    for (int k = 0; k < t; ++k) pthread_join(th[k], NULL);
}

/* ------------------------------------------------------------ image layout */
/* Little-endian image.  64-byte header:
 *   0  magic "SNAPIMG1"          8  u32 version (1)     12 u32 flags
 *   16 u64 chunk_bytes           24 u64 n_allocs        32 u64 total_state_bytes
 *   40 u64 generation            48 u64 parent_generation
 *   56 u32 CRC-32C of bytes 0..55                       60 u32 zero
 * flags: bit0 = incremental patch, bit1 = holds device state.
 * Full image, per allocation k in registration order:
 *   32-byte record header {u64 bytes_k, u64 n_k, u64 data_offset_k, u64 0},
 *   u32 hash[n_k], zero pad to a 4096-byte boundary,
 *   bytes_k data bytes at data_offset_k, zero pad to a 4096-byte boundary.
 * Patch, per allocation k:
 *   the same record header, all n_k new hashes, u32 n_dirty_k,
 *   u32 idx[n_dirty_k] (ascending chunk indices), zero pad to 4096,
 *   then each dirty chunk's bytes in index order, each padded to 4096. */
#define ORC_PAGE 4096u
#define ORC_HDR 64u
#define ORC_REC 32u
#define ORC_FLAG_INCR 1u
#define ORC_FLAG_DEV 2u
static const char orc_magic[8] = {'S','N','A','P','I','M','G','1'};

static uint64_t orc_up(uint64_t x) { return (x + ORC_PAGE - 1) / ORC_PAGE * ORC_PAGE; }

static void orc_put32(uint8_t *p, uint32_t v) { for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i)); }
static void orc_put64(uint8_t *p, uint64_t v) { for (int i = 0; i < 8; ++i) p[i] = (uint8_t)(v >> (8 * i)); }
static uint32_t orc_get32(const uint8_t *p) { uint32_t v = 0; for (int i = 3; i >= 0; --i) v = (v << 8) | p[i]; return v; }
static uint64_t orc_get64(const uint8_t *p) { uint64_t v = 0; for (int i = 7; i >= 0; --i) v = (v << 8) | p[i]; return v; }

static int orc_valid_chunk(uint64_t C) { return C >= ORC_PAGE && C % ORC_PAGE == 0 && C <= (1ull << 30); }

/* Bytes of a full image for these allocation sizes. */
uint64_t orc_image_bytes(uint64_t n, const uint64_t *sizes, uint64_t C)
{
    uint64_t off = ORC_HDR;
    for (uint64_t k = 0; k < n; ++k) {
        off = orc_up(off + ORC_REC + 4 * orc_n_chunks(sizes[k], C));
        off = orc_up(off + sizes[k]);
    }
    return off;
}

static void orc_write_header(uint8_t *h, uint32_t flags, uint64_t C, uint64_t n,
                             uint64_t total, uint64_t gen, uint64_t parent)
{
    memset(h, 0, ORC_HDR);
    memcpy(h, orc_magic, 8);
    orc_put32(h + 8, 1);
    orc_put32(h + 12, flags);
    orc_put64(h + 16, C);
    orc_put64(h + 24, n);
    orc_put64(h + 32, total);
    orc_put64(h + 40, gen);
    orc_put64(h + 48, parent);
    orc_put32(h + 56, orc_crc32c(h, 56));
}

/* Write the bytes [lo, hi) of the full image of n allocations into
 * out[0..cap): lo = 0 when k0 == 0 (the header is included), else the
 * offset of record k0; hi = the end of record k1 - 1 (the header's end when
 * k1 == 0).  Those are exactly the bytes the whole image holds there; only
 * data[k0..k1) is read (data[k] for k outside may be NULL), so an image too
 * large for memory can be produced and compared record by record.
 * *lo_out = lo, *used = hi - lo. */
int orc_write_full_window(uint64_t n, const uint8_t *const *data, const uint64_t *sizes,
                          uint64_t C, uint64_t generation, uint64_t k0, uint64_t k1,
                          uint8_t *out, uint64_t cap, uint64_t *lo_out, uint64_t *used)
{
    if (!orc_valid_chunk(C) || k0 > k1 || k1 > n) return ORC_EINVAL;
    uint64_t lo = k0 ? orc_image_bytes(k0, sizes, C) : 0;
    uint64_t hi = orc_image_bytes(k1, sizes, C);
    if (cap < hi - lo) return ORC_EINVAL;
    memset(out, 0, hi - lo);
    if (k0 == 0) {
        uint64_t total = 0;
        for (uint64_t k = 0; k < n; ++k) total += sizes[k];
        orc_write_header(out, ORC_FLAG_DEV, C, n, total, generation, 0);
    }
    uint64_t off = k0 ? lo : ORC_HDR;   /* image offset of record k */
    for (uint64_t k = k0; k < k1; ++k) {
        uint64_t nk = orc_n_chunks(sizes[k], C);
        uint64_t data_off = orc_up(off + ORC_REC + 4 * nk);
        uint8_t *rec = out + (off - lo);
        orc_put64(rec, sizes[k]);
        orc_put64(rec + 8, nk);
        orc_put64(rec + 16, data_off);
        orc_put64(rec + 24, 0);
        /* hashes are stored little-endian: compute, then serialise */
        uint32_t *h = (uint32_t *)malloc(4 * (nk ? nk : 1));
        if (!h) return ORC_ENOMEM;
        orc_chunk_hashes(data[k], sizes[k], C, h);
        for (uint64_t i = 0; i < nk; ++i) orc_put32(rec + ORC_REC + 4 * i, h[i]);
        free(h);
        memcpy(out + (data_off - lo), data[k], sizes[k]);
        off = orc_up(data_off + sizes[k]);
    }
    *lo_out = lo;
    *used = hi - lo;
    return ORC_OK;
}

/* Write the full image of n allocations into out[0..cap): the window of
 * every record. */
int orc_write_full(uint64_t n, const uint8_t *const *data, const uint64_t *sizes,
                   uint64_t C, uint64_t generation, uint8_t *out, uint64_t cap,
                   uint64_t *used)
{
    uint64_t lo = 0;
    return orc_write_full_window(n, data, sizes, C, generation, 0, n, out, cap, &lo, used);
}

/* Parsed view of an image (full or patch). */
typedef struct {
    uint32_t flags;
    uint64_t C, n, total, generation, parent;
} orc_header;

static int orc_parse_header(const uint8_t *img, uint64_t len, orc_header *h)
{
    if (len < ORC_HDR) return ORC_EFORMAT;
    if (memcmp(img, orc_magic, 8) != 0) return ORC_EFORMAT;
    if (orc_get32(img + 8) != 1) return ORC_EFORMAT;
    if (orc_get32(img + 56) != orc_crc32c(img, 56)) return ORC_EFORMAT;
    if (orc_get32(img + 60) != 0) return ORC_EFORMAT;
    h->flags = orc_get32(img + 12);
    h->C = orc_get64(img + 16);
    h->n = orc_get64(img + 24);
    h->total = orc_get64(img + 32);
    h->generation = orc_get64(img + 40);
    h->parent = orc_get64(img + 48);
    if (!(h->flags & ORC_FLAG_DEV) || (h->flags & ~3u)) return ORC_EFORMAT;
    if (!orc_valid_chunk(h->C)) return ORC_EFORMAT;
    return ORC_OK;
}

/* Header fields of an image, for tests: returns status. out6 =
 * {flags, C, n, total, generation, parent}. */
int orc_read_header(const uint8_t *img, uint64_t len, uint64_t *out6)
{
    orc_header h;
    int rc = orc_parse_header(img, len, &h);
    if (rc) return rc;
    out6[0] = h.flags; out6[1] = h.C; out6[2] = h.n; out6[3] = h.total;
    out6[4] = h.generation; out6[5] = h.parent;
    return ORC_OK;
}

/* Walk a full image's records; checks every field against the layout rule
 * and the expected sizes (if sizes != NULL).  data_off[k] receives the data
 * offset of allocation k, hash_off[k] the offset of its hash array. */
static int orc_walk_full(const uint8_t *img, uint64_t len, const orc_header *h,
                         uint64_t n_expect, const uint64_t *sizes,
                         uint64_t *data_off, uint64_t *hash_off)
{
    if (h->flags & ORC_FLAG_INCR) return ORC_EFORMAT;
    if (sizes && h->n != n_expect) return ORC_EMISMATCH;
    uint64_t off = ORC_HDR, total = 0;
    for (uint64_t k = 0; k < h->n; ++k) {
        if (off + ORC_REC > len) return ORC_EFORMAT;
        const uint8_t *rec = img + off;
        uint64_t bk = orc_get64(rec), nk = orc_get64(rec + 8), dk = orc_get64(rec + 16);
        if (orc_get64(rec + 24) != 0) return ORC_EFORMAT;
        if (sizes && bk != sizes[k]) return ORC_EMISMATCH;
        if (nk != orc_n_chunks(bk, h->C)) return ORC_EFORMAT;
        if (nk > (len - off) / 4) return ORC_EFORMAT;
        uint64_t expect = orc_up(off + ORC_REC + 4 * nk);
        if (dk != expect) return ORC_EFORMAT;
        if (dk > len || bk > len - dk) return ORC_EFORMAT;
        if (data_off) data_off[k] = dk;
        if (hash_off) hash_off[k] = off + ORC_REC;
        total += bk;
        off = orc_up(dk + bk);
    }
    if (off > len) return ORC_EFORMAT;
    if (total != h->total) return ORC_EFORMAT;
    return ORC_OK;
}

/* Restore: dst[k] <- data bytes of allocation k (Sec. 3.1.1 "restore").
 * sizes[] are the registered sizes; a count or size difference is a
 * mismatch, not a format error. */
int orc_restore(const uint8_t *img, uint64_t len, uint64_t n, uint8_t *const *dst,
                const uint64_t *sizes)
{
    orc_header h;
    int rc = orc_parse_header(img, len, &h);
    if (rc) return rc;
    if (h.flags & ORC_FLAG_INCR) return ORC_EFORMAT;   /* a patch is not restorable */
    if (h.n != n) return ORC_EMISMATCH;
    uint64_t *doff = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    if (!doff) return ORC_ENOMEM;
    rc = orc_walk_full(img, len, &h, n, sizes, doff, NULL);
    if (rc == ORC_OK)
        for (uint64_t k = 0; k < n; ++k) memcpy(dst[k], img + doff[k], sizes[k]);
    free(doff);
    return rc;
}

/* Verify: recompute every chunk's CRC of data[k] and compare with the
 * image's stored hash; *mismatch = number of differing chunks. */
int orc_verify(const uint8_t *img, uint64_t len, uint64_t n, const uint8_t *const *data,
               const uint64_t *sizes, uint64_t *mismatch)
{
    orc_header h;
    int rc = orc_parse_header(img, len, &h);
    if (rc) return rc;
    if (h.flags & ORC_FLAG_INCR) return ORC_EFORMAT;
    if (h.n != n) return ORC_EMISMATCH;
    uint64_t *hoff = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    if (!hoff) return ORC_ENOMEM;
    rc = orc_walk_full(img, len, &h, n, sizes, NULL, hoff);
    if (rc) { free(hoff); return rc; }
    uint64_t bad = 0;
    for (uint64_t k = 0; k < n; ++k) {
        uint64_t nk = orc_n_chunks(sizes[k], h.C);
        for (uint64_t i = 0; i < nk; ++i) {
            uint64_t lo = i * h.C, hi = lo + h.C < sizes[k] ? lo + h.C : sizes[k];
            if (orc_crc32c(data[k] + lo, hi - lo) != orc_get32(img + hoff[k] + 4 * i)) ++bad;
        }
    }
    free(hoff);
    *mismatch = bad;
    return ORC_OK;
}

/* ------------------------------------------------------------ incremental */
/* Dirty set D_k = { i : new_hash_k[i] != prev_hash_k[i] }, ascending.  A
 * chunk is dirty exactly when its hash differs; the byte-exact invariant
 * apply_patch(prev_full, patch) == full(current) holds unless a changed
 * chunk keeps its CRC (probability 2^-32 per changed chunk). */

/* Size of the patch for these allocations given per-allocation dirty lists
 * (n_dirty[k] entries each, ascending in idx[k]). */
static uint64_t orc_patch_size(uint64_t n, const uint64_t *sizes, uint64_t C,
                               const uint64_t *n_dirty, const uint32_t *const *idx)
{
    uint64_t off = ORC_HDR;
    for (uint64_t k = 0; k < n; ++k) {
        uint64_t nk = orc_n_chunks(sizes[k], C);
        off = orc_up(off + ORC_REC + 4 * nk + 4 + 4 * n_dirty[k]);
        for (uint64_t j = 0; j < n_dirty[k]; ++j) {
            uint64_t i = idx[k][j];
            uint64_t lo = i * C, hi = lo + C < sizes[k] ? lo + C : sizes[k];
            off += orc_up(hi - lo);
        }
    }
    return off;
}

/* Write the incremental patch of the current data against prev_hash.
 * generation is this checkpoint's number, parent the base image's. */
int orc_write_patch(uint64_t n, const uint8_t *const *data, const uint64_t *sizes,
                    uint64_t C, const uint32_t *const *prev_hash, uint64_t generation,
                    uint64_t parent, uint8_t *out, uint64_t cap, uint64_t *used,
                    uint64_t *n_dirty_total)
{
    if (!orc_valid_chunk(C)) return ORC_EINVAL;
    /* step 1: hash every chunk (the definition: all chunks, every time) */
    uint32_t **cur = (uint32_t **)calloc(n ? n : 1, sizeof(void *));
    uint32_t **idx = (uint32_t **)calloc(n ? n : 1, sizeof(void *));
    uint64_t *nd = (uint64_t *)calloc(n ? n : 1, sizeof(uint64_t));
    int rc = ORC_OK;
    uint64_t total = 0, dirty_all = 0;
    if (!cur || !idx || !nd) { free(cur); free(idx); free(nd); return ORC_ENOMEM; }
    for (uint64_t k = 0; k < n; ++k) {
        uint64_t nk = orc_n_chunks(sizes[k], C);
        total += sizes[k];
        cur[k] = (uint32_t *)malloc(4 * (nk ? nk : 1));
        idx[k] = (uint32_t *)malloc(4 * (nk ? nk : 1));
        if (!cur[k] || !idx[k]) { rc = ORC_ENOMEM; goto done; }
        orc_chunk_hashes(data[k], sizes[k], C, cur[k]);
        /* step 2: dirty list in ascending chunk order */
        nd[k] = 0;
        for (uint64_t i = 0; i < nk; ++i)
            if (cur[k][i] != prev_hash[k][i]) idx[k][nd[k]++] = (uint32_t)i;
        dirty_all += nd[k];
    }
    {
        uint64_t need = orc_patch_size(n, sizes, C, nd, (const uint32_t *const *)idx);
        if (cap < need) { rc = ORC_EINVAL; goto done; }
        memset(out, 0, need);
        orc_write_header(out, ORC_FLAG_DEV | ORC_FLAG_INCR, C, n, total, generation, parent);
        /* step 3: per allocation: record, hashes, dirty list, dirty bytes */
        uint64_t off = ORC_HDR;
        for (uint64_t k = 0; k < n; ++k) {
            uint64_t nk = orc_n_chunks(sizes[k], C);
            uint64_t data_off = orc_up(off + ORC_REC + 4 * nk + 4 + 4 * nd[k]);
            uint8_t *rec = out + off;
            orc_put64(rec, sizes[k]);
            orc_put64(rec + 8, nk);
            orc_put64(rec + 16, data_off);
            orc_put64(rec + 24, 0);
            for (uint64_t i = 0; i < nk; ++i) orc_put32(rec + ORC_REC + 4 * i, cur[k][i]);
            orc_put32(rec + ORC_REC + 4 * nk, (uint32_t)nd[k]);
            for (uint64_t j = 0; j < nd[k]; ++j) orc_put32(rec + ORC_REC + 4 * nk + 4 + 4 * j, idx[k][j]);
            uint64_t d = data_off;
            for (uint64_t j = 0; j < nd[k]; ++j) {
                uint64_t i = idx[k][j];
                uint64_t lo = i * C, hi = lo + C < sizes[k] ? lo + C : sizes[k];
                memcpy(out + d, data[k] + lo, hi - lo);
                d += orc_up(hi - lo);
            }
            off = d;
        }
        *used = need;
        if (n_dirty_total) *n_dirty_total = dirty_all;
    }
done:
    for (uint64_t k = 0; k < n; ++k) { free(cur[k]); free(idx[k]); }
    free(cur); free(idx); free(nd);
    return rc;
}

/* apply_patch(base, patch): base (a full image, generation == the patch's
 * parent) is updated in place: every allocation's hashes are replaced, each
 * dirty chunk is copied into its slot, and the header takes the patch's
 * generation.  The result is the full image of the patched state. */
int orc_apply_patch(uint8_t *base, uint64_t base_len, const uint8_t *patch, uint64_t patch_len)
{
    orc_header hb, hp;
    int rc = orc_parse_header(base, base_len, &hb);
    if (rc) return rc;
    rc = orc_parse_header(patch, patch_len, &hp);
    if (rc) return rc;
    if (hb.flags & ORC_FLAG_INCR) return ORC_EFORMAT;
    if (!(hp.flags & ORC_FLAG_INCR)) return ORC_EFORMAT;
    if (hp.C != hb.C || hp.n != hb.n || hp.total != hb.total) return ORC_EMISMATCH;
    if (hp.parent != hb.generation) return ORC_EMISMATCH;
    uint64_t n = hb.n;
    uint64_t *bdoff = (uint64_t *)malloc(8 * (n ? n : 1));
    uint64_t *bhoff = (uint64_t *)malloc(8 * (n ? n : 1));
    if (!bdoff || !bhoff) { free(bdoff); free(bhoff); return ORC_ENOMEM; }
    rc = orc_walk_full(base, base_len, &hb, 0, NULL, bdoff, bhoff);
    if (rc) goto out;
    /* first pass: validate the whole patch before touching the base */
    for (int pass = 0; pass < 2; ++pass) {
        uint64_t off = ORC_HDR;
        for (uint64_t k = 0; k < n; ++k) {
            if (off + ORC_REC > patch_len) { rc = ORC_EFORMAT; goto out; }
            const uint8_t *rec = patch + off;
            uint64_t bk = orc_get64(rec), nk = orc_get64(rec + 8), dk = orc_get64(rec + 16);
            uint64_t base_bk = orc_get64(base + bhoff[k] - ORC_REC);
            if (bk != base_bk) { rc = ORC_EMISMATCH; goto out; }
            if (nk != orc_n_chunks(bk, hp.C) || orc_get64(rec + 24) != 0) { rc = ORC_EFORMAT; goto out; }
            if (nk > (patch_len - off) / 4 || off + ORC_REC + 4 * nk + 4 > patch_len) { rc = ORC_EFORMAT; goto out; }
            uint64_t ndk = orc_get32(rec + ORC_REC + 4 * nk);
            if (ndk > nk || off + ORC_REC + 4 * nk + 4 + 4 * ndk > patch_len) { rc = ORC_EFORMAT; goto out; }
            const uint8_t *ix = rec + ORC_REC + 4 * nk + 4;
            if (dk != orc_up(off + ORC_REC + 4 * nk + 4 + 4 * ndk)) { rc = ORC_EFORMAT; goto out; }
            uint64_t d = dk;
            int64_t last = -1;
            for (uint64_t j = 0; j < ndk; ++j) {
                uint64_t i = orc_get32(ix + 4 * j);
                if (i >= nk || (int64_t)i <= last) { rc = ORC_EFORMAT; goto out; }
                last = (int64_t)i;
                uint64_t lo = i * hp.C, hi = lo + hp.C < bk ? lo + hp.C : bk;
                if (d > patch_len || hi - lo > patch_len - d) { rc = ORC_EFORMAT; goto out; }
                if (pass == 1) memcpy(base + bdoff[k] + lo, patch + d, hi - lo);
                d += orc_up(hi - lo);
            }
            if (pass == 1) memcpy(base + bhoff[k], rec + ORC_REC, 4 * nk);
            off = d;
        }
        if (off > patch_len) { rc = ORC_EFORMAT; goto out; }
    }
    /* new header: a full image at the patch's generation */
    orc_write_header(base, ORC_FLAG_DEV, hb.C, hb.n, hb.total, hp.generation, 0);
out:
    free(bdoff);
    free(bhoff);
    return rc;
}

/* Patch fields of allocation k, for tests: n_dirty and the index list. */
int orc_patch_dirty(const uint8_t *patch, uint64_t len, uint64_t k, uint64_t *n_dirty,
                    uint32_t *idx_out, uint64_t idx_cap)
{
    orc_header h;
    int rc = orc_parse_header(patch, len, &h);
    if (rc) return rc;
    if (!(h.flags & ORC_FLAG_INCR) || k >= h.n) return ORC_EINVAL;
    uint64_t off = ORC_HDR;
    for (uint64_t a = 0; a <= k; ++a) {
        if (off + ORC_REC > len) return ORC_EFORMAT;
        const uint8_t *rec = patch + off;
        uint64_t bk = orc_get64(rec), nk = orc_get64(rec + 8), dk = orc_get64(rec + 16);
        if (off + ORC_REC + 4 * nk + 4 > len) return ORC_EFORMAT;
        uint64_t ndk = orc_get32(rec + ORC_REC + 4 * nk);
        if (a == k) {
            *n_dirty = ndk;
            for (uint64_t j = 0; j < ndk && j < idx_cap; ++j)
                idx_out[j] = orc_get32(rec + ORC_REC + 4 * nk + 4 + 4 * j);
            return ORC_OK;
        }
        uint64_t d = dk;
        for (uint64_t j = 0; j < ndk; ++j) {
            uint64_t i = orc_get32(rec + ORC_REC + 4 * nk + 4 + 4 * j);
            uint64_t lo = i * h.C, hi = lo + h.C < bk ? lo + h.C : bk;
            d += orc_up(hi - lo);
        }
        off = d;
    }
    return ORC_EFORMAT;
}
