/*
 * snap_format.h -- on-host layout of libsnap checkpoint images.
 *
 * All integers are little-endian.  A full image is:
 *
 *   offset 0, 64-byte header
 *     0  char  magic[8] = "SNAPIMG1"
 *     8  u32   version = 1
 *     12 u32   flags: bit0 = incremental patch, bit1 = holds device state
 *              (the "contains GPU state" inventory flag of Sec. 3.1.1)
 *     16 u64   chunk_bytes C
 *     24 u64   n_allocs
 *     32 u64   total_state_bytes (sum of allocation sizes)
 *     40 u64   generation (0 for a set's first checkpoint, +1 per later one;
 *              a restore adopts the image's generation)
 *     48 u64   parent_generation (patches: generation of their base; else 0)
 *     56 u32   CRC-32C of bytes 0..55
 *     60 u32   0
 *   then, per allocation k in registration order:
 *     32-byte record {u64 bytes_k, u64 n_k = ceil(bytes_k / C),
 *                     u64 data_offset_k (absolute), u64 0}
 *     u32 hash[n_k]: CRC-32C of chunk i = bytes [i*C, min((i+1)*C, bytes_k))
 *     zero padding to a 4096-byte boundary
 *     bytes_k data bytes at data_offset_k, zero padding to 4096
 *
 * An incremental patch has the same header (flags bit0 set) and per
 * allocation: the same 32-byte record, all n_k new hashes, u32 n_dirty_k,
 * u32 idx[n_dirty_k] (ascending chunk indices whose hash changed), zero
 * padding to 4096, then each dirty chunk's bytes in index order, each padded
 * to 4096 (a full chunk is C bytes, C being a multiple of 4096).
 *
 * Chunks never span allocations; the last chunk of an allocation is hashed
 * over its real length; a zero-byte allocation has no chunks.
 */
#ifndef SNAP_FORMAT_H
#define SNAP_FORMAT_H

#define SNAP_IMG_MAGIC "SNAPIMG1"
#define SNAP_IMG_VERSION 1u
#define SNAP_IMG_HEADER_BYTES 64u
#define SNAP_IMG_RECORD_BYTES 32u
#define SNAP_IMG_PAGE 4096u
#define SNAP_IMG_FLAG_INCREMENTAL 1u
#define SNAP_IMG_FLAG_DEVICE_STATE 2u

#endif /* SNAP_FORMAT_H */
