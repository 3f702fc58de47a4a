// Checkpoint images persisted to storage, overlapped with the transfer.
//
// The paper's checkpoint ends with the memory write of the image (Table 2
// lists it as its own stage after the device copy).  Here the two overlap:
// the state streams through the set's pinned ring window by window, and the
// host workers that would copy a window into a pageable image write it to
// the image file instead (pwrite at the image offsets), while the GPU fills
// the next slots.  Restore reads windows from the file into slots while the
// scatter kernel empties earlier ones.  The image is written to a temporary
// name and renamed into place only when complete, so a failed checkpoint
// never leaves a partial image under the caller's name, and the committed
// base moves only after the rename (Sec. 3.1: only a completed checkpoint
// counts).
#include "snap.h"
#include "snap_format.h"
#include "snap_internal.h"
#include "runtime_internal.h"
#include "host_copy.h"

#include <algorithm>
#include <cerrno>
#include <cstring>
#include <fcntl.h>
#include <string>
#include <sys/stat.h>
#include <unistd.h>

using namespace snapk;

namespace snapk {

// Storage can be far slower than the link: the completion deadline of a file
// call grows with the image size, as if storage moved 64 MB/s.
static double io_deadline(const snap_set_s *s, double from, uint64_t bytes)
{
    return from + s->timeout_ms + (double)bytes / 65536.0;
}

static bool full_pwrite(int fd, const uint8_t *p, uint64_t n, uint64_t off)
{
    while (n) {
        const ssize_t w = ::pwrite(fd, p, std::min<uint64_t>(n, 1ull << 30), (off_t)off);
        if (w < 0 && errno == EINTR) continue;
        if (w <= 0) return false;
        p += w;
        n -= (uint64_t)w;
        off += (uint64_t)w;
    }
    return true;
}

static bool full_pread(int fd, uint8_t *p, uint64_t n, uint64_t off)
{
    while (n) {
        const ssize_t r = ::pread(fd, p, std::min<uint64_t>(n, 1ull << 30), (off_t)off);
        if (r < 0 && errno == EINTR) continue;
        if (r <= 0) return false;  // error, or the file ends early
        p += r;
        n -= (uint64_t)r;
        off += (uint64_t)r;
    }
    return true;
}

void ImageIO::put(uint64_t off, const void *src, uint64_t n)
{
    if (!n || err.load()) return;
    if (mem) {
        stream_copy(mem + off, src, n);
        return;
    }
    if (!full_pwrite(fd, static_cast<const uint8_t *>(src), n, off)) err.store(SNAP_EIO);
}

void ImageIO::get(uint64_t off, void *dst, uint64_t n)
{
    if (!n || err.load()) return;
    if (mem) {
        stream_copy(dst, mem + off, n);
        return;
    }
    if (!full_pread(fd, static_cast<uint8_t *>(dst), n, off)) err.store(SNAP_EIO);
}

void ImageIO::zero(uint64_t off, uint64_t n)
{
    if (mem && n) std::memset(mem + off, 0, n);
}

// fsync the directory holding `path`, so that a rename into it is durable.
static bool sync_dir(const std::string &path)
{
    const size_t sl = path.find_last_of('/');
    const std::string dir = sl == std::string::npos ? "." : (sl == 0 ? "/" : path.substr(0, sl));
    const int d = ::open(dir.c_str(), O_RDONLY | O_DIRECTORY | O_CLOEXEC);
    if (d < 0) return false;
    const bool ok = ::fsync(d) == 0;
    ::close(d);
    return ok;
}

}  // namespace snapk

extern "C" {

int snap_checkpoint_file(snap_set s, const char *path, int mode, int flags, uint64_t *used)
{
    const double t0 = now_ms();
    if (!s || !path || !*path) return SNAP_EINVAL;
    if (mode != SNAP_FULL && mode != SNAP_INCREMENTAL) return SNAP_EINVAL;
    if (flags & ~SNAP_FILE_SYNC) return SNAP_EINVAL;
    BusyGuard g(s);
    if (!g.ok) return SNAP_EBUSY;
    cudaSetDevice(s->device);
    const double deadline = t0 + s->timeout_ms;
    int rc = settle(s, deadline);
    if (rc) return rc;
    rc = build_layout(s);
    if (rc) return rc;
    if (mode == SNAP_INCREMENTAL && !s->has_base) return SNAP_ENOBASE;
    const std::string tmp = std::string(path) + ".tmp";
    const int fd = ::open(tmp.c_str(), O_CREAT | O_TRUNC | O_WRONLY | O_CLOEXEC, 0644);
    if (fd < 0) return SNAP_EIO;
    // Reserve the image's blocks up front (a patch: its upper bound, trimmed
    // at the end) so that the workers' concurrent writes land in contiguous
    // extents instead of interleaving in arrival order; where the file system
    // cannot preallocate, only set the size.  Ranges never written (the
    // padding) read back as zero either way.
    const uint64_t reserve = mode == SNAP_FULL ? s->full_bytes : s->patch_bound;
    if (::posix_fallocate(fd, 0, (off_t)reserve) != 0 && ::ftruncate(fd, (off_t)reserve) != 0) rc = SNAP_EIO;
    double tq = 0;
    if (rc == SNAP_OK) rc = quiesce(s, deadline);
    tq = now_ms();
    // the commit of ring_checkpoint is undone unless the file lands
    const int prev_idx = s->prev_idx;
    const bool has_base = s->has_base;
    const uint64_t base_gen = s->base_gen, next_gen = s->next_gen;
    uint64_t u = 0;
    ImageIO io;
    io.fd = fd;
    if (rc == SNAP_OK)
        rc = ring_checkpoint(s, io, mode == SNAP_FULL ? s->full_bytes : s->patch_bound, mode, &u, t0, tq,
                             io_deadline(s, tq, s->full_bytes));
    if (rc == SNAP_OK && mode == SNAP_INCREMENTAL && ::ftruncate(fd, (off_t)u) != 0) rc = SNAP_EIO;
    if (rc == SNAP_OK && (flags & SNAP_FILE_SYNC) && ::fsync(fd) != 0) rc = SNAP_EIO;
    if (::close(fd) != 0 && rc == SNAP_OK) rc = SNAP_EIO;
    if (rc == SNAP_OK && ::rename(tmp.c_str(), path) != 0) rc = SNAP_EIO;
    if (rc == SNAP_OK && (flags & SNAP_FILE_SYNC) && !sync_dir(path)) rc = SNAP_EIO;
    if (rc != SNAP_OK) {
        ::unlink(tmp.c_str());
        s->prev_idx = prev_idx;
        s->has_base = has_base;
        s->base_gen = base_gen;
        s->next_gen = next_gen;
        return rc;
    }
    if (used) *used = u;
    s->last.total_ms = now_ms() - t0;
    s->last.frozen_ms = s->last.total_ms;
    return SNAP_OK;
}

int snap_restore_file(const char *path, snap_set s)
{
    const double t0 = now_ms();
    if (!s || !path || !*path) return SNAP_EINVAL;
    BusyGuard g(s);
    if (!g.ok) return SNAP_EBUSY;
    cudaSetDevice(s->device);
    const double deadline = t0 + s->timeout_ms;
    int rc = settle(s, deadline);
    if (rc) return rc;
    rc = build_layout(s);
    if (rc) return rc;
    const int fd = ::open(path, O_RDONLY | O_CLOEXEC);
    if (fd < 0) return SNAP_EIO;
    struct Closer {
        int fd;
        ~Closer() { ::close(fd); }
    } closer{fd};
    struct stat sb{};
    if (::fstat(fd, &sb) != 0) return SNAP_EIO;
    const uint64_t len = (uint64_t)sb.st_size;
    uint8_t hdr[SNAP_IMG_HEADER_BYTES];
    if (len < sizeof hdr) return SNAP_EFORMAT;
    if (!full_pread(fd, hdr, sizeof hdr, 0)) return SNAP_EIO;
    ImageHeader h{};
    rc = parse_header(hdr, len, &h);
    if (rc) return rc;
    if (h.flags & SNAP_IMG_FLAG_INCREMENTAL) return SNAP_EFORMAT;  // merge patches first
    rc = walk_records_io(s, [fd](uint64_t off, void *dst, uint64_t n) {
        return full_pread(fd, static_cast<uint8_t *>(dst), n, off);
    }, len, h, s->h_hash_stage);
    if (rc) return rc;
    rc = quiesce(s, deadline);
    if (rc) return rc;
    const double tq = now_ms();
    ImageIO io;
    io.fd = fd;
    return ring_restore(s, io, h, t0, tq, io_deadline(s, tq, len));
}

}  // extern "C"
