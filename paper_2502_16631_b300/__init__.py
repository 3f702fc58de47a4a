"""Python binding of libsnap (GPU device-memory snapshot/restore, sm_103a).

Argument marshalling only: every step of the snapshot path runs in the CUDA
kernels of ``libsnap.so`` behind the C ABI declared in ``include/snap.h``.
PyTorch is used for device memory and streams (``tensor.data_ptr()``,
``torch.cuda.current_stream().cuda_stream``); nothing here falls back to a
CPU or PyTorch implementation -- if the extension is missing, importing the
library raises.

Paper: CRIUgpu (arXiv 2502.16631): checkpoint copies a process's device state
into host memory and restore copies it back (Sec. 3.1.1); the lock waits for
in-flight work with a 10 s timeout (Sec. 3.1.1); incremental checkpointing is
an optimisation Sec. 7 names.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsnap.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEDOUT, ENOBASE, EFORMAT, EMISMATCH, EBUSY, EBUDGET, EIO, EPEER = \
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10, -11
FILE_SYNC = 1
FULL, INCREMENTAL = 0, 1
INCR_COPY_DEFAULT, INCR_COPY_SM, INCR_COPY_DMA = 0, 1, 2
REQ_FULL, REQ_INCREMENTAL, REQ_RESTORE = 0, 1, 2

# Every entry point declared in include/snap.h.
EXPORTS = (
    "snap_set_create", "snap_set_destroy", "snap_set_prepare", "snap_register", "snap_image_bytes",
    "snap_host_alloc", "snap_host_free", "snap_host_register", "snap_host_unregister", "snap_checkpoint", "snap_checkpoint_async", "snap_checkpoint_wait",
    "snap_checkpoint_file", "snap_restore_file", "snap_restore", "snap_restore_async", "snap_restore_ready", "snap_restore_wait", "snap_verify",
    "snap_apply_patch", "snap_committed_hashes", "snap_last_stats", "snap_strerror",
    "snap_plain_checkpoint", "snap_plain_restore", "snap_hash_chunks", "snap_hash_chunks_noalloc",
    "snap_autotune", "snap_get_tuning", "snap_coordinate", "snap_checkpoint_coordinated", "snap_restore_coordinated",
    "snap_link_ceiling", "snap_host_copy_ceiling",
    "snap_server_create", "snap_server_destroy", "snap_server_submit", "snap_server_wait",
)


class SnapError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _lib().snap_strerror(status).decode() if _LIB is not None else str(status)
        super().__init__("%s: %s (%d)" % (what, msg, status) if what else "%s (%d)" % (msg, status))


class Opts(ctypes.Structure):
    _fields_ = [("chunk_bytes", ctypes.c_uint64), ("timeout_ms", ctypes.c_uint32),
                ("device", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("ctas_per_sm", ctypes.c_uint32), ("stages", ctypes.c_uint32),
                ("ring_bytes", ctypes.c_uint64), ("async_ctas", ctypes.c_uint32), ("hash_tma", ctypes.c_uint32),
                ("incr_copy", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("state_bytes", ctypes.c_uint64), ("image_bytes", ctypes.c_uint64),
                ("total_chunks", ctypes.c_uint64), ("dirty_chunks", ctypes.c_uint64),
                ("mismatches", ctypes.c_uint64), ("generation", ctypes.c_uint64),
                ("quiesce_ms", ctypes.c_double), ("hash_ms", ctypes.c_double),
                ("diff_ms", ctypes.c_double), ("copy_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("kernel_launches", ctypes.c_uint64),
                ("frozen_ms", ctypes.c_double), ("device_errors", ctypes.c_uint64),
                ("dma_copies", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


STEP_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p)
VOID_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p)
AGREE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int)


class CoordOps(ctypes.Structure):
    _fields_ = [("lock", STEP_FN), ("run", STEP_FN), ("commit", VOID_FN), ("abort", VOID_FN),
                ("agree", AGREE_FN)]


class Tuning(ctypes.Structure):
    _fields_ = [("warps", ctypes.c_uint32), ("stages", ctypes.c_uint32),
                ("piece_bytes", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("gbs", ctypes.c_double), ("chains", ctypes.c_uint32), ("tma", ctypes.c_uint32)]


_LIB = None


def _lib():
    """Load libsnap.so (building it in-tree first if sources changed)."""
    global _LIB
    if _LIB is None:
        if _build.stale():
            _build.build()
        L = ctypes.CDLL(LIB_PATH)
        vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        P = ctypes.POINTER
        sig = {
            "snap_set_create": [P(vp), P(Opts)],
            "snap_set_destroy": [vp],
            "snap_set_prepare": [vp, i32],
            "snap_register": [vp, vp, u64],
            "snap_image_bytes": [vp, i32, P(u64)],
            "snap_host_alloc": [u64, P(vp)],
            "snap_host_free": [vp],
            "snap_host_register": [vp, u64],
            "snap_host_unregister": [vp],
            "snap_checkpoint": [vp, vp, u64, i32, P(u64)],
            "snap_checkpoint_async": [vp, vp, u64, i32],
            "snap_checkpoint_wait": [vp, u32, P(u64)],
            "snap_restore": [vp, u64, vp],
            "snap_checkpoint_file": [vp, ctypes.c_char_p, i32, i32, P(u64)],
            "snap_restore_file": [ctypes.c_char_p, vp],
            "snap_restore_async": [vp, u64, vp, vp, u32],
            "snap_restore_ready": [vp, u32, vp],
            "snap_restore_wait": [vp, u32],
            "snap_verify": [vp, u64, vp, P(u64)],
            "snap_apply_patch": [vp, u64, vp, u64],
            "snap_committed_hashes": [vp, vp, u64, P(u64)],
            "snap_last_stats": [vp, P(Stats)],
            "snap_strerror": [i32],
            "snap_plain_checkpoint": [vp, vp, u64],
            "snap_plain_restore": [vp, u64, vp],
            "snap_hash_chunks": [vp, u64, u64, vp, vp],
            "snap_hash_chunks_noalloc": [P(vp), P(u64), u32, u64, vp, vp],
            "snap_autotune": [vp, i32, vp, u64, P(Tuning)],
            "snap_get_tuning": [vp, i32, P(Tuning)],
            "snap_coordinate": [P(CoordOps), vp],
            "snap_link_ceiling": [i32, i32, u64, i32, P(ctypes.c_double)],
            "snap_host_copy_ceiling": [i32, i32, u64, i32, i32, P(ctypes.c_double)],
            "snap_checkpoint_coordinated": [vp, vp, u64, i32, P(u64), AGREE_FN, vp],
            "snap_restore_coordinated": [vp, u64, vp, AGREE_FN, vp],
            "snap_server_create": [P(vp), u64, u64, P(Opts)],
            "snap_server_destroy": [vp],
            "snap_server_submit": [vp, vp, i32, vp, u64, P(u64)],
            "snap_server_wait": [vp, u64, u32, P(i32), P(Stats)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name == "snap_strerror" else ctypes.c_int
        _LIB = L
    return _LIB


def lib():
    return _lib()


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise SnapError(rc, what)
    return rc


def strerror(status: int) -> str:
    return _lib().snap_strerror(status).decode()


def _addr(x) -> int:
    """Device/host address of a torch tensor, HostBuffer, numpy array or int."""
    if isinstance(x, int):
        return x
    if isinstance(x, HostBuffer):
        return x.ptr
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("the library reads and writes one contiguous byte range: pass a contiguous array")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("the library reads and writes one contiguous byte range: pass a contiguous tensor")
        return x.data_ptr()
    raise TypeError("cannot take the address of %r" % type(x))


def _nbytes(x) -> int:
    if isinstance(x, HostBuffer):
        return x.nbytes
    if isinstance(x, np.ndarray):
        return x.nbytes
    if hasattr(x, "untyped_storage"):
        return x.numel() * x.element_size()
    raise TypeError("cannot size %r" % type(x))


def _span(x, n=None, writable=False):
    """(address, byte count) of a caller's buffer for a call that reads, or
    with `writable` writes, its first `n` bytes (all of it by default).  A
    count beyond a sized buffer, or a read-only array the library would
    write, is refused here, before the library could touch memory outside
    the buffer; a raw integer address is passed on with its count as given."""
    if isinstance(x, int):
        if n is None:
            raise TypeError("a raw address needs an explicit byte count")
        return x, n
    size = _nbytes(x)
    if n is None:
        n = size
    elif n < 0 or n > size:
        raise ValueError("byte count %d outside the %d-byte buffer" % (n, size))
    if writable and isinstance(x, np.ndarray) and not x.flags.writeable:
        raise ValueError("the library writes this buffer: pass a writable array")
    return _addr(x), n


class HostBuffer:
    """Pinned, device-mapped host memory from snap_host_alloc."""

    def __init__(self, nbytes: int):
        p = ctypes.c_void_p()
        _check(_lib().snap_host_alloc(nbytes, ctypes.byref(p)), "snap_host_alloc")
        self.ptr = p.value
        self.nbytes = nbytes
        self.array = np.ctypeslib.as_array((ctypes.c_uint8 * nbytes).from_address(self.ptr))

    def view(self, n: int | None = None) -> np.ndarray:
        return self.array[: self.nbytes if n is None else n]

    def close(self):
        if self.ptr:
            self.array = None
            _lib().snap_host_free(self.ptr)
            self.ptr = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Set:
    """A set of registered device allocations (snap_set)."""

    def __init__(self, chunk_bytes: int = 0, timeout_ms: int = 0, device: int = -1, stream=None,
                 ctas_per_sm: int = 0, stages: int = 0, ring_bytes: int = 0, async_ctas: int = 0,
                 hash_tma: bool = False, incr_copy: int = 0):
        o = Opts(chunk_bytes, timeout_ms, device, _stream_handle(stream), ctas_per_sm, stages, ring_bytes,
                 async_ctas, 1 if hash_tma else 0, incr_copy)
        h = ctypes.c_void_p()
        _check(_lib().snap_set_create(ctypes.byref(h), ctypes.byref(o)), "snap_set_create")
        self.h = h.value
        self.tensors = []

    def close(self):
        if self.h:
            _lib().snap_set_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register(self, t, nbytes: int | None = None) -> int:
        """Register a device tensor (or a raw device address with nbytes)."""
        addr, nbytes = _span(t, nbytes)
        if not isinstance(t, int):
            self.tensors.append(t)
        return _check(_lib().snap_register(self.h, addr, nbytes), "snap_register")

    def prepare(self, layout: bool = True, ring: bool = False, shadow: bool = False) -> None:
        """One-time setup now (device tables, pinned ring, async shadow), not in the first call."""
        what = (1 if layout else 0) | (2 if ring else 0) | (4 if shadow else 0)
        _check(_lib().snap_set_prepare(self.h, what), "snap_set_prepare")

    def image_bytes(self, mode: int = FULL) -> int:
        v = ctypes.c_uint64()
        _check(_lib().snap_image_bytes(self.h, mode, ctypes.byref(v)), "snap_image_bytes")
        return v.value

    def checkpoint(self, image, mode: int = FULL, cap: int | None = None) -> int:
        used = ctypes.c_uint64()
        _check(_lib().snap_checkpoint(self.h, *_span(image, cap, True), mode,
                                      ctypes.byref(used)), "snap_checkpoint")
        return used.value

    def checkpoint_status(self, image, mode: int = FULL, cap: int | None = None):
        used = ctypes.c_uint64()
        rc = _lib().snap_checkpoint(self.h, *_span(image, cap, True), mode,
                                    ctypes.byref(used))
        return rc, used.value

    def checkpoint_async(self, image, mode: int = FULL, cap: int | None = None) -> None:
        """Start an asynchronous checkpoint; returns once the cut is taken."""
        _check(self.checkpoint_async_status(image, mode, cap), "snap_checkpoint_async")

    def checkpoint_async_status(self, image, mode: int = FULL, cap: int | None = None) -> int:
        return _lib().snap_checkpoint_async(self.h, *_span(image, cap, True), mode)

    def checkpoint_wait(self, timeout_ms: int = 60000) -> int:
        """Finish the pending asynchronous checkpoint; returns the image bytes."""
        rc, used = self.checkpoint_wait_status(timeout_ms)
        _check(rc, "snap_checkpoint_wait")
        return used

    def checkpoint_wait_status(self, timeout_ms: int = 60000):
        used = ctypes.c_uint64()
        rc = _lib().snap_checkpoint_wait(self.h, timeout_ms, ctypes.byref(used))
        return rc, used.value

    def checkpoint_coordinated(self, image, agree, mode: int = FULL, cap: int | None = None):
        """One rank of a coordinated checkpoint; `agree(phase, status) ->
        global status` is the transport (see all_reduce_agree).  Returns
        (status, image bytes)."""
        used = ctypes.c_uint64()
        cb = _agree_callback(agree)
        rc = _lib().snap_checkpoint_coordinated(self.h, *_span(image, cap, True), mode,
                                                ctypes.byref(used), cb, None)
        return rc, used.value

    def restore_coordinated(self, image, agree, nbytes: int | None = None) -> int:
        """One rank of a coordinated restore; returns the status."""
        cb = _agree_callback(agree)
        return _lib().snap_restore_coordinated(*_span(image, nbytes), self.h,
                                               cb, None)

    def restore(self, image, nbytes: int | None = None) -> None:
        _check(self.restore_status(image, nbytes), "snap_restore")

    def checkpoint_file(self, path: str, mode: int = FULL, sync: bool = False) -> int:
        """Checkpoint straight into a file (written as <path>.tmp, renamed when complete)."""
        rc, used = self.checkpoint_file_status(path, mode, sync)
        _check(rc, "snap_checkpoint_file")
        return used

    def checkpoint_file_status(self, path: str, mode: int = FULL, sync: bool = False):
        used = ctypes.c_uint64()
        rc = _lib().snap_checkpoint_file(self.h, os.fsencode(path), mode, FILE_SYNC if sync else 0,
                                         ctypes.byref(used))
        return rc, used.value

    def restore_file(self, path: str) -> None:
        _check(self.restore_file_status(path), "snap_restore_file")

    def restore_file_status(self, path: str) -> int:
        return _lib().snap_restore_file(os.fsencode(path), self.h)

    def restore_async(self, image, first=(), nbytes: int | None = None) -> None:
        """Start a prioritised restore: the allocations in `first` come back
        first, the rest follow in waves."""
        _check(self.restore_async_status(image, first, nbytes), "snap_restore_async")

    def restore_async_status(self, image, first=(), nbytes: int | None = None) -> int:
        arr = (ctypes.c_uint32 * max(1, len(first)))(*first)
        return _lib().snap_restore_async(*_span(image, nbytes), self.h,
                                         ctypes.cast(arr, ctypes.c_void_p), len(first))

    def restore_ready(self, index: int, stream=None) -> None:
        """Make `stream` (torch stream or handle; None: the set's) wait for
        allocation `index` of the pending prioritised restore."""
        _check(_lib().snap_restore_ready(self.h, index, _stream_handle(stream)), "snap_restore_ready")

    def restore_wait(self, timeout_ms: int = 60000) -> None:
        _check(self.restore_wait_status(timeout_ms), "snap_restore_wait")

    def restore_wait_status(self, timeout_ms: int = 60000) -> int:
        return _lib().snap_restore_wait(self.h, timeout_ms)

    def restore_status(self, image, nbytes: int | None = None) -> int:
        return _lib().snap_restore(*_span(image, nbytes), self.h)

    def verify(self, image, nbytes: int | None = None) -> int:
        bad = ctypes.c_uint64()
        _check(_lib().snap_verify(*_span(image, nbytes), self.h,
                                  ctypes.byref(bad)), "snap_verify")
        return bad.value

    def committed_hashes(self, n: int) -> tuple[np.ndarray, int]:
        out = np.zeros(max(n, 1), dtype=np.uint32)
        gen = ctypes.c_uint64()
        _check(_lib().snap_committed_hashes(self.h, out.ctypes.data, n, ctypes.byref(gen)),
               "snap_committed_hashes")
        return out[:n], gen.value

    def stats(self) -> dict:
        s = Stats()
        _check(_lib().snap_last_stats(self.h, ctypes.byref(s)), "snap_last_stats")
        return s.as_dict()

    def plain_checkpoint(self, image, cap: int | None = None) -> None:
        _check(_lib().snap_plain_checkpoint(self.h, *_span(image, cap, True)),
               "snap_plain_checkpoint")

    def plain_restore(self, image, nbytes: int | None = None) -> None:
        _check(_lib().snap_plain_restore(*_span(image, nbytes), self.h),
               "snap_plain_restore")

    def autotune(self, mode: int = INCREMENTAL, image=None) -> dict:
        t = Tuning()
        _check(_lib().snap_autotune(self.h, mode, *(_span(image, None, True) if image is not None else (None, 0)),
                                    ctypes.byref(t)),
               "snap_autotune")
        return {k: getattr(t, k) for k, _ in t._fields_}

    def tuning(self, mode: int = INCREMENTAL) -> dict:
        """The launch shape the set uses for `mode` (snap_get_tuning)."""
        t = Tuning()
        _check(_lib().snap_get_tuning(self.h, mode, ctypes.byref(t)), "snap_get_tuning")
        return {k: getattr(t, k) for k, _ in t._fields_}


def apply_patch(base, patch, base_bytes: int | None = None, patch_bytes: int | None = None) -> None:
    """Merge `patch` into the full image `base` in place (host memory)."""
    _check(apply_patch_status(base, patch, base_bytes, patch_bytes), "snap_apply_patch")


def apply_patch_status(base, patch, base_bytes=None, patch_bytes=None) -> int:
    return _lib().snap_apply_patch(*_span(base, base_bytes, True), *_span(patch, patch_bytes))


def hash_chunks(dev_tensor, chunk_bytes: int, out, nbytes: int | None = None, stream=None) -> None:
    """CRC-32C of every chunk of a device buffer into the device array `out`."""
    addr, n = _span(dev_tensor, nbytes)
    if not isinstance(out, int) and chunk_bytes > 0 and _nbytes(out) < 4 * ((n + chunk_bytes - 1) // chunk_bytes):
        raise ValueError("`out` holds fewer than ceil(nbytes / chunk_bytes) 32-bit hashes")
    _check(_lib().snap_hash_chunks(addr, n, chunk_bytes, _addr(out), _stream_handle(stream)), "snap_hash_chunks")


NOALLOC_MAX_BUFFERS = 1024


def hash_chunks_noalloc(buffers, chunk_bytes: int, out, stream=None) -> int:
    """Chunk hashes of several device buffers (tensors, or (address, nbytes)
    pairs) into the device array `out`, buffer after buffer, without any
    GPU memory allocation (for callers that cannot allocate).  Returns the
    status (0 on success)."""
    n = len(buffers)
    ptrs = (ctypes.c_void_p * max(1, n))()
    sizes = (ctypes.c_uint64 * max(1, n))()
    for k, b in enumerate(buffers):
        if isinstance(b, tuple):
            ptrs[k], sizes[k] = b[0], b[1]
        else:
            ptrs[k], sizes[k] = _addr(b), _nbytes(b)
    return _lib().snap_hash_chunks_noalloc(ptrs, sizes, n, chunk_bytes, _addr(out), _stream_handle(stream))


def _agree_callback(agree):
    def f(_ctx, phase, status):
        try:
            return int(agree(phase, status))
        except Exception:  # the transport failed: report it as a failure
            return ETIMEDOUT
    return AGREE_FN(f)


def host_register(array: np.ndarray) -> None:
    """Pin and map a caller's host array (snap_host_register) so that calls
    and server requests use it as an image directly, without staging."""
    _check(_lib().snap_host_register(array.ctypes.data, array.nbytes), "snap_host_register")


def host_unregister(array: np.ndarray) -> None:
    """Undo host_register (before the array is freed)."""
    _check(_lib().snap_host_unregister(array.ctypes.data), "snap_host_unregister")


def host_copy_ceiling(threads: int, direction: int = 2, nbytes: int = 2 << 30, reps: int = 3,
                      with_link: bool = False) -> float:
    """GB/s that `threads` host threads copy between pinned and pageable
    memory with the workers' copy routine (0: pinned to pageable, 1: the
    other way, 2: both at once), optionally under link load."""
    v = ctypes.c_double()
    _check(_lib().snap_host_copy_ceiling(threads, direction, nbytes, reps, 1 if with_link else 0, ctypes.byref(v)),
           "snap_host_copy_ceiling")
    return v.value


def link_ceiling(direction: int = 0, nbytes: int = 1 << 30, reps: int = 3, device: int = -1) -> float:
    """GB/s that SM loads/stores reach over the host link (0: device to host,
    1: host to device, 2: both at once, the two directions' bytes together):
    the gather and scatter kernels' ceiling, and a mixed launch's."""
    v = ctypes.c_double()
    _check(_lib().snap_link_ceiling(device, direction, nbytes, reps, ctypes.byref(v)), "snap_link_ceiling")
    return v.value


def coordinate(agree, lock=None, run=None, commit=None, abort=None) -> int:
    """Run snap_coordinate's two-phase protocol over Python steps: lock() and
    run() return a status, commit() and abort() nothing, agree(phase, status)
    returns the global status.  A step that raises counts as ECUDA."""
    def step(fn):
        if fn is None:
            return STEP_FN()

        def f(_ctx):
            try:
                return int(fn())
            except Exception:
                return ECUDA
        return STEP_FN(f)

    def vstep(fn):
        if fn is None:
            return VOID_FN()
        return VOID_FN(lambda _ctx: fn())

    ops = CoordOps(step(lock), step(run), vstep(commit), vstep(abort), _agree_callback(agree))
    return _lib().snap_coordinate(ctypes.byref(ops), None)


def all_reduce_agree(group=None):
    """agree() over torch.distributed: the minimum status of all ranks (every
    failure is negative), through a CPU tensor (a gloo group)."""
    import torch
    import torch.distributed as dist

    def agree(phase, status):
        t = torch.tensor([status], dtype=torch.int32)
        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
        return int(t.item())
    return agree


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Server:
    """Serving loop over tenant sets (snap_server)."""

    def __init__(self, pinned_budget: int, hbm_budget: int, chunk_bytes: int = 0, timeout_ms: int = 0,
                 device: int = -1, ring_bytes: int = 0):
        o = Opts(chunk_bytes, timeout_ms, device, None, 0, 0, ring_bytes)
        h = ctypes.c_void_p()
        _check(_lib().snap_server_create(ctypes.byref(h), pinned_budget, hbm_budget, ctypes.byref(o)),
               "snap_server_create")
        self.h = h.value

    def close(self):
        if self.h:
            _lib().snap_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, tenant: Set, kind: int, image, cap: int | None = None) -> int:
        t = ctypes.c_uint64()
        _check(_lib().snap_server_submit(self.h, tenant.h, kind, *_span(image, cap, kind != REQ_RESTORE),
                                         ctypes.byref(t)),
               "snap_server_submit")
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 60000):
        st = ctypes.c_int()
        s = Stats()
        rc = _lib().snap_server_wait(self.h, ticket, timeout_ms, ctypes.byref(st), ctypes.byref(s))
        return rc, st.value, s.as_dict()
