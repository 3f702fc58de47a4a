"""CPU oracle for the snapshot/restore path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this module.  The product package never imports it,
and the two share no code: the oracle is ``snap_oracle.c`` (plain C, one byte
at a time) behind this ctypes wrapper.

Paper: CRIUgpu (arXiv 2502.16631).  Checkpoint copies device state into a
host image (Sec. 3.1.1, checkpoint action); restore puts it back byte for byte
(Sec. 3.1.1, restore action; Sec. 6); incremental checkpointing is the
optimisation named in Sec. 7 (Check-N-Run).  CRC-32C per RFC 3720.

Parity pins live in ``tests/test_oracle_*.py``; no function here is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snap_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, ENOMEM, EFORMAT, EMISMATCH = 0, -1, -2, -6, -7


def build(force: bool = False) -> str:
    """Compile the oracle library in-tree (gcc, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u8p, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
        pp = ctypes.POINTER(ctypes.c_void_p)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.orc_crc32c.restype = u32
        L.orc_crc32c.argtypes = [u8p, u64]
        L.orc_crc32c_update.restype = u32
        L.orc_crc32c_update.argtypes = [u32, u8p, u64]
        L.orc_n_chunks.restype = u64
        L.orc_n_chunks.argtypes = [u64, u64]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_get_threads.restype = ctypes.c_int
        L.orc_chunk_hashes.argtypes = [u8p, u64, u64, u8p]
        L.orc_image_bytes.restype = u64
        L.orc_image_bytes.argtypes = [u64, u64p, u64]
        L.orc_write_full.argtypes = [u64, pp, u64p, u64, u64, u8p, u64, u64p]
        L.orc_write_full_window.argtypes = [u64, pp, u64p, u64, u64, u64, u64, u8p, u64, u64p, u64p]
        L.orc_read_header.argtypes = [u8p, u64, u64p]
        L.orc_restore.argtypes = [u8p, u64, u64, pp, u64p]
        L.orc_verify.argtypes = [u8p, u64, u64, pp, u64p, u64p]
        L.orc_write_patch.argtypes = [u64, pp, u64p, u64, pp, u64, u64, u8p, u64, u64p, u64p]
        L.orc_apply_patch.argtypes = [u8p, u64, u8p, u64]
        L.orc_patch_dirty.argtypes = [u8p, u64, u64, u64p, u8p, u64]
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _bufs(datas):
    arrs = [np.ascontiguousarray(d, dtype=np.uint8).reshape(-1) for d in datas]
    ptrs = (ctypes.c_void_p * max(1, len(arrs)))(*[_ptr(a) for a in arrs])
    sizes = (ctypes.c_uint64 * max(1, len(arrs)))(*[a.size for a in arrs])
    return arrs, ptrs, sizes


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def crc32c(data) -> int:
    a = np.frombuffer(bytes(data), dtype=np.uint8) if isinstance(data, (bytes, bytearray)) else \
        np.ascontiguousarray(data, dtype=np.uint8).reshape(-1)
    return int(lib().orc_crc32c(_ptr(a) if a.size else None, a.size))


def crc32c_update(state: int, data) -> int:
    a = np.frombuffer(bytes(data), dtype=np.uint8) if isinstance(data, (bytes, bytearray)) else \
        np.ascontiguousarray(data, dtype=np.uint8).reshape(-1)
    return int(lib().orc_crc32c_update(state & 0xFFFFFFFF, _ptr(a) if a.size else None, a.size))


def n_chunks(nbytes: int, chunk: int) -> int:
    return int(lib().orc_n_chunks(nbytes, chunk))


def chunk_hashes(data, chunk: int) -> np.ndarray:
    a = np.ascontiguousarray(data, dtype=np.uint8).reshape(-1)
    out = np.zeros(max(1, n_chunks(a.size, chunk)), dtype=np.uint32)
    lib().orc_chunk_hashes(_ptr(a) if a.size else None, a.size, chunk, _ptr(out))
    return out[: n_chunks(a.size, chunk)]


def image_bytes(sizes, chunk: int) -> int:
    s = (ctypes.c_uint64 * max(1, len(sizes)))(*sizes)
    return int(lib().orc_image_bytes(len(sizes), s, chunk))


def write_full(datas, chunk: int, generation: int = 0, out: np.ndarray | None = None):
    """Full image of the allocations `datas` (list of uint8 arrays).

    Returns (status, image array)."""
    arrs, ptrs, sizes = _bufs(datas)
    need = image_bytes([a.size for a in arrs], chunk) if chunk >= 4096 else 64
    if out is None:
        out = np.empty(need, dtype=np.uint8)
    used = ctypes.c_uint64(0)
    rc = lib().orc_write_full(len(arrs), ptrs, sizes, chunk, generation, _ptr(out), out.size,
                              ctypes.byref(used))
    return rc, out[: used.value]


def write_full_window(sizes, datas, chunk: int, generation: int, k0: int, k1: int):
    """Bytes [lo, hi) of the full image of allocations of `sizes`: from the
    header (k0 == 0) or record k0 to the end of record k1 - 1; `datas` holds
    the bytes of allocations k0..k1-1 only.  Returns (status, lo, array)."""
    n = len(sizes)
    arrs = [np.ascontiguousarray(d, dtype=np.uint8).reshape(-1) for d in datas]
    assert len(arrs) == k1 - k0
    ptrs = (ctypes.c_void_p * max(1, n))()
    for j, a in enumerate(arrs):
        assert a.size == sizes[k0 + j]
        ptrs[k0 + j] = _ptr(a) if a.size else None
    sz = (ctypes.c_uint64 * max(1, n))(*sizes)
    lo_b = image_bytes(list(sizes[:k0]), chunk) if k0 else 0
    out = np.empty(max(1, image_bytes(list(sizes[:k1]), chunk) - lo_b), dtype=np.uint8)
    lo, used = ctypes.c_uint64(0), ctypes.c_uint64(0)
    rc = lib().orc_write_full_window(n, ptrs, sz, chunk, generation, k0, k1, _ptr(out), out.size,
                                     ctypes.byref(lo), ctypes.byref(used))
    return rc, int(lo.value), out[: used.value]


def read_header(img: np.ndarray):
    o = (ctypes.c_uint64 * 6)()
    rc = lib().orc_read_header(_ptr(img), img.size, o)
    keys = ("flags", "chunk_bytes", "n_allocs", "total_state_bytes", "generation",
            "parent_generation")
    return rc, dict(zip(keys, (int(v) for v in o)))


def restore(img: np.ndarray, sizes):
    """Returns (status, list of restored arrays)."""
    outs = [np.zeros(s, dtype=np.uint8) for s in sizes]
    _, ptrs, sz = _bufs(outs)
    rc = lib().orc_restore(_ptr(img), img.size, len(outs), ptrs, sz)
    return rc, outs


def verify(img: np.ndarray, datas):
    arrs, ptrs, sizes = _bufs(datas)
    bad = ctypes.c_uint64(0)
    rc = lib().orc_verify(_ptr(img), img.size, len(arrs), ptrs, sizes, ctypes.byref(bad))
    return rc, int(bad.value)


def write_patch(datas, chunk: int, prev_hashes, generation: int, parent: int):
    """Incremental patch of `datas` against `prev_hashes` (list of uint32 arrays).

    Returns (status, patch array, total dirty chunks)."""
    arrs, ptrs, sizes = _bufs(datas)
    ph = [np.ascontiguousarray(h, dtype=np.uint32) for h in prev_hashes]
    hptrs = (ctypes.c_void_p * max(1, len(ph)))(*[_ptr(h) if h.size else None for h in ph])
    # a patch never exceeds the full image plus, per allocation, the dirty
    # count, the index list and one page of rounding
    cap = image_bytes([a.size for a in arrs], chunk) + \
        sum(4096 + 4 + 4 * n_chunks(a.size, chunk) for a in arrs)
    out = np.empty(cap, dtype=np.uint8)
    used, nd = ctypes.c_uint64(0), ctypes.c_uint64(0)
    rc = lib().orc_write_patch(len(arrs), ptrs, sizes, chunk, hptrs, generation, parent,
                               _ptr(out), out.size, ctypes.byref(used), ctypes.byref(nd))
    return rc, out[: used.value], int(nd.value)


def apply_patch(base: np.ndarray, patch: np.ndarray):
    """Applies `patch` to a copy of `base`; returns (status, new image)."""
    b = base.copy()
    rc = lib().orc_apply_patch(_ptr(b), b.size, _ptr(patch), patch.size)
    return rc, b


def patch_dirty(patch: np.ndarray, k: int):
    nd = ctypes.c_uint64(0)
    cap = 1 << 22
    idx = np.zeros(cap, dtype=np.uint32)
    rc = lib().orc_patch_dirty(_ptr(patch), patch.size, k, ctypes.byref(nd), _ptr(idx), cap)
    return rc, idx[: nd.value].copy()
