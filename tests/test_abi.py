"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/snap.h declares (no GPU needed; no compute calls)."""
import ctypes
import os
import re
import subprocess

import paper_2502_16631_b300 as snap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        names |= set(re.findall(r"SNAP_API\s+[\w\s\*]*?\b(snap_\w+)\s*\(", src))
    return names


def test_header_declares_the_binding_exports():
    assert declared_symbols() == set(snap.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = snap.lib()
    out = subprocess.check_output(["nm", "-D", "--defined-only", snap.LIB_PATH], text=True)
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    for name in declared_symbols():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_library_is_built_for_sm_103a():
    out = subprocess.check_output(["cuobjdump", "--list-elf", snap.LIB_PATH], text=True)
    assert "sm_103a" in out


def test_strerror_names_every_status():
    for st in range(0, -12, -1):
        assert snap.strerror(st) != "unknown status"
    assert snap.strerror(-99) == "unknown status"


def test_no_gpu_means_a_loud_error_not_a_fallback():
    """Without a CUDA device every compute entry point fails with a status
    (the binding raises); nothing falls back to a CPU path."""
    import ctypes

    import pytest
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(snap.SnapError):
        snap.Set(chunk_bytes=65536)
    out = ctypes.c_void_p()
    assert snap.lib().snap_host_alloc(4096, ctypes.byref(out)) != snap.OK
    v = ctypes.c_double()
    assert snap.lib().snap_link_ceiling(-1, 0, 1 << 20, 1, ctypes.byref(v)) != snap.OK
    buf = (ctypes.c_uint32 * 4)()
    assert snap.lib().snap_hash_chunks(ctypes.cast(buf, ctypes.c_void_p), 16, 4096,
                                       ctypes.cast(buf, ctypes.c_void_p), None) != snap.OK


def test_host_only_calls_work_without_a_gpu():
    """The host-side entry points (status names, the two-phase protocol,
    argument checks) need no device."""
    assert snap.strerror(snap.EPEER) != "unknown status"
    seen = []
    rc = snap.coordinate(lambda ph, st: st, lock=lambda: seen.append("l") or 0,
                         run=lambda: seen.append("r") or 0, commit=lambda: seen.append("c"))
    assert rc == snap.OK and seen == ["l", "r", "c"]
    # argument checks come before any device call
    buf = (ctypes.c_uint8 * 16)()
    assert snap.lib().snap_host_register(None, 4096) == snap.EINVAL
    assert snap.lib().snap_host_register(ctypes.cast(buf, ctypes.c_void_p), 0) == snap.EINVAL
    assert snap.lib().snap_host_unregister(None) == snap.EINVAL
    # the measurement probes check their arguments first too
    v = ctypes.c_double()
    L = snap.lib()
    assert L.snap_host_copy_ceiling(0, 0, 1 << 30, 1, 0, ctypes.byref(v)) == snap.EINVAL   # no threads
    assert L.snap_host_copy_ceiling(4, 3, 1 << 30, 1, 0, ctypes.byref(v)) == snap.EINVAL   # no direction 3
    assert L.snap_host_copy_ceiling(1, 2, 1 << 30, 1, 0, ctypes.byref(v)) == snap.EINVAL   # both ways needs 2
    assert L.snap_host_copy_ceiling(4, 0, 4096, 1, 0, ctypes.byref(v)) == snap.EINVAL      # under 1 MiB
    assert L.snap_host_copy_ceiling(4, 0, 1 << 30, 0, 0, ctypes.byref(v)) == snap.EINVAL   # no rounds
    assert L.snap_host_copy_ceiling(4, 0, 1 << 30, 1, 0, None) == snap.EINVAL
    assert L.snap_link_ceiling(-1, 3, 1 << 20, 1, ctypes.byref(v)) == snap.EINVAL
    t = snap.Tuning()
    assert L.snap_get_tuning(None, 0, ctypes.byref(t)) == snap.EINVAL
    # set options are checked before the device is touched
    h = ctypes.c_void_p()
    for bad in (snap.Opts(chunk_bytes=1000), snap.Opts(chunk_bytes=32 << 20),
                snap.Opts(incr_copy=snap.INCR_COPY_DMA + 1)):
        assert L.snap_set_create(ctypes.byref(h), ctypes.byref(bad)) == snap.EINVAL and not h.value
