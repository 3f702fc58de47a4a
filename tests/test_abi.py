"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/snap.h declares (no GPU needed; no compute calls)."""
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
