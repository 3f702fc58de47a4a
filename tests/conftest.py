import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HERE = os.path.dirname(os.path.abspath(__file__))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")


def _build_hwcrc():
    src = os.path.join(HERE, "_hwcrc.c")
    so = os.path.join(HERE, "_hwcrc.so")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-msse4.2", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, so)
    lib = ctypes.CDLL(so)
    lib.hw_crc32c.restype = ctypes.c_uint32
    lib.hw_crc32c.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    lib.hw_chunk_hashes.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
    return lib


class HwCrc:
    """CRC-32C by the SSE4.2 instruction (independent of the oracle)."""

    def __init__(self):
        self.lib = _build_hwcrc()

    def crc(self, data) -> int:
        a = np.ascontiguousarray(np.frombuffer(bytes(data), dtype=np.uint8)
                                 if isinstance(data, (bytes, bytearray)) else data,
                                 dtype=np.uint8).reshape(-1)
        return int(self.lib.hw_crc32c(a.ctypes.data if a.size else None, a.size))

    def chunks(self, data, C) -> np.ndarray:
        a = np.ascontiguousarray(data, dtype=np.uint8).reshape(-1)
        n = (a.size + C - 1) // C
        out = np.zeros(max(n, 1), dtype=np.uint32)
        self.lib.hw_chunk_hashes(a.ctypes.data if a.size else None, a.size, C, out.ctypes.data)
        return out[:n]


@pytest.fixture(scope="session")
def hwcrc():
    return HwCrc()


def load_golden_vectors():
    out = []
    with open(os.path.join(HERE, "golden", "crc32c_vectors.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, msg, exp = line.split()
            kind, arg = msg.split(":", 1)
            if kind == "ascii":
                data = arg.encode()
            elif kind == "hex":
                data = bytes.fromhex(arg)
            else:
                b, cnt = arg.split("x")
                b, cnt = int(b, 16), int(cnt)
                if kind == "fill":
                    data = bytes([b]) * cnt
                elif kind == "inc":
                    data = bytes((b + i) & 0xFF for i in range(cnt))
                else:
                    data = bytes((b - i) & 0xFF for i in range(cnt))
            out.append((name, data, int(exp, 16)))
    return out
