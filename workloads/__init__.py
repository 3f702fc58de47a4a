"""Seeded synthetic workloads shared by the tests, the smoke check and bench.py.

This module holds no arithmetic of the snapshot method (no hashing, no image
layout): it only produces allocation-size lists, model-shaped tensor lists,
byte contents and mutation sets.  Both the CUDA path and the oracle consume
what it generates; the oracle always reads back the actual device bytes, so
the choice of random generator never affects parity.

Workloads (synthetic stand-ins for the paper's training/HPC state, Sec. 5):
  * random allocations: log-uniform sizes, rounded to 4 KiB, scaled to an
    exact total; bytes from per-allocation xorshift64* streams;
  * GPT-2-small training state (124,439,808 params, 148 tensors x 4 kinds
    fp32 + a 256 MiB bf16 activation buffer = 2,259,472,384 B);
  * Llama-7B-shaped state (6,738,415,616 params, bf16 weights + fp32
    master/m/v + 20 GiB bf16 activations);
  * clustered mutation runs (geometric run length, mean 16 units).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

M64 = (1 << 64) - 1
PAGE = 4096
KiB, MiB, GiB = 1 << 10, 1 << 20, 1 << 30


# --------------------------------------------------------------- generators
def splitmix64(x: int) -> int:
    """One output of Vigna's splitmix64 for state x (state advance included)."""
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


class Rng:
    """xorshift64* (Vigna) seeded through splitmix64; for small draws."""

    def __init__(self, seed: int):
        self.x = splitmix64(seed & M64) or 0x9E3779B97F4A7C15

    def next_u64(self) -> int:
        x = self.x
        x ^= x >> 12
        x ^= (x << 25) & M64
        x ^= x >> 27
        self.x = x
        return (x * 0x2545F4914F6CDD1D) & M64

    def uniform(self) -> float:
        """U in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) / float(1 << 53)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + int(self.uniform() * (hi - lo + 1))

    def geometric(self, p: float) -> int:
        """Number of trials to the first success (>= 1)."""
        u = self.uniform()
        return 1 + int(math.floor(math.log1p(-u) / math.log1p(-p)))


_FILL_SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_fill.c")
_FILL_LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfill.so")
_fill = None


def _fill_lib():
    global _fill
    if _fill is None:
        if not os.path.exists(_FILL_LIB) or os.path.getmtime(_FILL_LIB) < os.path.getmtime(_FILL_SRC):
            tmp = _FILL_LIB + ".tmp%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _FILL_SRC])
            os.replace(tmp, _FILL_LIB)
        _fill = ctypes.CDLL(_FILL_LIB)
        _fill.fill_xorshift64star.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]
    return _fill


def xorshift_bytes(nbytes: int, seed: int, k: int = 0) -> np.ndarray:
    """Bytes of the xorshift64* stream for allocation k: state seeded with
    splitmix64(seed ^ k); each step emits 8 little-endian bytes."""
    out = np.empty(nbytes, dtype=np.uint8)
    if nbytes:
        s = splitmix64((seed ^ k) & M64) or 0x9E3779B97F4A7C15
        _fill_lib().fill_xorshift64star(out.ctypes.data, nbytes, s)
    return out


# ------------------------------------------------------------------- sizes
def _round_page(x: float) -> int:
    return max(PAGE, int(round(x / PAGE)) * PAGE)


def log_uniform_sizes(n: int, lo: int, hi: int, total: int | None, seed: int) -> list[int]:
    """n sizes log-uniform in [lo, hi], rounded to 4 KiB (min 4 KiB); if total
    is given they are scaled to sum to exactly `total` (floor to 4 KiB, then
    the remainder goes to the largest, lowest index on ties)."""
    r = Rng(seed)
    s = [_round_page(math.exp(r.uniform() * math.log(hi / lo)) * lo) for _ in range(n)]
    if total is None:
        return s
    tot = sum(s)
    s2 = [max(PAGE, (int(v * total / tot) // PAGE) * PAGE) for v in s]
    big = max(range(n), key=lambda i: (s2[i], -i))
    s2[big] += total - sum(s2)
    assert sum(s2) == total and min(s2) > 0
    return s2


def config1_sizes(seed: int = 1) -> list[int]:
    """16 allocations, log-uniform [64 KiB, 16 MiB], exactly 64 MiB total."""
    return log_uniform_sizes(16, 64 * KiB, 16 * MiB, 64 * MiB, seed)


def config3_sizes(seed: int = 1, total: int = 20 * GiB, n: int = 2000) -> list[int]:
    """2,000 allocations, log-uniform [4 KiB, 256 MiB], scaled to 20 GiB."""
    return log_uniform_sizes(n, 4 * KiB, 256 * MiB, total, seed)


def config5_tenants(seed: int = 1, n_tenants: int = 32, cap: int = 4 * GiB,
                    lo: int = 1 * MiB, hi: int = 2 * GiB) -> list[list[int]]:
    """32 tenants; each 8-64 allocations log-uniform [1 MiB, 2 GiB]; a
    tenant whose sum exceeds 4 GiB is scaled down to exactly 4 GiB."""
    r = Rng(seed ^ 0x5E4F)
    out = []
    for t in range(n_tenants):
        n = r.randint(8, 64)
        s = log_uniform_sizes(n, lo, hi, None, seed * 1000003 + t)
        if sum(s) > cap:
            s = log_uniform_sizes(n, lo, hi, cap, seed * 1000003 + t)
        out.append(s)
    return out


# ------------------------------------------------------------ model shapes
def gpt2_small_tensors(vocab=50257, ctx=1024, d=768, layers=12):
    """HF GPT-2 layout with biases, tied LM head: 148 tensors."""
    t = [("wte", vocab * d), ("wpe", ctx * d)]
    for i in range(layers):
        p = "h.%d." % i
        t += [(p + "ln_1.weight", d), (p + "ln_1.bias", d),
              (p + "attn.c_attn.weight", d * 3 * d), (p + "attn.c_attn.bias", 3 * d),
              (p + "attn.c_proj.weight", d * d), (p + "attn.c_proj.bias", d),
              (p + "ln_2.weight", d), (p + "ln_2.bias", d),
              (p + "mlp.c_fc.weight", d * 4 * d), (p + "mlp.c_fc.bias", 4 * d),
              (p + "mlp.c_proj.weight", 4 * d * d), (p + "mlp.c_proj.bias", d)]
    t += [("ln_f.weight", d), ("ln_f.bias", d)]
    return t


def llama7b_tensors(vocab=32000, d=4096, ffn=11008, layers=32):
    """Llama-7B layout, untied head, no biases: 291 tensors."""
    t = [("embed_tokens", vocab * d)]
    for i in range(layers):
        p = "layers.%d." % i
        t += [(p + "q_proj", d * d), (p + "k_proj", d * d), (p + "v_proj", d * d),
              (p + "o_proj", d * d), (p + "gate_proj", ffn * d), (p + "up_proj", ffn * d),
              (p + "down_proj", d * ffn), (p + "input_layernorm", d),
              (p + "post_attention_layernorm", d)]
    t += [("norm", d), ("lm_head", vocab * d)]
    return t


def gpt2_state_spec(act_bytes: int = 256 * MiB):
    """(name, numel, dtype, dist, std) per allocation of the GPT-2-small
    training state: fp32 W ~N(0,0.02), G ~N(0,1e-3), m ~N(0,1e-4),
    v = |N(0,1e-6)|, plus one bf16 activation buffer ~N(0,1)."""
    spec = []
    for kind, std, absval in (("w", 0.02, False), ("g", 1e-3, False), ("m", 1e-4, False),
                              ("v", 1e-6, True)):
        for name, n in gpt2_small_tensors():
            spec.append((kind + "." + name, n, "float32", "abs_normal" if absval else "normal", std))
    spec.append(("activations", act_bytes // 2, "bfloat16", "normal", 1.0))
    return spec


def llama7b_state_spec(act_total: int = 20 * GiB, act_bufs: int = 32):
    """Llama-7B-shaped state: bf16 W ~N(0,0.02), fp32 master ~N(0,0.02),
    fp32 m ~N(0,1e-4), fp32 v = |N(0,1e-6)|, 32 bf16 activation buffers."""
    spec = []
    for kind, dtype, std, absval in (("w", "bfloat16", 0.02, False), ("master", "float32", 0.02, False),
                                     ("m", "float32", 1e-4, False), ("v", "float32", 1e-6, True)):
        for name, n in llama7b_tensors():
            spec.append((kind + "." + name, n, dtype, "abs_normal" if absval else "normal", std))
    per = act_total // act_bufs
    for i in range(act_bufs):
        spec.append(("activations.%d" % i, per // 2, "bfloat16", "normal", 1.0))
    return spec


def spec_bytes(spec) -> list[int]:
    return [n * (2 if dt == "bfloat16" else 4) for _, n, dt, _, _ in spec]


# ---------------------------------------------------------------- mutation
def mutation_units(n_units: int, frac: float, seed: int, mean_run: int = 16) -> np.ndarray:
    """Distinct unit indices (ascending) to mutate: runs over the global unit
    index space, start uniform, length ~ Geometric(1/mean_run) >= 1, clipped
    at the end; repeated until round(frac*N) distinct units, last run trimmed."""
    target = int(round(frac * n_units))
    r = Rng(seed ^ 0x4D55)
    hit = np.zeros(n_units, dtype=bool)
    count = 0
    while count < target:
        start = r.randint(0, n_units - 1)
        length = r.geometric(1.0 / mean_run)
        for u in range(start, min(n_units, start + length)):
            if not hit[u]:
                hit[u] = True
                count += 1
                if count == target:
                    break
    return np.nonzero(hit)[0]


# ------------------------------------------------------- device fill helpers
def torch_fill_spec(tensors, spec, seed: int):
    """Fill device tensors (one per spec entry) with their distributions,
    using a seeded CUDA generator."""
    import torch
    g = torch.Generator(device=tensors[0].device)
    g.manual_seed(seed)
    for t, (_, n, dt, dist, std) in zip(tensors, spec):
        tt = t.view(torch.bfloat16 if dt == "bfloat16" else torch.float32)
        tt.normal_(0.0, std, generator=g)
        if dist == "abs_normal":
            tt.abs_()


def torch_random_bytes(t, seed: int):
    """Fill a uint8 device tensor with seeded random bytes."""
    import torch
    g = torch.Generator(device=t.device)
    g.manual_seed(seed)
    t.copy_(torch.randint(0, 256, t.shape, dtype=torch.uint8, device=t.device, generator=g))
