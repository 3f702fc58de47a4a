#!/usr/bin/env python
"""Benchmark of the snapshot/restore hot path on B300.

Default step (`--workload llama7b`): the Llama-7B-shaped training state
(1,196 allocations, 115,812,655,104 B; 64 KiB chunks), the largest state of
the workloads that fits one GPU:

  1. full checkpoint  (quiesce, then window by window: CRC-32C of every chunk
                       fused with the gather into a slot of the set's 4 GiB
                       pinned ring, host workers copying filled slots into
                       the pageable host image)
  2. restore          (the image back through the ring into a second,
                       separately allocated set of device buffers)

The two buffer sets swap roles every step, so each step checkpoints what the
previous step restored.  `value` = 2 x state bytes per step / step time
(CUDA events around the timed steps); per-call rates, the kernels' roofline
against the host link, and the GPT-2-small step (`gpt2_step`: full +
incremental + verify + restore with pinned images, and the plain
one-cudaMemcpyAsync-per-allocation form) are reported beside it.
`--impl reference` runs the CPU oracle (the same step on a bounded sample of
the same state) instead; `--workload` selects the other workloads.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "snapshot/restore GB/s vs host-link roofline; incremental GB/s; p99 latency"
KiB, MiB, GiB = 1 << 10, 1 << 20, 1 << 30
UNIT = 65536


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["snap", "reference"], default="snap")
    p.add_argument("--dirty", type=float, default=0.10)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-bytes", type=int, default=512 * MiB)
    p.add_argument("--no-gpt2-extra", action="store_true", help="llama7b: skip the GPT-2-small step "
                   "reported beside the default line")
    p.add_argument("--workload", default="llama7b",
                   choices=["gpt2", "random64m", "incr20g", "llama7b", "serving", "async", "lazy", "file", "hash"],
                   help="llama7b: 115.8 GB Llama-7B state through the pinned ring, checkpoint + restore into "
                        "other buffers (default); gpt2: GPT-2-small training state, full + incremental + "
                        "verify + restore; random64m: 16 random allocations, "
                        "64 MiB; incr20g: 20 GiB incremental at 1/10/50%% dirty with the chunk-size sweep; "
                        "serving: 32 tenants, "
                        "Poisson arrivals; async: GPT-2 state checkpointed asynchronously under a bf16 "
                        "matmul load, against the synchronous call; lazy: GPT-2 state restored weights "
                        "first, time until the weights are usable; file: GPT-2 state checkpointed to and "
                        "restored from an image file; hash: the chunk hasher alone over 8 GiB")
    p.add_argument("--file-dir", default=None, help="file: directory for the image files (default: the "
                   "system temporary directory)")
    p.add_argument("--load-gemms", type=int, default=0, help="async: matmuls per step (0: about 3x the "
                   "background part)")
    p.add_argument("--async-ctas", default="0,4,37", help="async: background grids to measure (0: the "
                   "library default, which gives the reported value)")
    p.add_argument("--incr-chunks", default="16,32,64,128,256,512,1024",
                   help="incr20g: chunk sizes of the sweep (KiB, comma-separated)")
    p.add_argument("--arrivals", type=int, default=1200, help="serving: requests")
    p.add_argument("--rate", type=float, default=20.0, help="serving: arrivals per second")
    p.add_argument("--serve-pool-gib", type=int, default=24, help="serving: pinned staging pool (GiB, within "
                   "the 64 GB pinned budget)")
    p.add_argument("--no-plain", action="store_true", help="serving: skip the serial plain-copy comparison")
    p.add_argument("--serve-lower-rates", default="12", help="serving: further arrival rates (comma-separated) "
                   "run for context after the main one, each over half the main run's span")
    p.add_argument("--serve-pin-gb", type=float, default=0.0, help="serving: GB of tenant images to pin "
                   "(snap_host_register) for direct access, within the 64 GB pinned budget beside the pool "
                   "(default 0: measured slower under this mix)")
    return p.parse_args()


# ------------------------------------------------------------------ ranks
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def reduce_max(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def link_peak(torch, nbytes=1 * GiB, reps=5):
    """Pinned cudaMemcpyAsync D2H / H2D GB/s, best of reps (the copy engine:
    the host-link roofline the gather and scatter kernels are held to)."""
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    out = {}
    for name, (dst, src) in (("d2h", (h, d)), ("h2d", (d, h))):
        best = 0.0
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            dst.copy_(src, non_blocking=True)
            b.record()
            torch.cuda.synchronize()
            best = max(best, nbytes / (a.elapsed_time(b) * 1e-3) / 1e9)
        out[name] = best
    del d, h
    import paper_2502_16631_b300 as snap
    # the ceiling of SM-initiated traffic, which the gather and scatter use
    out["sm_d2h"] = snap.link_ceiling(0, nbytes, 3)
    out["sm_h2d"] = snap.link_ceiling(1, nbytes, 3)
    return out


def link_peak_both(torch, nbytes=1 * GiB, reps=3):
    """Both link directions at once (the serving loop's case): copy engines on
    two streams, and SM loads/stores with half the warps each way; GB/s of
    the two directions' bytes together."""
    import paper_2502_16631_b300 as snap
    d1 = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d2 = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    h1 = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h2 = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    best = 0.0
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s1):
            h1.copy_(d1, non_blocking=True)
        with torch.cuda.stream(s2):
            d2.copy_(h2, non_blocking=True)
        torch.cuda.synchronize()
        best = max(best, 2 * nbytes / (time.perf_counter() - t0) / 1e9)
    del d1, d2, h1, h2
    return {"ce_both": best, "sm_both": snap.link_ceiling(2, nbytes, 3)}


def kernel_source_key(path: str) -> str:
    """sha256[:16] of a CUDA source with comments and whitespace removed: the
    key under which measured counters stay valid (a comment edit keeps it)."""
    import re
    src = open(path, encoding="utf-8").read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return hashlib.sha256("".join(src.split()).encode()).hexdigest()[:16]


def traffic_ratio_from_profiles(kernel: str):
    """DRAM bytes per state byte of `kernel` from the committed ncu summary
    (profiles/traffic.txt, `ratio` rows), valid only while the kernel source
    (its code, not its comments) is unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = os.path.join(ROOT, "paper_2502_16631_b300", "csrc", "kernels.cu")
    try:
        sha = kernel_source_key(src)
        for line in open(path):
            parts = line.split()
            if len(parts) >= 4 and parts[0] == kernel and parts[1] == "ratio" and parts[3] == sha:
                return float(parts[2])
    except (OSError, ValueError):
        pass
    return None


def gather_traffic(state_bytes: int):
    """DRAM bytes of one full-gather launch over `state_bytes`: the committed
    per-launch figure for this kernel code, else its committed ratio times
    the state bytes (one read per state byte), else None."""
    t = traffic_from_profiles("snap_tiles_gather")
    if t is None:
        r = traffic_ratio_from_profiles("snap_tiles_gather")
        t = None if r is None else int(r * state_bytes)
    return t


def traffic_from_profiles(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, valid
    only while the kernel source (its code, not its comments) is unchanged
    since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = os.path.join(ROOT, "paper_2502_16631_b300", "csrc", "kernels.cu")
    try:
        sha = kernel_source_key(src)
        for line in open(path):
            parts = line.split()
            if len(parts) >= 4 and parts[0] == kernel and parts[1] != "ratio" and parts[3] == sha:
                return int(parts[2])
    except (OSError, ValueError):
        pass
    return None


def gpt2_layout():
    spec = workloads.gpt2_state_spec()
    sizes = workloads.spec_bytes(spec)
    starts, off = [], 0
    for n in sizes:  # every allocation starts on a 64 KiB unit of the arena
        starts.append(off)
        off += (n + UNIT - 1) // UNIT * UNIT
    return spec, sizes, starts, off


def dirty_units(sizes, starts, frac, seed):
    """Arena units of the mutated chunks: the chunk set is drawn over the
    global chunk index space (clustered runs, mean 16), then mapped to units."""
    nch = [(n + UNIT - 1) // UNIT for n in sizes]
    chunk0 = np.concatenate([[0], np.cumsum(nch)])
    chosen = workloads.mutation_units(int(chunk0[-1]), frac, seed)
    k = np.searchsorted(chunk0, chosen, side="right") - 1
    i = chosen - chunk0[k]
    return (np.asarray(starts)[k] // UNIT + i).astype(np.int64)


# ---------------------------------------------------------------- CPU arm
def oracle_step_sample(sample, frac, seed):
    """The same step run by the CPU oracle on host copies of a sample of
    allocations; returns a callable and the sample's byte count."""
    import oracle
    nb = sum(a.size for a in sample)
    rng = np.random.default_rng(seed)
    units = []
    for k, a in enumerate(sample):
        n = (a.size + UNIT - 1) // UNIT
        for i in range(n):
            if rng.random() < frac:
                units.append((k, i))
    masks = [rng.integers(1, 256, min(UNIT, sample[k].size - i * UNIT), dtype=np.uint8) for k, i in units]
    state = [a.copy() for a in sample]

    def step():
        rc, img = oracle.write_full(state, UNIT, 0)
        prev = [oracle.chunk_hashes(a, UNIT) for a in state]
        for (k, i), m in zip(units, masks):
            state[k][i * UNIT: i * UNIT + m.size] ^= m
        rc, patch, _ = oracle.write_patch(state, UNIT, prev, 1, 0)
        rc, _ = oracle.verify(img, state)
        rc, restored = oracle.restore(img, [a.size for a in state])
        for a, r in zip(state, restored):
            a[:] = r
    return step, nb


def oracle_ckpt_restore_sample(sample):
    """The default step (full checkpoint + restore) run by the CPU oracle on
    host copies of a sample of allocations; returns a callable and the
    sample's byte count."""
    import oracle
    nb = sum(a.size for a in sample)
    sizes = [a.size for a in sample]
    state = [a.copy() for a in sample]

    def step():
        rc, img = oracle.write_full(state, UNIT, 0)
        rc2, restored = oracle.restore(img, sizes)
        if rc or rc2:
            raise RuntimeError("oracle step failed: %d %d" % (rc, rc2))
        for a, r in zip(state, restored):
            a[:] = r
    return step, nb


def cpu_baseline(sample, args, seconds_target=15.0, kind="gpt2", what=""):
    """The oracle as it stands, on the host cores: the workload's step on a
    bounded sample (`kind` "gpt2": full + incremental + verify + restore,
    4 x sample bytes per step; "llama7b": full + restore, 2 x)."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    mult = 4 if kind == "gpt2" else 2

    def make():
        if kind == "gpt2":
            return oracle_step_sample(sample, args.dirty, args.seed)
        return oracle_ckpt_restore_sample(sample)
    oracle.set_threads(cores)
    step, nb = make()
    step()  # warm
    t0 = time.perf_counter()
    n = 0
    while True:
        step()
        n += 1
        if time.perf_counter() - t0 > seconds_target or n >= 50:
            break
    dt = (time.perf_counter() - t0) / n
    # the same step on one thread (a few seconds)
    oracle.set_threads(1)
    step1, _ = make()
    t1 = time.perf_counter()
    n1 = 0
    while n1 < 1 or (time.perf_counter() - t1 < seconds_target / 3 and n1 < 10):
        step1()
        n1 += 1
    dt1 = (time.perf_counter() - t1) / n1
    oracle.set_threads(cores)
    steps = "full+incremental+verify+restore" if kind == "gpt2" else "full checkpoint + restore"
    return {"value": mult * nb / dt / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "value_1_thread": mult * nb / dt1 / 1e9,
            "sample": "first %d %s allocations (%d B), %d steps of %s, %.1f s on %d cores; %d steps on 1 "
                      "thread; host copies of the state, so no device read-back is timed"
                      % (len(sample), what or kind, nb, n, steps, dt * n, cores, n1)}


def sample_allocations(spec, cap_bytes, seed):
    """Host copies of the first allocations of a state spec (up to cap_bytes),
    drawn from the same distributions as the device state."""
    rng = np.random.default_rng(seed)
    out, tot = [], 0
    for (name, n, dt, dist, std) in spec:
        if tot >= cap_bytes:
            break
        if dt == "bfloat16":
            x = (rng.standard_normal(n, dtype=np.float32) * np.float32(std)).view(np.uint32) >> 16
            b = x.astype(np.uint16).view(np.uint8)
        else:
            x = rng.standard_normal(n, dtype=np.float32) * np.float32(std)
            if dist == "abs_normal":
                x = np.abs(x)
            b = x.view(np.uint8)
        out.append(b)
        tot += b.size
    return out


def run_reference(args, rank, world):
    """The CPU oracle on a bounded sample of the workload of `--workload`
    (llama7b: the default step, full checkpoint + restore; gpt2: its
    four-call step), timed on the host cores."""
    if rank != 0:
        return
    import oracle
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    if args.workload == "gpt2":
        sample = sample_allocations(workloads.gpt2_state_spec(), args.cpu_sample_bytes, args.seed)
        step, nb = oracle_step_sample(sample, args.dirty, args.seed)
        mult, config, what = 4, gpt2_config(args), "GPT-2-state"
    else:
        sample = sample_allocations(workloads.llama7b_state_spec(), args.cpu_sample_bytes, args.seed)
        step, nb = oracle_ckpt_restore_sample(sample)
        mult, config, what = 2, llama7b_config(args), "Llama-7B-state"
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    v = mult * nb / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": "first %d %s allocations (%d B) per step" % (len(sample), what, nb)},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def gpt2_config(args):
    return {"workload": "GPT-2-small training state: 593 allocations (148 tensors x fp32 W/G/m/v + 256 MiB "
                        "bf16 activations), 2,259,472,384 B, 64 KiB CRC-32C chunks",
            "step": "full checkpoint + %.0f%% clustered mutation + incremental checkpoint + verify + restore"
                    % (100 * args.dirty),
            "state_bytes": 2259472384, "chunk_bytes": UNIT, "dirty_frac": args.dirty,
            "image": "pinned, device-mapped host memory",
            "l2": "inputs (2.26 GB) larger than the 126 MB L2; no flush"}


def llama7b_config(args, state_bytes=115812655104, n_allocs=1196, reduced=None):
    c = {"workload": "Llama-7B-shaped training state: %d allocations (291 tensors x bf16 W, fp32 master, fp32 "
                     "Adam m and v + 32 bf16 activation buffers of 640 MiB), %d B, 64 KiB CRC-32C chunks"
                     % (n_allocs, state_bytes),
         "step": "full checkpoint through the 4 GiB pinned ring into a pageable host image + restore of that "
                 "image into a second, separately allocated set of device buffers (the sets swap roles "
                 "every step)",
         "state_bytes": state_bytes, "chunk_bytes": UNIT, "ring_bytes": 4 * GiB,
         "image": "pageable host memory (mmap, populated before the timed region)",
         "l2": "115.8 GB state, far larger than the 126 MB L2; no flush"}
    if reduced:
        c["reduced"] = reduced
    return c


# ---------------------------------------------------------------- GPU arm
def measure_gpt2(args, rank, world, local, pg, steps, warmup, with_cpu):
    """The GPT-2-small step (full checkpoint + mutation + incremental +
    verify + restore, pinned images); returns its JSON line."""
    import torch
    import paper_2502_16631_b300 as snap
    torch.cuda.set_device(local)
    spec, sizes, starts, arena_bytes = gpt2_layout()
    arena = torch.zeros(arena_bytes, dtype=torch.uint8, device="cuda")
    views = [arena[s: s + n] for s, n in zip(starts, sizes)]
    workloads.torch_fill_spec(views, spec, seed=args.seed + rank)
    B = sum(sizes)
    s = snap.Set(chunk_bytes=UNIT)
    for v in views:
        s.register(v)
    full = snap.HostBuffer(s.image_bytes(snap.FULL))
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    units = torch.from_numpy(dirty_units(sizes, starts, args.dirty, args.seed)).cuda()
    g = torch.Generator(device="cuda")
    g.manual_seed(args.seed + 1000)
    masks = torch.randint(1, 256, (units.numel(), UNIT), dtype=torch.uint8, device="cuda", generator=g)
    grid = arena.view(-1, UNIT)

    per = {"full": [], "incr": [], "verify": [], "restore": [], "gather_kernel": [], "scatter_kernel": [],
           "hash_kernel": [], "diff": [], "dirty_gather": [], "verify_kernel": []}
    counts = {"kernels": 0, "patch_bytes": 0, "dirty": 0}

    def step(record):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        e[0].record()
        used_full = s.checkpoint(full, snap.FULL)
        st_full = s.stats()
        e[1].record()
        grid[units] ^= masks  # the training step between snapshots (not libsnap)
        e[2].record()
        used_patch = s.checkpoint(patch, snap.INCREMENTAL)
        st_incr = s.stats()
        e[3].record()
        bad = s.verify(patch, used_patch)
        st_ver = s.stats()
        e[4].record()
        s.restore(full, used_full)
        st_res = s.stats()
        e[5].record()
        if bad != 0:  # the patch's hashes describe the mutated state exactly
            raise RuntimeError("verify against the patch found %d mismatches" % bad)
        if record:
            torch.cuda.synchronize()
            per["full"].append(e[0].elapsed_time(e[1]))
            per["incr"].append(e[2].elapsed_time(e[3]))
            per["verify"].append(e[3].elapsed_time(e[4]))
            per["restore"].append(e[4].elapsed_time(e[5]))
            per["gather_kernel"].append(st_full["copy_ms"])
            per["scatter_kernel"].append(st_res["copy_ms"])
            per["hash_kernel"].append(st_incr["hash_ms"])
            per["verify_kernel"].append(st_ver["hash_ms"])
            per["diff"].append(st_incr["diff_ms"])
            per["dirty_gather"].append(st_incr["copy_ms"])
            counts["kernels"] += sum(int(x["kernel_launches"]) for x in (st_full, st_incr, st_ver, st_res))
            counts["patch_bytes"] = used_patch
            counts["dirty"] = st_incr["dirty_chunks"]
        return used_full, used_patch

    for _ in range(warmup):
        step(False)
    peaks = link_peak(torch)
    clocks = ClockSampler(local)
    barrier(pg)
    torch.cuda.synchronize()
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    h0 = time.perf_counter()
    t_start.record()
    for _ in range(steps):
        used_full, used_patch = step(True)
    t_end.record()
    torch.cuda.synchronize()
    h1 = time.perf_counter()
    barrier(pg)
    clk = clocks.stop()
    ms = t_start.elapsed_time(t_end) / steps
    ms_max = reduce_max(pg, ms)
    host_ms_max = reduce_max(pg, (h1 - h0) * 1e3 / steps)
    total_bytes = reduce_sum(pg, 4.0 * B)
    value = total_bytes / (ms_max * 1e-3) / 1e9

    # the same step with ordinary pageable images (numpy arrays): the library
    # streams them through its pinned ring, host copies included
    pg_full = np.empty(full.nbytes, np.uint8)
    pg_patch = np.empty(patch.nbytes, np.uint8)

    def step_pageable():
        uf = s.checkpoint(pg_full, snap.FULL)
        grid[units] ^= masks
        up = s.checkpoint(pg_patch, snap.INCREMENTAL)
        bad = s.verify(pg_patch, up)
        s.restore(pg_full, uf)
        if bad != 0:
            raise RuntimeError("verify against the pageable patch found %d mismatches" % bad)
    step_pageable()
    torch.cuda.synchronize()
    n_pageable = 3
    h2 = time.perf_counter()
    for _ in range(n_pageable):
        step_pageable()
    torch.cuda.synchronize()
    pageable_ms = (time.perf_counter() - h2) * 1e3 / n_pageable
    del pg_full, pg_patch

    # plain form (one cudaMemcpyAsync per allocation, full copy every time)
    plain_c, plain_r = [], []
    for _ in range(3):
        t0 = time.perf_counter()
        s.plain_checkpoint(full)
        t1 = time.perf_counter()
        s.plain_restore(full)
        t2 = time.perf_counter()
        plain_c.append(t1 - t0)
        plain_r.append(t2 - t1)
    plain_ckpt_gbs = B / min(plain_c) / 1e9
    incr_gbs = B / (statistics.median(per["incr"]) * 1e-3) / 1e9

    gather_ms = statistics.mean(per["gather_kernel"])
    achieved = B / (gather_ms * 1e-3) / 1e9
    pk = measured_peaks()
    hbm_peak = pk.get("hbm_gbs", 6400.0)
    # the hash pass alone: the verify call's kernel (hash + compare with the
    # patch's hashes) over the whole state; the incremental call's hash phase
    # overlaps its dirty gather (pipelined), so it is not a clean figure
    hash_ms = statistics.mean(per["verify_kernel"])
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": gpt2_config(args),
        "roofline": {"bound": "host_link", "kernel": "snap_tiles (OP_GATHER, full checkpoint)",
                     "achieved": achieved, "peak": peaks["d2h"], "unit": "GB/s", "frac": achieved / peaks["d2h"],
                     "peak_source": "pinned cudaMemcpyAsync D2H, 1 GiB, best of 5, measured in this run",
                     "traffic": gather_traffic(B),
                     "sm_path_peak": peaks["sm_d2h"], "frac_of_sm_path": achieved / peaks["sm_d2h"]},
        "roofline_restore": {"bound": "host_link", "kernel": "snap_tiles (OP_SCATTER)",
                             "achieved": B / (statistics.mean(per["scatter_kernel"]) * 1e-3) / 1e9,
                             "peak": peaks["h2d"], "unit": "GB/s",
                             "frac": B / (statistics.mean(per["scatter_kernel"]) * 1e-3) / 1e9 / peaks["h2d"],
                             "sm_path_peak": peaks["sm_h2d"],
                             "frac_of_sm_path": B / (statistics.mean(per["scatter_kernel"]) * 1e-3) / 1e9
                             / peaks["sm_h2d"]},
        "roofline_hash": {"bound": "hbm", "kernel": "snap_tiles (OP_VERIFY: the hash pass plus the compare)",
                          "achieved": B / (hash_ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                          "frac": B / (hash_ms * 1e-3) / 1e9 / hbm_peak,
                          "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
        "breakdown": {
            "full_checkpoint_gbs": B / (statistics.median(per["full"]) * 1e-3) / 1e9,
            "incremental_gbs": incr_gbs,
            "verify_gbs": B / (statistics.median(per["verify"]) * 1e-3) / 1e9,
            "restore_gbs": B / (statistics.median(per["restore"]) * 1e-3) / 1e9,
            "plain_checkpoint_gbs": plain_ckpt_gbs,
            "plain_restore_gbs": B / min(plain_r) / 1e9,
            "incremental_vs_plain_full": incr_gbs / plain_ckpt_gbs,
            "dirty_chunks": counts["dirty"], "patch_bytes": counts["patch_bytes"],
            "hash_ms": hash_ms, "incremental_hash_phase_ms": statistics.mean(per["hash_kernel"]),
            "diff_ms": statistics.mean(per["diff"]),
            "dirty_gather_ms": statistics.mean(per["dirty_gather"]),
            "gather_kernel_ms": gather_ms, "scatter_kernel_ms": statistics.mean(per["scatter_kernel"]),
            # per call over the timed steps: median and standard deviation (ms)
            "call_ms": {k: {"median": statistics.median(per[k]),
                            "std": statistics.stdev(per[k]) if len(per[k]) > 1 else 0.0}
                        for k in ("full", "incr", "verify", "restore")},
        },
        "link_peak_gbs": peaks,
        "e2e": {"value": total_bytes / (host_ms_max * 1e-3) / 1e9, "unit": "GB/s",
                # restored state bytes + the hash tables uploaded by restore and verify
                "h2d_bytes_per_step": B + 2 * 4 * sum((n + UNIT - 1) // UNIT for n in sizes),
                # the full image and the patch written over the link
                "d2h_bytes_per_step": used_full + used_patch,
                "note": "host wall clock around the public API calls of the step (Python binding -> C ABI "
                        "-> graph launch -> completion), images in pinned host memory"},
        "e2e_pageable": {"value": total_bytes / (reduce_max(pg, pageable_ms) * 1e-3) / 1e9, "unit": "GB/s",
                         "steps": n_pageable,
                         "note": "the same step with numpy (pageable) images, streamed through the library's "
                                 "pinned ring with host copies; host wall clock"},
        "gpu_launches": counts["kernels"],
        "clocks": clk,
    }
    if with_cpu and rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = [v.cpu().numpy() for v in views[: max(1, _first_n(sizes, args.cpu_sample_bytes))]]
        line["cpu_baseline"] = cpu_baseline(sample, args, kind="gpt2", what="GPT-2-state")
    s.close()
    full.close()
    patch.close()
    del arena, views, grid, masks, units
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return line


def run_snap(args, rank, world, local, pg):
    line = measure_gpt2(args, rank, world, local, pg, args.steps, max(3, args.warmup), True)
    if rank == 0:
        print(json.dumps(line))


# ------------------------------------------------------ further workloads
def _line(args, world, value, ms, config, extra):
    d = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
         "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
         "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": config}
    d.update(extra)
    return d


def _ev():
    import torch
    return torch.cuda.Event(enable_timing=True)


def run_random64m(args, rank, world, local, pg):
    """16 allocations log-uniform in [64 KiB, 16 MiB], exactly 64 MiB of
    xorshift64* bytes; step = full checkpoint + restore."""
    import torch
    import oracle
    import paper_2502_16631_b300 as snap
    sizes = workloads.config1_sizes(args.seed)
    host = [workloads.xorshift_bytes(n, args.seed, k) for k, n in enumerate(sizes)]
    ts = [torch.from_numpy(h).cuda() for h in host]
    B = sum(sizes)
    s = snap.Set(chunk_bytes=UNIT)
    for t in ts:
        s.register(t)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    used = s.checkpoint(img, snap.FULL)
    ok_img = bool(np.array_equal(img.view(used), oracle.write_full(host, UNIT, 0)[1]))
    s.restore(img, used)
    ok_rest = all(np.array_equal(t.cpu().numpy(), h) for t, h in zip(ts, host))
    for _ in range(max(3, args.warmup)):
        s.checkpoint(img, snap.FULL)
        s.restore(img, used)
    peaks = link_peak(torch)
    clocks = ClockSampler(local)
    clocks.start()
    g, sc, kern = [], [], 0
    # a 64 MiB step takes ~3 ms: repeat the K steps until the timed region
    # lasts a second, so that the clock sampler sees it
    reps = max(1, int(1000.0 / (3.0 * args.steps)) + 1)
    a, b = _ev(), _ev()
    torch.cuda.synchronize()
    a.record()
    for _ in range(args.steps * reps):
        s.checkpoint(img, snap.FULL)
        st = s.stats()
        g.append(st["copy_ms"])
        kern += st["kernel_launches"]
        s.restore(img, used)
        st = s.stats()
        sc.append(st["copy_ms"])
        kern += st["kernel_launches"]
    b.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = a.elapsed_time(b) / (args.steps * reps)
    ach = B / (statistics.mean(g) * 1e-3) / 1e9
    oracle.set_threads(len(os.sched_getaffinity(0)))
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < 10 and n < 20:
        rc, im = oracle.write_full(host, UNIT, 0)
        oracle.restore(im, sizes)
        n += 1
    cpu = {"value": 2 * B / ((time.perf_counter() - t0) / n) / 1e9, "unit": "GB/s",
           "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
           "sample": "the whole 64 MiB state, %d full image writes + restores" % n}
    print(json.dumps(_line(args, world, 2 * B / (ms * 1e-3) / 1e9, ms,
                           {"workload": "16 random allocations, log-uniform [64 KiB, 16 MiB], 67,108,864 B, "
                                        "64 KiB chunks", "step": "full checkpoint + restore",
                            "l2": "64 MiB fits in L2: steps run back to back without a flush"},
                           {"roofline": {"bound": "host_link", "kernel": "snap_tiles (OP_GATHER)", "achieved": ach,
                                         "peak": peaks["d2h"], "unit": "GB/s", "frac": ach / peaks["d2h"]},
                            "parity": {"image_equals_oracle": ok_img, "restore_equals_original": ok_rest},
                            "cpu_baseline": cpu, "clocks": clk, "gpu_launches": kern,
                            "timed_steps": args.steps * reps,
                            "e2e": {"value": 2 * B / (ms * 1e-3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": B,
                                    "d2h_bytes_per_step": used}})))


def run_incr20g(args, rank, world, local, pg):
    """20 GiB in 2,000 allocations; incremental checkpoints at 1, 10 and 50 %
    clustered dirty chunks (10 consecutive steps each), for every chunk size
    of the autotuner's sweep (16 KiB - 1 MiB); graph-captured."""
    import torch
    import paper_2502_16631_b300 as snap
    sizes = workloads.config3_sizes(args.seed)
    B = sum(sizes)
    align = 1 << 20
    starts, off = [], 0
    for n in sizes:
        starts.append(off)
        off += (n + align - 1) // align * align
    arena = torch.empty(off, dtype=torch.uint8, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(args.seed)
    step = 1 << 30
    for p in range(0, off, step):
        q = min(off, p + step)
        arena[p:q].copy_(torch.randint(0, 256, (q - p,), dtype=torch.uint8, device="cuda", generator=g))
    views = [arena[s0: s0 + n] for s0, n in zip(starts, sizes)]
    grid = arena.view(-1, UNIT)
    fracs = [0.01, 0.10, 0.50]
    units = {f: torch.from_numpy(dirty_units(sizes, starts, f, args.seed + int(f * 1000))).cuda() for f in fracs}
    # 64 KiB is always swept: the plain form and the copy-form comparison use it
    chunks = sorted({int(x) * KiB for x in args.incr_chunks.split(",")} | {64 * KiB})
    sets = {}
    cap_full = cap_patch = 0
    for C in chunks:
        s = snap.Set(chunk_bytes=C)
        for v in views:
            s.register(v)
        sets[C] = s
        cap_full = max(cap_full, s.image_bytes(snap.FULL))
        cap_patch = max(cap_patch, s.image_bytes(snap.INCREMENTAL))
    full = snap.HostBuffer(cap_full)
    patch = snap.HostBuffer(cap_patch)
    # plain form: one cudaMemcpyAsync per allocation, full copy
    s64 = sets[64 * KiB]
    s64.plain_checkpoint(full)
    plain = []
    for _ in range(3):
        t0 = time.perf_counter()
        s64.plain_checkpoint(full)
        plain.append(time.perf_counter() - t0)
    plain_gbs = B / min(plain) / 1e9
    table, tune, kern = {}, {}, 0
    clocks = ClockSampler(local)
    clocks.start()

    def measure(s, f):
        nonlocal kern
        times, dirty, hashms, copies = [], [], [], []
        for i in range(3 + 10):
            grid[units[f]] ^= 0x5A  # the training step: every byte of each chosen unit changes
            torch.cuda.synchronize()
            a, b = _ev(), _ev()
            a.record()
            used = s.checkpoint(patch, snap.INCREMENTAL)
            b.record()
            torch.cuda.synchronize()
            st = s.stats()
            if i >= 3:
                times.append(a.elapsed_time(b))
                dirty.append(st["dirty_chunks"])
                hashms.append(st["hash_ms"])
                copies.append(st["dma_copies"])
                kern += st["kernel_launches"]
        assert s.verify(patch, used) == 0
        ms = statistics.median(times)
        return {"ms": ms, "effective_gbs": B / (ms * 1e-3) / 1e9, "dirty_chunks": int(statistics.median(dirty)),
                "hash_ms": statistics.median(hashms), "vs_plain_full": (B / (ms * 1e-3) / 1e9) / plain_gbs,
                "dma_copies": int(statistics.median(copies))}

    for C in chunks:
        s = sets[C]
        tune[C] = s.autotune(snap.INCREMENTAL)
        s.checkpoint(full, snap.FULL)
        table[C] = {f: measure(s, f) for f in fracs}
    # both ways of moving the dirty chunks, on the same state at 64 KiB
    # chunks: gather CTAs of the fused launch (SM loads and stores) and the
    # copy engines (one copy per dirty run, every SM but one hashing)
    forms = {}
    for name, mode in (("sm", snap.INCR_COPY_SM), ("dma", snap.INCR_COPY_DMA)):
        s = snap.Set(chunk_bytes=64 * KiB, incr_copy=mode)
        for v in views:
            s.register(v)
        s.autotune(snap.INCREMENTAL)
        s.checkpoint(full, snap.FULL)
        forms[name] = {f: measure(s, f) for f in fracs}
        s.close()
    clk = clocks.stop()
    best = {f: max(chunks, key=lambda C: table[C][f]["effective_gbs"]) for f in fracs}
    v10 = table[best[0.10]][0.10]
    pk = measured_peaks().get("hbm_gbs", 6400.0)
    link = link_peak(torch)["d2h"]
    hash_gbs = max(tune[C]["gbs"] for C in chunks)  # the autotuner's timing of the hash pass alone

    def roof(f):
        # incremental roofline: the slower of reading every state byte from
        # HBM and moving the dirty bytes over the link (both at measured peaks)
        C = best[f]
        t_roof = max(B / (pk * 1e9), table[C][f]["dirty_chunks"] * C / (link * 1e9))
        return {"ms": table[C][f]["ms"], "roofline_ms": t_roof * 1e3, "frac": t_roof * 1e3 / table[C][f]["ms"]}
    out = _line(args, world, v10["effective_gbs"], v10["ms"],
                {"workload": "20 GiB in 2,000 allocations log-uniform [4 KiB, 256 MiB], random bytes; clustered "
                             "dirty runs (mean 16 x 64 KiB)", "dirty_frac": 0.10, "chunk_bytes": best[0.10],
                 "l2": "20 GiB state, larger than L2"},
                {"incremental": {str(C // KiB) + "KiB": {str(int(f * 100)) + "%": table[C][f] for f in fracs}
                                 for C in chunks},
                 "autotuned_chunk": {str(int(f * 100)) + "%": best[f] // KiB for f in fracs},
                 "autotuned_shape": {str(C // KiB) + "KiB": tune[C] for C in chunks},
                 "speedup_vs_plain_full": {str(int(f * 100)) + "%": table[best[f]][f]["vs_plain_full"] for f in fracs},
                 "plain_full_gbs": plain_gbs,
                 "roofline": {"bound": "host_link", "kernel": "fused incremental (hash, diff and metadata in one launch; "
                                                        "dirty runs by the copy engines by default)",
                              "achieved": v10["effective_gbs"], "peak": B / (roof(0.10)["roofline_ms"] * 1e-3) / 1e9,
                              "unit": "GB/s", "frac": roof(0.10)["frac"],
                              "note": "10 % case; roofline = max(state bytes / measured HBM, dirty bytes / "
                                      "measured D2H copy rate)"},
                 "roofline_by_frac": {str(int(f * 100)) + "%": roof(f) for f in fracs},
                 "copy_forms_64KiB": {name: {str(int(f * 100)) + "%": dict(
                     t, roofline_frac=max(B / (pk * 1e9), t["dirty_chunks"] * 64 * KiB / (link * 1e9)) * 1e3 / t["ms"])
                     for f, t in tab.items()} for name, tab in forms.items()},
                 "roofline_hash": {"bound": "hbm", "kernel": "snap_tiles (OP_HASH)", "achieved": hash_gbs,
                                   "peak": pk, "unit": "GB/s", "frac": hash_gbs / pk,
                                   "note": "the autotuner's timing of the hash pass alone, best chunk size"},
                 "gpu_launches": kern, "clocks": clk})
    print(json.dumps(out))


def llama7b_sizes_for_host(spec, world):
    """The Llama-7B state spec, or, when this host cannot hold every rank's
    pageable image, its longest prefix that fits (stated in the line)."""
    sizes = workloads.spec_bytes(spec)
    avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    per_rank = avail // max(1, world) - 24 * GiB  # rings, the CPU sample, the process itself
    if sum(sizes) <= per_rank:
        return spec, None
    keep, tot = [], 0
    for e, n in zip(spec, sizes):
        if tot + n > per_rank:
            break
        keep.append(e)
        tot += n
    return keep, ("host memory (%.0f GiB free for %d rank(s)) holds only the first %d of 1,196 allocations "
                  "(%d B) per rank" % (avail / GiB, world, len(keep), tot))


def run_llama7b(args, rank, world, local, pg):
    """Default step: the Llama-7B-shaped training state (bf16 W, fp32
    master/m/v, 20 GiB bf16 activations; 1,196 allocations, 115,812,655,104 B):
    full checkpoint through the set's 4 GiB pinned ring into a pageable host
    image, then restore of that image into a second, separately allocated set
    of device buffers.  The two buffer sets swap roles every step, so each
    step checkpoints what the previous one restored."""
    import mmap
    import torch
    import oracle
    import paper_2502_16631_b300 as snap
    from struct import unpack_from
    torch.cuda.set_device(local)
    gpt2 = None
    if not args.no_gpt2_extra:
        g2 = measure_gpt2(args, rank, world, local, pg, 10, 3, False)
        gpt2 = {k: g2[k] for k in ("value", "unit", "ms_per_step", "config", "roofline", "roofline_restore",
                                   "roofline_hash", "breakdown", "e2e", "e2e_pageable", "gpu_launches")}
        gpt2["note"] = ("the GPT-2-small step with pinned, device-mapped images, 10 timed steps: full + 10 % "
                        "incremental + verify + restore; breakdown.plain_* is the plain form (one "
                        "cudaMemcpyAsync per allocation, full copy every time): the batched kernel is slower "
                        "than it on full copies (the SM-initiated link ceiling is below the copy engines'), "
                        "and 8-9x faster on the 10 % incremental")
    spec, reduced = llama7b_sizes_for_host(workloads.llama7b_state_spec(), world)
    sizes = workloads.spec_bytes(spec)
    B = sum(sizes)
    nch = [(n + UNIT - 1) // UNIT for n in sizes]
    n_chunks = sum(nch)
    bufs = [[torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes] for _ in range(2)]
    workloads.torch_fill_spec(bufs[0], spec, seed=args.seed + rank)
    for t in bufs[1]:
        t.fill_(0xA5)  # the other set starts with a pattern: the first restore must overwrite it
    sets = []
    for b in bufs:
        s = snap.Set(chunk_bytes=UNIT, ring_bytes=4 * GiB)
        for t in b:
            s.register(t)
        s.prepare(layout=True, ring=True)
        sets.append(s)
    nimg = sets[0].image_bytes(snap.FULL)
    t0 = time.perf_counter()
    m = mmap.mmap(-1, nimg, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS | getattr(mmap, "MAP_POPULATE", 0))
    img = np.frombuffer(m, dtype=np.uint8)
    populate_s = time.perf_counter() - t0
    # sampled chunks of the original state, checked against the last step's
    # image and restored buffers after the timed region
    rng = np.random.default_rng(args.seed)
    c0 = np.concatenate([[0], np.cumsum(nch)])
    picks = sorted(set(int(x) for x in rng.integers(0, c0[-1], 62)) | {0, int(c0[-1] - 1)})
    samples = []
    for c in picks:
        k = int(np.searchsorted(c0, c, side="right") - 1)
        i = c - int(c0[k])
        lo, hi = i * UNIT, min((i + 1) * UNIT, sizes[k])
        samples.append((k, i, lo, hi, bufs[0][k][lo:hi].cpu().numpy().copy()))
    peaks = link_peak(torch)
    per = {"ckpt": [], "rest": [], "gather_kernel": [], "scatter_kernel": []}
    counts = {"kernels": 0, "windows": 0}

    def step(i, record):
        src, dst = sets[i % 2], sets[(i + 1) % 2]
        a, b, c = _ev(), _ev(), _ev()
        a.record()
        used = src.checkpoint(img, snap.FULL)
        stc = src.stats()
        b.record()
        dst.restore(img, used)
        str_ = dst.stats()
        c.record()
        if record:
            c.synchronize()
            per["ckpt"].append(a.elapsed_time(b))
            per["rest"].append(b.elapsed_time(c))
            per["gather_kernel"].append(stc["copy_ms"])
            per["scatter_kernel"].append(str_["copy_ms"])
            counts["kernels"] += int(stc["kernel_launches"]) + int(str_["kernel_launches"])
            counts["windows"] = int(stc["kernel_launches"])
        return used

    warm = max(3, args.warmup)
    first_hashes = None
    for i in range(warm):
        used = step(i, False)
        if i == 0:
            first_hashes = sets[0].committed_hashes(n_chunks)[0].copy()
    clocks = ClockSampler(local)
    barrier(pg)
    torch.cuda.synchronize()
    clocks.start()
    t_start, t_end = _ev(), _ev()
    h0 = time.perf_counter()
    t_start.record()
    for j in range(args.steps):
        used = step(warm + j, True)
    t_end.record()
    torch.cuda.synchronize()
    h1 = time.perf_counter()
    barrier(pg)
    clk = clocks.stop()
    ms = t_start.elapsed_time(t_end) / args.steps
    ms_max = reduce_max(pg, ms)
    host_ms_max = reduce_max(pg, (h1 - h0) * 1e3 / args.steps)
    total_bytes = reduce_sum(pg, 2.0 * B)
    value = total_bytes / (ms_max * 1e-3) / 1e9

    # parity after the timed region: the last image and the buffers it was
    # restored into hold the original state (every step round-tripped it)
    holder = sets[(warm + args.steps) % 2]
    final_hashes, gen = holder.committed_hashes(n_chunks)
    chain_ok = bool(np.array_equal(first_hashes, final_hashes))
    rec, o = [], 64
    for n, k in zip(sizes, nch):
        rec.append(o)
        d = (o + 32 + 4 * k + 4095) // 4096 * 4096
        o = (d + n + 4095) // 4096 * 4096
    hb = bufs[(warm + args.steps) % 2]
    ok_img = ok_hash = ok_dev = True
    for k, i, lo, hi, data in samples:
        d_off = unpack_from("<Q", m, rec[k] + 16)[0]
        ok_img &= bytes(img[d_off + lo: d_off + hi]) == data.tobytes()
        ok_hash &= unpack_from("<I", m, rec[k] + 32 + 4 * i)[0] == oracle.crc32c(data)
        ok_dev &= bool(np.array_equal(hb[k][lo:hi].cpu().numpy(), data))
    mism = holder.verify(img, used)

    gather_ms = statistics.mean(per["gather_kernel"])
    scatter_ms = statistics.mean(per["scatter_kernel"])
    ach_g = B / (gather_ms * 1e-3) / 1e9
    ach_s = B / (scatter_ms * 1e-3) / 1e9
    W = max(1, counts["windows"])
    ratio = traffic_ratio_from_profiles("snap_tiles_gather")
    line = _line(args, world, value, ms_max, llama7b_config(args, B, len(sizes), reduced), {
        "roofline": {"bound": "host_link", "kernel": "snap_tiles (OP_GATHER into ring slots, full checkpoint)",
                     "achieved": ach_g, "peak": peaks["d2h"], "unit": "GB/s", "frac": ach_g / peaks["d2h"],
                     "peak_source": "pinned cudaMemcpyAsync D2H, 1 GiB, best of 5, measured in this run",
                     "launches_per_call": W, "bytes_per_launch": B / W,
                     "traffic": None if ratio is None else ratio * B / W,
                     "traffic_note": "DRAM bytes per launch (one ring window): the committed ncu ratio of DRAM "
                                     "bytes to state bytes of this kernel code x the window's state bytes",
                     "sm_path_peak": peaks["sm_d2h"], "frac_of_sm_path": ach_g / peaks["sm_d2h"],
                     "note": "achieved = state bytes / the summed device time (CUDA events on the library "
                             "stream) of the call's gather launches, one per ring window"},
        "roofline_restore": {"bound": "host_link", "kernel": "snap_tiles (OP_SCATTER from ring slots)",
                             "achieved": ach_s, "peak": peaks["h2d"], "unit": "GB/s", "frac": ach_s / peaks["h2d"],
                             "sm_path_peak": peaks["sm_h2d"], "frac_of_sm_path": ach_s / peaks["sm_h2d"]},
        "breakdown": {
            "checkpoint_gbs": B / (statistics.median(per["ckpt"]) * 1e-3) / 1e9,
            "restore_gbs": B / (statistics.median(per["rest"]) * 1e-3) / 1e9,
            "gather_kernel_ms": gather_ms, "scatter_kernel_ms": scatter_ms,
            "call_ms": {k: {"median": statistics.median(per[k]),
                            "std": statistics.stdev(per[k]) if len(per[k]) > 1 else 0.0} for k in ("ckpt", "rest")},
            "image_bytes": used, "ring_windows_per_call": W},
        "parity": {"sampled_chunks": len(samples), "image_bytes_equal_original": bool(ok_img),
                   "image_hashes_equal_oracle": bool(ok_hash), "restored_bytes_equal_original": bool(ok_dev),
                   "hash_table_unchanged_over_all_steps": chain_ok, "verify_mismatches": mism,
                   "generation": gen},
        "link_peak_gbs": peaks,
        "e2e": {"value": total_bytes / (host_ms_max * 1e-3) / 1e9, "unit": "GB/s",
                # restore: the state bytes read from the image + the hash table uploaded
                "h2d_bytes_per_step": B + 4 * n_chunks,
                # checkpoint: the state bytes written into the image + the hash table read back
                "d2h_bytes_per_step": B + 4 * n_chunks,
                "note": "host wall clock around the same timed steps (Python binding -> C ABI -> ring pipeline "
                        "-> return); the step itself moves the state to and from pageable host memory, so this "
                        "equals value up to the host's call overhead"},
        "image_populate_s": populate_s,
        "memory": {"host_image_bytes": nimg, "host_pinned_ring_bytes": 2 * 4 * GiB,
                   "device_state_bytes": 2 * B,
                   "note": "one pageable image of the whole state; a 4 GiB pinned ring per buffer set; two "
                           "resident buffer sets on the device (the checkpointed one and the restore target)"},
        "gpu_launches": counts["kernels"],
        "clocks": clk,
    })
    if gpt2 is not None:
        line["gpt2_step"] = gpt2
    for st_ in sets:
        st_.close()
    del bufs, hb
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = sample_allocations(spec, args.cpu_sample_bytes, args.seed)
        line["cpu_baseline"] = cpu_baseline(sample, args, kind="llama7b", what="Llama-7B-state")
    if rank == 0:
        print(json.dumps(line))
    del img
    m.close()


def run_serving(args, rank, world, local, pg):
    """32 tenants (8-64 allocations log-uniform [1 MiB, 2 GiB], <= 4 GiB
    each), Poisson arrivals at 20/s of full / incremental (5 % dirty) /
    restore requests, budgets 64 GB pinned and 150 GB HBM; p50/p99 latency
    and GB/s, against serial plain full copies of the same arrivals."""
    import mmap
    import threading
    import torch
    import paper_2502_16631_b300 as snap
    tenants = workloads.config5_tenants(args.seed)
    g = torch.Generator(device="cuda")
    g.manual_seed(args.seed)
    T = []
    for sizes in tenants:
        ts = [torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda", generator=g) for n in sizes]
        s = snap.Set(chunk_bytes=UNIT)
        for t in ts:
            s.register(t)
        nf = s.image_bytes(snap.FULL)
        npb = min(s.image_bytes(snap.INCREMENTAL), nf // 8 + 64 * MiB)  # 5 % dirty fits easily
        flags = mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS | getattr(mmap, "MAP_POPULATE", 0)
        full = np.frombuffer(mmap.mmap(-1, nf, flags=flags), dtype=np.uint8)
        patch = np.frombuffer(mmap.mmap(-1, npb, flags=flags), dtype=np.uint8)
        nunits = sum((n + UNIT - 1) // UNIT for n in sizes)
        rec, o = [], 64  # record offsets of the full image (the image layout)
        for n in sizes:
            nk = (n + UNIT - 1) // UNIT
            rec.append(o)
            o = ((o + 32 + 4 * nk + 4095) // 4096 * 4096 + n + 4095) // 4096 * 4096
        T.append({"set": s, "ts": ts, "full": full, "patch": patch, "bytes": sum(sizes), "units": nunits,
                  "has_image": False, "sizes": sizes, "rec": rec})
    torch.cuda.synchronize()
    def arrivals(rate, n, seed):
        r = workloads.Rng(seed)
        t, reqs = 0.0, []
        legal = [{"full"} for _ in T]
        for i in range(n):
            t += -np.log(1.0 - r.uniform()) / rate
            k = r.randint(0, len(T) - 1)
            kinds = sorted(legal[k])
            kind = kinds[r.randint(0, len(kinds) - 1)]
            reqs.append((t, k, kind))
            legal[k] |= {"incremental", "restore"}
        return reqs

    def mutate(tk, seed):
        """5 % of each allocation's whole 64 KiB units, every byte changed."""
        gg = torch.Generator(device="cuda")
        gg.manual_seed(seed)
        for x in tk["ts"]:
            n = x.numel() // UNIT
            if n == 0:
                continue
            idx = torch.nonzero(torch.rand(n, generator=gg, device="cuda") < 0.05).flatten()
            if idx.numel():
                v = x[: n * UNIT].view(n, UNIT)
                v[idx] ^= 0x5A
        torch.cuda.synchronize()

    # the pinned budget holds the staging pool and, if asked, whole tenants'
    # images pinned for direct access (the others stay pageable)
    pin_left = min(args.serve_pin_gb * 1e9, 64 * 10 ** 9 - args.serve_pool_gib * GiB)
    pinned_tenants = []
    t_pin = time.perf_counter()
    for k, tk in enumerate(T):
        need = tk["full"].nbytes + tk["patch"].nbytes
        if need > pin_left:
            break
        snap.host_register(tk["full"])
        snap.host_register(tk["patch"])
        pinned_tenants.append(k)
        pin_left -= need
    t_pin = time.perf_counter() - t_pin
    from struct import unpack_from

    def sample_request(i, tk, kind, buf, rng):
        """Two chunks of a completed request: the tenant's device bytes (which
        stay as the request left them until the tenant's next request), the
        image's or patch's bytes of that chunk and its stored CRC."""
        out = []
        sizes = tk["sizes"]
        if kind == "incremental":
            off, recs = 64, []
            for n in sizes:  # walk the patch: record, hashes, dirty list, dirty chunks
                nk = (n + UNIT - 1) // UNIT
                dk = unpack_from("<Q", buf, off + 16)[0]
                nd = unpack_from("<I", buf, off + 32 + 4 * nk)[0]
                idx = np.frombuffer(buf, dtype="<u4", count=nd, offset=off + 36 + 4 * nk)
                recs.append((off, dk, idx))
                off = dk + sum((min(UNIT, n - int(c) * UNIT) + 4095) // 4096 * 4096 for c in idx)
            cand = [k for k, (_, _, idx) in enumerate(recs) if idx.size]
            for _ in range(2 if cand else 0):
                k = cand[int(rng.integers(0, len(cand)))]
                off, dk, idx = recs[k]
                j = int(rng.integers(0, idx.size))
                c = int(idx[j])
                pos = dk + sum((min(UNIT, sizes[k] - int(x) * UNIT) + 4095) // 4096 * 4096 for x in idx[:j])
                lo, hi = c * UNIT, min((c + 1) * UNIT, sizes[k])
                out.append((i, tk["ts"][k][lo:hi].cpu().numpy(), buf[pos: pos + hi - lo].copy(),
                            unpack_from("<I", buf, off + 32 + 4 * c)[0]))
            return out
        img = tk["full"]
        for _ in range(2):
            k = int(rng.integers(0, len(sizes)))
            nk = (sizes[k] + UNIT - 1) // UNIT
            if nk == 0:
                continue
            c = int(rng.integers(0, nk))
            lo, hi = c * UNIT, min((c + 1) * UNIT, sizes[k])
            d_off = unpack_from("<Q", img, tk["rec"][k] + 16)[0]
            out.append((i, tk["ts"][k][lo:hi].cpu().numpy(), img[d_off + lo: d_off + hi].copy(),
                        unpack_from("<I", img, tk["rec"][k] + 32 + 4 * c)[0]))
        return out

    def simulate(reqs, tag):
        """Run the arrivals `reqs` against a fresh server; per-request
        latency (arrival to completion), status, bytes, and sampled chunks."""
        sv = snap.Server(pinned_budget=64 * 10 ** 9, hbm_budget=150 * 10 ** 9, chunk_bytes=UNIT,
                         ring_bytes=args.serve_pool_gib * GiB)
        lat = [None] * len(reqs)
        moved = [0] * len(reqs)
        link = [0] * len(reqs)  # bytes over the host link: image or patch written, or image restored
        status = [0] * len(reqs)
        samples = []  # (request, device bytes, image bytes, stored CRC): checked after the run
        per_tenant = [[] for _ in T]
        for i, (ta, k, kind) in enumerate(reqs):
            per_tenant[k].append(i)
        start = time.perf_counter() + 0.5
        lock = threading.Lock()

        def tenant_loop(k):
            tk = T[k]
            torch.cuda.set_device(local)
            for i in per_tenant[k]:
                ta, _, kind = reqs[i]
                # the tenant's own work between its requests (before the arrival)
                if kind == "incremental":
                    mutate(tk, 7 * i + 1 + tag)
                    rk, buf = snap.REQ_INCREMENTAL, tk["patch"]
                elif kind == "restore":
                    for x in tk["ts"]:
                        x.fill_(0x33)  # scribble: the restore must bring the image back
                    torch.cuda.synchronize()
                    rk, buf = snap.REQ_RESTORE, tk["full"]
                else:
                    rk, buf = snap.REQ_FULL, tk["full"]
                delay = start + ta - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                ticket = sv.submit(tk["set"], rk, buf)
                rc, st_, stats = sv.wait(ticket, 600000)
                done = time.perf_counter()
                with lock:
                    lat[i] = (done - (start + ta)) * 1e3
                    status[i] = st_
                    moved[i] = tk["bytes"]
                    link[i] = int(stats["image_bytes"]) if kind == "incremental" else tk["bytes"]
                if st_ == 0:
                    got = sample_request(i, tk, kind, buf, np.random.default_rng(i + tag))
                    with lock:
                        samples.extend(got)

        th = [threading.Thread(target=tenant_loop, args=(k,)) for k in range(len(T))]
        t0 = time.perf_counter()
        for x in th:
            x.start()
        for x in th:
            x.join()
        wall = time.perf_counter() - max(t0, start)
        sv.close()
        good = [l for l, s_ in zip(lat, status) if s_ == 0 and l is not None]
        return {"lat": lat, "status": status, "good": good, "wall": wall, "samples": samples,
                "gbs": sum(m_ for m_, s_ in zip(moved, status) if s_ == 0) / wall / 1e9,
                "link_gbs": sum(b_ for b_, s_ in zip(link, status) if s_ == 0) / wall / 1e9,
                "offered_gbs": (sum(T[k]["bytes"] for _, k, kind in reqs if kind != "incremental")
                                + sum(0.05 * T[k]["bytes"] for _, k, kind in reqs if kind == "incremental"))
                               / reqs[-1][0] / 1e9}

    reqs = arrivals(args.rate, args.arrivals, args.seed ^ 0xA77)
    main = simulate(reqs, 0)
    lower = []
    for rate in [float(x) for x in args.serve_lower_rates.split(",") if x.strip()]:
        n_low = max(1, int(round(args.arrivals * rate / args.rate / 2)))  # half the span of the main run
        low = simulate(arrivals(rate, n_low, (args.seed ^ 0xA77) + int(rate * 100)), 1 << 20)
        lower.append({"rate": rate, "arrivals": n_low, "p50": float(np.percentile(low["good"], 50)),
                      "p99": float(np.percentile(low["good"], 99)), "completed": len(low["good"]),
                      "gbs": low["gbs"], "link_gbs": low["link_gbs"], "offered_link_gbs": low["offered_gbs"]})
        main["samples"].extend(low["samples"])
    lat, status, good, wall, samples = main["lat"], main["status"], main["good"], main["wall"], main["samples"]
    gbs, link_gbs, offered_gbs = main["gbs"], main["link_gbs"], main["offered_gbs"]
    # after the runs: the sampled chunks against the oracle's CRC-32C and the
    # device bytes
    import oracle
    bad = [i for i, d, im, h in samples if not (np.array_equal(d, im) and oracle.crc32c(d) == h)]
    parity = {"requests_sampled": len(set(i for i, _, _, _ in samples)), "chunks_checked": len(samples),
              "mismatches": len(bad),
              "check": "per completed request (every run), two chunks: the tenant's device bytes == the image's "
                       "(or the patch's dirty-chunk) bytes, and the oracle's CRC-32C of them == the stored hash"}
    both = link_peak_both(torch)
    workers = int(os.environ.get("SNAP_WORKERS", "0")) or min(40, max(2, ((os.cpu_count() or 2) * 5 + 3) // 4))
    # (the server's copy workers: 5 per 4 host threads unless SNAP_WORKERS says otherwise).  The copy
    # ceiling is probed with one thread per host CPU: the probe times its slowest thread, and more threads
    # than CPUs make that a preempted thread's time, not the memory's
    probe_threads = max(2, min(workers, os.cpu_count() or 2))
    hc = snap.host_copy_ceiling(probe_threads, 2, 2 * GiB, 3)
    hc_link = snap.host_copy_ceiling(probe_threads, 2, 2 * GiB, 3, with_link=True)
    # a staged byte costs host DRAM a read and a write for the copy plus one
    # access for the link transfer; the copy probe moves 2 DRAM bytes per byte
    host_bound = 2.0 * hc / 3.0
    peak = min(both["sm_both"], host_bound)
    # serial plain full copies of the same arrivals (FIFO single server; each
    # request's service time measured by running it, start = max(arrival,
    # previous end)); the first 240 arrivals
    nb = 0 if args.no_plain else min(len(reqs), 240)
    end, plain_lat = 0.0, []
    for i in range(nb):
        ta, k, kind = reqs[i]
        tk = T[k]
        t1 = time.perf_counter()
        if kind == "restore":
            tk["set"].plain_restore(tk["full"])
        else:
            tk["set"].plain_checkpoint(tk["full"])
        svc = time.perf_counter() - t1
        begin = max(ta, end)
        end = begin + svc
        plain_lat.append((end - ta) * 1e3)
    for k in pinned_tenants:
        snap.host_unregister(T[k]["full"])
        snap.host_unregister(T[k]["patch"])
    ours_prefix = sorted(lat[:nb])
    out = _line(args, world, gbs, wall * 1e3 / len(reqs),
                {"workload": "serving: 32 tenants (8-64 allocations log-uniform [1 MiB, 2 GiB], <= 4 GiB each, "
                             "%.1f GiB total), Poisson %.0f req/s, %d arrivals, full/incremental(5%%)/restore"
                             % (sum(tk["bytes"] for tk in T) / GiB, args.rate, len(reqs)),
                 "budgets": {"pinned": "64 GB", "hbm": "150 GB"}, "image": "pageable host memory"},
                {"parity": parity,
                 "latency_ms": {"p50": float(np.percentile(good, 50)), "p99": float(np.percentile(good, 99)),
                                "max": float(max(good)), "completed": len(good), "failed": len(reqs) - len(good)},
                 "latency_at_lower_rates": lower,
                 "plain_serial_first_%d" % nb: ({"p50": float(np.percentile(plain_lat, 50)),
                                                 "p99": float(np.percentile(plain_lat, 99)),
                                                 "ours_p50": float(np.percentile(ours_prefix, 50)),
                                                 "ours_p99": float(np.percentile(ours_prefix, 99))} if nb else None),
                 "roofline": {"bound": "host_memory" if host_bound < both["sm_both"] else "host_link (both directions)",
                              "kernel": "serving rounds (mixed gather + scatter launches) + host copies",
                              "achieved": link_gbs, "peak": peak, "unit": "GB/s", "frac": link_gbs / peak,
                              "link_peak_both": both["sm_both"], "ce_both": both["ce_both"],
                              "host_copy_gbs": hc, "host_copy_gbs_under_link_load": hc_link,
                              "host_memory_bound": host_bound, "copy_workers": workers,
                              "probe_threads": probe_threads, "offered": offered_gbs,
                              "note": "achieved = image, patch and restore bytes over the link / wall time; peak = "
                                      "min(SM loads/stores in both directions at once (snap_link_ceiling 2), "
                                      "2/3 x the workers' pinned<->pageable copy rate (snap_host_copy_ceiling 2): "
                                      "every staged byte is one host copy (a DRAM read and write) plus one link "
                                      "transfer (a DRAM access)); offered = the arrivals' link bytes / arrival "
                                      "span (patches at 5 %)"},
                 "staging_pool_gib": args.serve_pool_gib,
                 "pinned_tenants": {"count": len(pinned_tenants),
                                    "gb": sum(T[k]["full"].nbytes + T[k]["patch"].nbytes for k in pinned_tenants) / 1e9,
                                    "register_s": t_pin,
                                    "note": "these tenants' images are registered and read/written directly; the "
                                            "rest are pageable and staged through the pool"},
                 "kinds": {k_: sum(1 for _, _, kk in reqs if kk == k_) for k_ in ("full", "incremental", "restore")}})
    print(json.dumps(out))


def run_async(args, rank, world, local, pg):
    """GPT-2-small training state (593 allocations, 2,259,472,384 B) under a
    training-like load on the caller's stream (bf16 8192^3 matmuls).  Each
    step times, from the caller's side (host clock, device synchronised at
    both ends):
      load   n matmuls alone,
      sync   snap_checkpoint, then the n matmuls,
      async  snap_checkpoint_async, the n matmuls, snap_checkpoint_wait.
    The checkpoint's cost to the caller is (sync or async) - load; `value`
    is state bytes per second of that cost for the asynchronous call."""
    import torch
    import oracle
    import paper_2502_16631_b300 as snap
    from struct import unpack_from
    spec = workloads.gpt2_state_spec()
    sizes = workloads.spec_bytes(spec)
    B = sum(sizes)
    ts = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
    workloads.torch_fill_spec(ts, spec, seed=args.seed)
    s = snap.Set(chunk_bytes=UNIT)
    for t in ts:
        s.register(t)
    s.prepare(layout=True, shadow=True)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    # parity at full size: chunks sampled before the cut are overwritten as
    # soon as the call returns; the image must hold the values at the cut
    rng = np.random.default_rng(args.seed)
    nch = [(n + UNIT - 1) // UNIT for n in sizes]
    c0 = np.concatenate([[0], np.cumsum(nch)])
    picks = sorted(set(int(x) for x in rng.integers(0, c0[-1], 64)) | {int(c0[-1] - 1)})
    samples = []
    for c in picks:
        k = int(np.searchsorted(c0, c, side="right") - 1)
        lo, hi = (c - int(c0[k])) * UNIT, min((c - int(c0[k]) + 1) * UNIT, sizes[k])
        samples.append((k, c - int(c0[k]), lo, hi, ts[k][lo:hi].cpu().numpy().copy()))
    torch.cuda.synchronize()
    s.checkpoint_async(img, snap.FULL)
    for k, i, lo, hi, _ in samples:
        ts[k][lo:hi] ^= 0xFF
    used = s.checkpoint_wait()
    ok, off, rec = True, 64, []
    for n in sizes:
        _, _, dk, _ = unpack_from("<QQQQ", img.array, off)
        rec.append((off, dk))
        off = (dk + n + 4095) // 4096 * 4096
    for k, i, lo, hi, data in samples:
        roff, dk = rec[k]
        ok &= bytes(img.array[dk + lo: dk + hi]) == data.tobytes()
        ok &= unpack_from("<I", img.array, roff + 32 + 4 * i)[0] == oracle.crc32c(data)
        ok &= not np.array_equal(ts[k][lo:hi].cpu().numpy(), data)
    for k, i, lo, hi, _ in samples:
        ts[k][lo:hi] ^= 0xFF
    torch.cuda.synchronize()

    a = torch.randn(8192, 8192, dtype=torch.bfloat16, device="cuda")
    b = torch.randn(8192, 8192, dtype=torch.bfloat16, device="cuda")
    c = torch.empty(8192, 8192, dtype=torch.bfloat16, device="cuda")

    def load(n):
        for _ in range(n):
            torch.matmul(a, b, out=c)

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3

    load(20)
    gemm_ms = timed(lambda: load(50)) / 50
    med = statistics.median

    def background_ms(sx):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sx.checkpoint_async(img, snap.FULL)
        sx.checkpoint_wait()
        return (time.perf_counter() - t0) * 1e3

    sets = {}
    for ctas in [int(x) for x in args.async_ctas.split(",")]:
        sx = s if ctas == 0 else snap.Set(chunk_bytes=UNIT, async_ctas=ctas)
        if ctas:
            for t in ts:
                sx.register(t)
            sx.prepare(layout=True, shadow=True)
        sets[ctas] = (sx, med([background_ms(sx) for _ in range(3)]))
    bg = max(v[1] for v in sets.values())
    n = args.load_gemms or max(10, int(2 * (bg + 10) / gemm_ms))

    def sync_step():
        s.checkpoint(img, snap.FULL)
        load(n)

    def async_step(sx):
        sx.checkpoint_async(img, snap.FULL)
        load(n)
        torch.cuda.current_stream().synchronize()
        sx.checkpoint_wait()

    for _ in range(max(3, args.warmup)):
        timed(sync_step)
    peaks = measured_peaks()
    L, S, sync_ms, kern = [], [], [], 0
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.steps):
        L.append(timed(lambda: load(n)))
        S.append(timed(sync_step))
        sync_ms.append(s.stats()["frozen_ms"])
        kern += s.stats()["kernel_launches"]
    sweep = {}
    for ctas, (sx, bgx) in sets.items():
        for _ in range(max(3, args.warmup)):
            timed(lambda: async_step(sx))
        A, fz, q, cut = [], [], [], []
        for _ in range(args.steps):
            A.append(timed(lambda: async_step(sx)))
            st = sx.stats()
            fz.append(st["frozen_ms"])
            q.append(st["quiesce_ms"])
            cut.append(st["frozen_ms"] - st["quiesce_ms"])
            kern += st["kernel_launches"]
        sweep[ctas] = {"frozen_ms": med(fz), "quiesce_ms": med(q), "cut_ms": med(cut), "background_ms_alone": bgx,
                       "async_step_ms": med(A), "caller_cost_ms": max(1e-3, med(A) - med(L))}
        if ctas:
            sx.close()
    # incremental checkpoints after a 10 % clustered mutation: how long the
    # caller is held, synchronous call against asynchronous cut
    nchk = [(n + UNIT - 1) // UNIT for n in sizes]
    c0s = np.concatenate([[0], np.cumsum(nchk)])
    patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
    s.checkpoint(img, snap.FULL)  # the base

    def mutate(seed):
        for u in workloads.mutation_units(int(c0s[-1]), args.dirty, seed):
            k = int(np.searchsorted(c0s, u, side="right") - 1)
            lo = int(u - c0s[k]) * UNIT
            ts[k][lo: min(lo + UNIT, sizes[k])].bitwise_not_()
        torch.cuda.synchronize()

    inc_sync, inc_frozen, inc_total = [], [], []
    for i in range(max(3, args.warmup) + args.steps):
        mutate(1000 + 2 * i)
        s.checkpoint(patch, snap.INCREMENTAL)
        t_sync = s.stats()["total_ms"]
        mutate(1001 + 2 * i)
        s.checkpoint_async(patch, snap.INCREMENTAL)
        s.checkpoint_wait()
        st = s.stats()
        if i >= max(3, args.warmup):
            inc_sync.append(t_sync)
            inc_frozen.append(st["frozen_ms"])
            inc_total.append(st["total_ms"])
            kern += st["kernel_launches"]
    clk = clocks.stop()
    d = sweep[0] if 0 in sweep else next(iter(sweep.values()))
    over_sync = max(1e-3, med(S) - med(L))
    cut_gbs = 2 * B / (d["cut_ms"] * 1e-3) / 1e9  # read + write of every state byte
    value = B / (d["caller_cost_ms"] * 1e-3) / 1e9
    line = _line(args, world, value, d["async_step_ms"],
                 {"workload": "GPT-2-small training state, 593 allocations, 2,259,472,384 B, 64 KiB chunks, "
                              "under %d bf16 8192^3 matmuls on the caller's stream" % n,
                  "step": "load alone; sync checkpoint + load; async checkpoint + load + wait",
                  "l2": "2.26 GB state, larger than L2"},
                 {"async": {"default_ctas": 8,
                            "by_ctas": {str(k): v for k, v in sweep.items()},
                            "sync_checkpoint_ms": med(sync_ms), "load_ms": med(L), "sync_step_ms": med(S),
                            "incremental_10pct": {"sync_call_ms": med(inc_sync), "async_frozen_ms": med(inc_frozen),
                                                  "async_cut_to_commit_ms": med(inc_total)},
                            "caller_cost_sync_ms": over_sync, "sync_equivalent_gbs": B / (over_sync * 1e-3) / 1e9,
                            "matmul_ms": gemm_ms},
                  "roofline": {"bound": "hbm", "kernel": "k_shadow_copy (the cut)", "achieved": cut_gbs,
                               "peak": peaks.get("hbm_gbs", 6400.0), "unit": "GB/s",
                               "frac": cut_gbs / peaks.get("hbm_gbs", 6400.0),
                               "note": "host-observed cut time (launch + event poll included), of measured"},
                  "parity": {"sampled_chunks": len(samples), "image_holds_state_at_cut": bool(ok)},
                  "clocks": clk, "gpu_launches": kern,
                  "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": used}})
    line["metric"] = "async checkpoint: state bytes per second of caller time lost"
    print(json.dumps(line))


def run_lazy(args, rank, world, local, pg):
    """GPT-2-small training state (593 allocations, 2,259,472,384 B).  A
    restored trainer needs its fp32 weights (148 allocations, 497,759,232 B)
    before its first forward pass; the optimizer state and gradients later.
    Each step restores the same image twice, into zeroed buffers:
      sync        snap_restore, then the caller's stream may run;
      prioritised snap_restore_async(weights first) + snap_restore_ready for
                  every weight on the caller's stream, snap_restore_wait.
    Timed on the caller's stream with CUDA events from just before the call
    to the point where the weights are usable, and to full completion."""
    import torch
    import oracle
    import paper_2502_16631_b300 as snap
    spec = workloads.gpt2_state_spec()
    sizes = workloads.spec_bytes(spec)
    B = sum(sizes)
    weights = [k for k, e in enumerate(spec) if e[0].startswith("w.")]
    WB = sum(sizes[k] for k in weights)
    ts = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
    workloads.torch_fill_spec(ts, spec, seed=args.seed)
    s = snap.Set(chunk_bytes=UNIT)
    for t in ts:
        s.register(t)
    s.prepare(layout=True)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    used = s.checkpoint(img, snap.FULL)
    # parity at full size: sampled chunks of the image against their bytes
    rng = np.random.default_rng(args.seed)
    samples = []
    for k in sorted(set(rng.integers(0, len(sizes), 40).tolist()) | set(weights[:4])):
        lo = int(rng.integers(0, max(1, sizes[k] // UNIT))) * UNIT
        hi = min(lo + UNIT, sizes[k])
        samples.append((k, lo, hi, ts[k][lo:hi].cpu().numpy().copy()))
    st = torch.cuda.Stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def zero():
        for t in ts:
            t.zero_()
        torch.cuda.synchronize()

    def sync_restore():
        zero()
        a, b = ev(), ev()
        a.record(st)
        s.restore(img, used)
        b.record(st)
        torch.cuda.synchronize()
        x = a.elapsed_time(b)
        return x, x, s.stats()["kernel_launches"]

    def prio_restore():
        zero()
        a, r, b = ev(), ev(), ev()
        a.record(st)
        s.restore_async(img, weights)
        for k in weights:
            s.restore_ready(k, st)
        r.record(st)
        s.restore_wait()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(r), a.elapsed_time(b), s.stats()["kernel_launches"]

    for _ in range(max(3, args.warmup)):
        sync_restore()
        prio_restore()
    # weights checked right at their readiness point, and the whole state after
    zero()
    s.restore_async(img, weights)
    with torch.cuda.stream(st):
        for k in weights:
            s.restore_ready(k, st)
        early = {k: ts[k][lo:hi].clone() for k, lo, hi, _ in samples if k in weights}
    s.restore_wait()
    torch.cuda.synchronize()
    ok = all(np.array_equal(early[k].cpu().numpy(), d) for k, lo, hi, d in samples if k in early)
    ok &= all(np.array_equal(ts[k][lo:hi].cpu().numpy(), d) for k, lo, hi, d in samples)
    mism = s.verify(img, used)
    peaks = link_peak(torch)
    clocks = ClockSampler(local)
    clocks.start()
    S, P, kern = [], [], 0
    for _ in range(args.steps):
        x = sync_restore()
        S.append(x)
        y = prio_restore()
        P.append(y)
        kern += x[2] + y[2]
    clk = clocks.stop()
    med = statistics.median
    w_sync, all_sync = med([x[0] for x in S]), med([x[1] for x in S])
    w_prio, all_prio = med([x[0] for x in P]), med([x[1] for x in P])
    rest_gbs = B / (all_prio * 1e-3) / 1e9
    line = _line(args, world, w_prio, w_prio,
                 {"workload": "GPT-2-small training state, 593 allocations, 2,259,472,384 B, 64 KiB chunks; "
                              "fp32 weights (148 allocations, %d B) first" % WB,
                  "step": "sync restore; prioritised restore (weights first) with stream readiness",
                  "l2": "2.26 GB state, larger than L2"},
                 {"lazy": {"weights_ready_ms": w_prio, "weights_ready_ms_sync": w_sync,
                           "speedup_to_weights": w_sync / w_prio, "complete_ms": all_prio,
                           "complete_ms_sync": all_sync, "weights_gbs": WB / (w_prio * 1e-3) / 1e9},
                  "roofline": {"bound": "host_link", "kernel": "snap_tiles (OP_SCATTER, waves)", "achieved": rest_gbs,
                               "peak": peaks["h2d"], "unit": "GB/s", "frac": rest_gbs / peaks["h2d"]},
                  "parity": {"sampled_chunks": len(samples), "bytes_equal_at_readiness_and_end": bool(ok),
                             "verify_mismatches": mism},
                  "clocks": clk, "gpu_launches": kern,
                  "e2e": {"value": w_prio, "unit": "ms", "h2d_bytes_per_step": 2 * B, "d2h_bytes_per_step": 0}})
    line["metric"] = "prioritised restore: ms until the weights are usable"
    line["unit"] = "ms"
    line["higher_is_better"] = False
    print(json.dumps(line))


def run_file(args, rank, world, local, pg):
    """GPT-2-small training state (593 allocations, 2,259,472,384 B) persisted
    to an image file.  Per step:
      overlapped   snap_checkpoint_file: windows written while the GPU
                   gathers the next ones (page cache; and with fsync);
      sequential   snap_checkpoint into pinned memory, then one write of the
                   image to a file (the paper's order: device copy, then the
                   memory write), same fsync rule;
      restore      snap_restore_file (file in the page cache).
      incremental  snap_checkpoint_file(INCREMENTAL) after a 10 % clustered
                   mutation (the patch alone is written), with fsync.
    `value` = state bytes / overlapped checkpoint time (with fsync); the
    roofline peak is the storage itself: 2 GiB written with pwrite by 1 or 8
    threads (the better), then fsync, measured in the same run."""
    import shutil
    import threading
    import torch
    import oracle
    import paper_2502_16631_b300 as snap
    spec = workloads.gpt2_state_spec()
    sizes = workloads.spec_bytes(spec)
    B = sum(sizes)
    d = args.file_dir or tempfile.gettempdir()
    free = shutil.disk_usage(d).free
    if free < 3 * B:
        print(json.dumps({"metric": "checkpoint to file GB/s", "unavailable":
                          "%s has %d free bytes, needs %d" % (d, free, 3 * B)}))
        return
    ts = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
    workloads.torch_fill_spec(ts, spec, seed=args.seed)
    s = snap.Set(chunk_bytes=UNIT)
    for t in ts:
        s.register(t)
    s.prepare(layout=True, ring=True)
    img = snap.HostBuffer(s.image_bytes(snap.FULL))
    path = os.path.join(d, "snap_bench_%d.img" % os.getpid())
    seq_path = path + ".seq"
    # parity at full size: the file equals the in-memory image; sampled
    # chunks equal the device bytes; restore from the file verifies clean
    used = s.checkpoint_file(path, snap.FULL)
    s.checkpoint(img, snap.FULL)
    fimg = np.fromfile(path, dtype=np.uint8)
    same_header_free = bool(np.array_equal(fimg[64:], img.view(used)[64:]))
    del fimg
    rng = np.random.default_rng(args.seed)
    samples = []
    for k in sorted(set(rng.integers(0, len(sizes), 32).tolist())):
        lo = int(rng.integers(0, max(1, sizes[k] // UNIT))) * UNIT
        samples.append((k, lo, min(lo + UNIT, sizes[k])))

    def seq(sync):
        s.checkpoint(img, snap.FULL)
        with open(seq_path, "wb") as f:
            f.write(memoryview(img.array))
            if sync:
                f.flush()
                os.fsync(f.fileno())

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    def storage_peak(nbytes=2 * GiB, threads=8):
        buf = np.frombuffer(np.random.default_rng(0).bytes(64 * MiB), dtype=np.uint8)
        fd = os.open(seq_path, os.O_CREAT | os.O_TRUNC | os.O_WRONLY, 0o644)
        per = nbytes // threads

        def worker(i):
            off = i * per
            while off < (i + 1) * per:
                off += os.pwrite(fd, buf, off)

        t0 = time.perf_counter()
        th = [threading.Thread(target=worker, args=(i,)) for i in range(threads)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        os.fsync(fd)
        dt = time.perf_counter() - t0
        os.close(fd)
        return nbytes / dt / 1e9

    starts = np.concatenate([[0], np.cumsum(sizes)])
    units = workloads.mutation_units(int(starts[-1] // UNIT), args.dirty, args.seed)

    def mutate():
        flat = [(int(np.searchsorted(starts, u * UNIT, side="right") - 1), u) for u in units]
        for k, u in flat:
            lo = u * UNIT - int(starts[k])
            if 0 <= lo < sizes[k]:
                ts[k][lo: min(lo + UNIT, sizes[k])].bitwise_not_()

    def incr():
        mutate()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u = s.checkpoint_file(path + ".patch", snap.INCREMENTAL, sync=True)
        return time.perf_counter() - t0, u

    for _ in range(max(3, args.warmup)):
        s.checkpoint_file(path, snap.FULL)
        seq(False)
    clocks = ClockSampler(local)
    clocks.start()
    O, OS, Q, QS, R, kern = [], [], [], [], [], 0
    for _ in range(args.steps):
        O.append(timed(lambda: s.checkpoint_file(path, snap.FULL)))
        kern += s.stats()["kernel_launches"]
        OS.append(timed(lambda: s.checkpoint_file(path, snap.FULL, sync=True)))
        kern += s.stats()["kernel_launches"]
        Q.append(timed(lambda: seq(False)))
        QS.append(timed(lambda: seq(True)))
        R.append(timed(lambda: s.restore_file(path)))
        kern += s.stats()["kernel_launches"]
    host = {k: ts[k][lo:hi].cpu().numpy() for k, lo, hi in samples}  # the state the file at `path` holds
    I = [incr() for _ in range(args.steps)]
    clk = clocks.stop()
    speak = max(storage_peak(threads=1), storage_peak(threads=8))
    for t in ts:
        t.zero_()
    s.restore_file(path)
    ok = same_header_free and all(np.array_equal(ts[k][lo:hi].cpu().numpy(), host[k]) for k, lo, hi in samples)
    mism = s.verify(img, used)
    med = statistics.median
    g = lambda x: B / med(x) / 1e9  # noqa: E731
    peaks = link_peak(torch)
    line = _line(args, world, g(OS), med(OS) * 1e3,
                 {"workload": "GPT-2-small training state, 593 allocations, 2,259,472,384 B, 64 KiB chunks, "
                              "image file on %s" % d,
                  "step": "overlapped checkpoint to file (with and without fsync), sequential checkpoint then "
                          "write, restore from file",
                  "l2": "2.26 GB state, larger than L2"},
                 {"file": {"overlapped_gbs": g(O), "overlapped_fsync_gbs": g(OS), "sequential_gbs": g(Q),
                           "sequential_fsync_gbs": g(QS), "restore_gbs": g(R),
                           "overlap_speedup": med(Q) / med(O), "overlap_speedup_fsync": med(QS) / med(OS),
                           "incremental_10pct_fsync_gbs": B / med([x[0] for x in I]) / 1e9,
                           "incremental_patch_bytes": med([x[1] for x in I]),
                           "storage_write_peak_gbs": speak, "d2h_link_gbs": peaks["d2h"]},
                  "roofline": {"bound": "storage", "kernel": "ring checkpoint to file (gather + pwrite + fsync)",
                               "achieved": g(OS), "peak": speak, "unit": "GB/s", "frac": g(OS) / speak,
                               "note": "peak = best of 1- and 8-thread pwrite + fsync of 2 GiB to the same "
                                       "directory, this run"},
                  "parity": {"file_equals_memory_image": same_header_free, "sampled_chunks": len(samples),
                             "restore_bytes_equal": bool(ok), "verify_mismatches": mism},
                  "clocks": clk, "gpu_launches": kern,
                  "e2e": {"value": g(OS), "unit": "GB/s", "h2d_bytes_per_step": B, "d2h_bytes_per_step": 2 * used}})
    line["metric"] = "checkpoint to an image file (fsync), GB/s of state"
    for p in (path, seq_path, path + ".patch"):
        try:
            os.unlink(p)
        except OSError:
            pass
    print(json.dumps(line))


def run_hash(args, rank, world, local, pg):
    """The chunk hasher alone (snap_hash_chunks): CRC-32C of every 64 KiB
    chunk of an 8 GiB device buffer of random bytes, timed with CUDA events
    on the launching stream, inputs 64x the L2.  Parity: 256 sampled chunks
    against the oracle, and the last (ragged) chunk of a 8 GiB - 4,097 B
    prefix."""
    import torch
    import oracle
    import paper_2502_16631_b300 as snap
    n = 8 * GiB
    x = torch.empty(n, dtype=torch.uint8, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(args.seed)
    for p in range(0, n, GiB):
        x[p: p + GiB].copy_(torch.randint(0, 256, (GiB,), dtype=torch.uint8, device="cuda", generator=g))
    nch = n // UNIT
    out = torch.empty(nch, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        snap.hash_chunks(x, UNIT, out, stream=st)
    clocks = ClockSampler(local)
    clocks.start()
    times = []
    t_end = time.perf_counter() + 1.0  # at least a second, so the clock sampler sees the load
    while len(times) < args.steps or time.perf_counter() < t_end:
        a, b = _ev(), _ev()
        a.record(st)
        snap.hash_chunks(x, UNIT, out, stream=st)
        b.record(st)
        b.synchronize()
        times.append(a.elapsed_time(b))
    clk = clocks.stop()
    got = out.cpu().numpy().view(np.uint32)
    rng = np.random.default_rng(args.seed)
    picks = sorted(set(rng.integers(0, nch, 256).tolist()) | {0, nch - 1})
    ok = all(int(got[c]) == oracle.crc32c(x[c * UNIT: (c + 1) * UNIT].cpu().numpy()) for c in picks)
    m = n - 4097
    tail = torch.empty((m + UNIT - 1) // UNIT, dtype=torch.int32, device="cuda")
    snap.hash_chunks(x, UNIT, tail, nbytes=m, stream=st)
    torch.cuda.synchronize()
    last = (m - 1) // UNIT
    ok &= int(tail[last].cpu().numpy().view(np.uint32)) == oracle.crc32c(x[last * UNIT: m].cpu().numpy())
    pk = measured_peaks().get("hbm_gbs", 6400.0)
    best, med = min(times), statistics.median(times)
    gbs = n / (med * 1e-3) / 1e9
    line = _line(args, world, gbs, med,
                 {"workload": "8 GiB device buffer of random bytes, 131,072 chunks of 64 KiB",
                  "step": "snap_hash_chunks over the whole buffer", "l2": "8 GiB, 64x the L2: no flush"},
                 {"roofline": {"bound": "hbm", "kernel": "snap_tiles (OP_HASH)", "achieved": gbs, "peak": pk,
                               "unit": "GB/s", "frac": gbs / pk, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of "
                               "measured)", "best_gbs": n / (best * 1e-3) / 1e9},
                  "parity": {"sampled_chunks": len(picks) + 1, "hashes_equal_oracle": bool(ok)},
                  "clocks": clk, "gpu_launches": len(times), "timed_launches": len(times),
                  "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    line["metric"] = "chunk hasher GB/s (CRC-32C per 64 KiB chunk)"
    print(json.dumps(line))


def _first_n(sizes, cap):
    tot, n = 0, 0
    for x in sizes:
        if tot >= cap:
            break
        tot += x
        n += 1
    return n


def main():
    args = parse()
    rank, world, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "gpt2":
        run_snap(args, rank, world, local, pg)
    else:
        {"random64m": run_random64m, "incr20g": run_incr20g, "llama7b": run_llama7b,
         "serving": run_serving, "async": run_async, "lazy": run_lazy,
         "file": run_file, "hash": run_hash}[args.workload](args, rank, world, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
