#!/usr/bin/env python
"""Benchmark of the snapshot/restore hot path on B300.

One step = one pass of the whole single-set hot path over the GPT-2-small
training state (593 allocations, 2,259,472,384 B; 64 KiB chunks):

  1. full checkpoint  (quiesce, CRC-32C of every chunk fused with the TMA
                       gather into the pinned, mapped host image)
  2. mutation         (the "training step": XOR 10% of the chunks, clustered
                       runs with mean length 16, with nonzero random bytes)
  3. incremental      (hash every chunk, diff against the committed table,
                       ordered compaction, gather dirty chunks into a patch)
  4. verify           (re-hash the device state against the patch's hashes)
  5. restore          (scatter the full image back; the state is again the
                       step's starting state)

`value` = device-state bytes covered by the four snapshot calls per second
(4 x state bytes / step time), timed with CUDA events around the step; the
per-call rates are reported beside it.  `--impl reference` runs the CPU
oracle (the same step on a bounded sample of the same state) instead.
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
    return out


def traffic_from_profiles(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, valid
    only while the kernel source is unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = os.path.join(ROOT, "paper_2502_16631_b300", "csrc", "kernels.cu")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for line in open(path):
            parts = line.split()
            if len(parts) >= 4 and parts[0] == kernel and parts[3] == sha:
                return int(parts[2])
    except OSError:
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


def cpu_baseline(sample, args, seconds_target=15.0):
    import oracle
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    step, nb = oracle_step_sample(sample, args.dirty, args.seed)
    step()  # warm
    t0 = time.perf_counter()
    n = 0
    while True:
        step()
        n += 1
        if time.perf_counter() - t0 > seconds_target or n >= 50:
            break
    dt = (time.perf_counter() - t0) / n
    return {"value": 4 * nb / dt / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": "first %d GPT-2-state allocations (%d B), %d steps of full+incremental+verify+restore, "
                      "%.1f s" % (len(sample), nb, n, dt * n)}


def sample_allocations(sizes, cap_bytes, seed):
    spec = workloads.gpt2_state_spec()
    rng = np.random.default_rng(seed)
    out, tot = [], 0
    for (name, n, dt, dist, std) in spec:
        if tot >= cap_bytes:
            break
        if dt == "bfloat16":
            x = (rng.standard_normal(n, dtype=np.float32) * std).view(np.uint32) >> 16
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
    if rank != 0:
        return
    import oracle
    _, sizes, _, _ = gpt2_layout()
    sample = sample_allocations(sizes, args.cpu_sample_bytes, args.seed)
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    step, nb = oracle_step_sample(sample, args.dirty, args.seed)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    v = 4 * nb / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": workload_config(args),
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": "first %d GPT-2-state allocations (%d B) per step" % (len(sample), nb)},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def workload_config(args):
    return {"workload": "GPT-2-small training state: 593 allocations (148 tensors x fp32 W/G/m/v + 256 MiB "
                        "bf16 activations), 2,259,472,384 B, 64 KiB CRC-32C chunks",
            "step": "full checkpoint + %.0f%% clustered mutation + incremental checkpoint + verify + restore"
                    % (100 * args.dirty),
            "state_bytes": 2259472384, "chunk_bytes": UNIT, "dirty_frac": args.dirty,
            "image": "pinned, device-mapped host memory",
            "l2": "inputs (2.26 GB) larger than the 126 MB L2; no flush"}


# ---------------------------------------------------------------- GPU arm
def run_snap(args, rank, world, local, pg):
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
           "hash_kernel": [], "diff": [], "dirty_gather": []}
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
            per["diff"].append(st_incr["diff_ms"])
            per["dirty_gather"].append(st_incr["copy_ms"])
            counts["kernels"] += sum(int(x["kernel_launches"]) for x in (st_full, st_incr, st_ver, st_res))
            counts["patch_bytes"] = used_patch
            counts["dirty"] = st_incr["dirty_chunks"]
        return used_full, used_patch

    for _ in range(max(3, args.warmup)):
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
    for _ in range(args.steps):
        used_full, used_patch = step(True)
    t_end.record()
    torch.cuda.synchronize()
    h1 = time.perf_counter()
    barrier(pg)
    clk = clocks.stop()
    ms = t_start.elapsed_time(t_end) / args.steps
    ms_max = reduce_max(pg, ms)
    host_ms_max = reduce_max(pg, (h1 - h0) * 1e3 / args.steps)
    total_bytes = reduce_sum(pg, 4.0 * B)
    value = total_bytes / (ms_max * 1e-3) / 1e9

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
    hash_ms = statistics.mean(per["hash_kernel"])
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": workload_config(args),
        "roofline": {"bound": "host_link", "kernel": "snap_tiles (OP_GATHER, full checkpoint)",
                     "achieved": achieved, "peak": peaks["d2h"], "unit": "GB/s", "frac": achieved / peaks["d2h"],
                     "peak_source": "pinned cudaMemcpyAsync D2H, 1 GiB, best of 5, measured in this run",
                     "traffic": traffic_from_profiles("snap_tiles_gather")},
        "roofline_restore": {"bound": "host_link", "kernel": "snap_tiles (OP_SCATTER)",
                             "achieved": B / (statistics.mean(per["scatter_kernel"]) * 1e-3) / 1e9,
                             "peak": peaks["h2d"], "unit": "GB/s",
                             "frac": B / (statistics.mean(per["scatter_kernel"]) * 1e-3) / 1e9 / peaks["h2d"]},
        "roofline_hash": {"bound": "hbm", "kernel": "snap_tiles (OP_HASH, incremental hash pass)",
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
            "hash_ms": hash_ms, "diff_ms": statistics.mean(per["diff"]),
            "dirty_gather_ms": statistics.mean(per["dirty_gather"]),
            "gather_kernel_ms": gather_ms, "scatter_kernel_ms": statistics.mean(per["scatter_kernel"]),
        },
        "link_peak_gbs": peaks,
        "e2e": {"value": total_bytes / (host_ms_max * 1e-3) / 1e9, "unit": "GB/s",
                # restored state bytes + the hash tables uploaded by restore and verify
                "h2d_bytes_per_step": B + 2 * 4 * sum((n + UNIT - 1) // UNIT for n in sizes),
                # the full image and the patch written over the link
                "d2h_bytes_per_step": used_full + used_patch,
                "note": "host wall clock around the public API calls of the step (Python binding -> C ABI "
                        "-> graph launch -> completion), images in pinned host memory"},
        "gpu_launches": counts["kernels"],
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = [v.cpu().numpy() for v in views[: max(1, _first_n(sizes, args.cpu_sample_bytes))]]
        line["cpu_baseline"] = cpu_baseline(sample, args)
    if rank == 0:
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
    else:
        run_snap(args, rank, world, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
