"""bench.py's host-side pieces, without a GPU: the committed ncu traffic
figures parse for the current kernel code, and the reference arm (the CPU
oracle on a sample of the default step) prints one well-formed line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_rows_parse():
    r = bench.traffic_ratio_from_profiles("snap_tiles_gather")
    assert r is None or 0.99 < r < 1.1
    t = bench.gather_traffic(2259472384)
    assert t is None or 2.2e9 < t < 2.5e9
    bench.traffic_from_profiles("snap_tiles_gather")  # never raises


def test_reference_arm_prints_one_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-sample-bytes", str(16 << 20)],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "GB/s"
    assert d["config"]["workload"].startswith("Llama-7B")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_default_state_fits_every_rank_of_the_host(monkeypatch):
    """Each rank of the default step holds one pageable image of its state:
    with more ranks than the host's memory allows, every rank keeps the same
    longest prefix of allocations that fits (and the line says so), so N
    ranks never ask for more host memory than there is."""
    import workloads
    GiB = 1 << 30
    spec = workloads.llama7b_state_spec()
    full = sum(workloads.spec_bytes(spec))

    def fake_sysconf(avail_bytes):
        page = 4096
        return lambda name: page if name == "SC_PAGE_SIZE" else avail_bytes // page

    monkeypatch.setattr(os, "sysconf", fake_sysconf(196 * GiB))
    kept, reduced = bench.llama7b_sizes_for_host(spec, 1)
    assert kept == spec and reduced is None and full < 196 * GiB
    for world in (2, 4, 8):
        kept, reduced = bench.llama7b_sizes_for_host(spec, world)
        per_rank = 196 * GiB // world - 24 * GiB
        assert reduced and sum(workloads.spec_bytes(kept)) <= max(per_rank, 0)
        assert kept == spec[: len(kept)]
