"""The two-phase coordination of snap_coordinate (the library's host code, no
GPU) on CPU ranks: gloo, world size 2, statuses combined by all-reduce.

Sec. 3.1: every task is locked before any is checkpointed, and the operation
counts only if it succeeded for all; a failure on one rank must abort the
others (no commit anywhere), and a rank that never answers must not leave
the others committed."""
import datetime
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


# (name, per-rank failures); every scenario runs in the same two processes
SCENARIOS = [
    ("ok", {}),
    ("lock_fail", {1: {"lock": -4}}),        # ETIMEDOUT on rank 1
    ("run_fail", {0: {"run": -3}}),          # ECUDA on rank 0
    ("both_fail", {0: {"run": -10}, 1: {"run": -3}}),  # EIO, ECUDA
]


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import paper_2502_16631_b300 as snap
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=30))
    agree = snap.all_reduce_agree()
    for name, fails in SCENARIOS:
        log = []
        fail = fails.get(rank, {})

        def step(what, status):
            def f():
                log.append(what)
                return status
            return f

        rc = snap.coordinate(agree, lock=step("lock", fail.get("lock", snap.OK)),
                             run=step("run", fail.get("run", snap.OK)),
                             commit=lambda: log.append("commit"), abort=lambda: log.append("abort"))
        q.put((name, rank, rc, log))
        dist.barrier()
    # a rank that leaves mid-protocol: rank 1 answers phase 0, then exits
    pg = dist.new_group(backend="gloo", timeout=datetime.timedelta(seconds=3))
    if rank == 1:
        t = torch.tensor([snap.OK], dtype=torch.int32)
        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=pg)
        q.put(("leave", rank, "left", ["lock"]))
        q.close()
        q.join_thread()  # flush the queue before leaving without cleanup
        os._exit(0)
    log = []
    rc = snap.coordinate(snap.all_reduce_agree(pg), lock=lambda: log.append("lock") or snap.OK,
                         run=lambda: log.append("run") or snap.OK, commit=lambda: log.append("commit"),
                         abort=lambda: log.append("abort"))
    q.put(("leave", rank, rc, log))
    q.close()
    q.join_thread()
    os._exit(0)  # the group cannot be torn down cleanly with its peer gone


@pytest.fixture(scope="module")
def results():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = {}
    for _ in range(2 * (len(SCENARIOS) + 1)):
        name, rank, rc, log = q.get(timeout=180)
        out[(name, rank)] = (rc, log)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def test_all_ranks_succeed_all_commit(results):
    for r in (0, 1):
        assert results[("ok", r)] == (0, ["lock", "run", "commit"])


def test_lock_failure_on_one_rank_stops_every_rank_before_running(results):
    import paper_2502_16631_b300 as snap
    assert results[("lock_fail", 0)] == (snap.EPEER, ["lock"])
    assert results[("lock_fail", 1)] == (snap.ETIMEDOUT, ["lock"])


def test_run_failure_on_one_rank_aborts_every_rank(results):
    import paper_2502_16631_b300 as snap
    assert results[("run_fail", 0)] == (snap.ECUDA, ["lock", "run", "abort"])
    assert results[("run_fail", 1)] == (snap.EPEER, ["lock", "run", "abort"])


def test_failures_on_both_ranks_keep_their_own_status(results):
    import paper_2502_16631_b300 as snap
    assert results[("both_fail", 0)] == (snap.EIO, ["lock", "run", "abort"])
    assert results[("both_fail", 1)] == (snap.ECUDA, ["lock", "run", "abort"])


def test_rank_that_leaves_mid_protocol_aborts_the_other(results):
    """Rank 1 agrees on phase 0 and exits without answering phase 1: rank 0's
    all-reduce fails (peer gone, or the group's 3 s timeout), which the
    binding reports as a failure, so rank 0 aborts and never commits."""
    import paper_2502_16631_b300 as snap
    assert results[("leave", 0)] == (snap.EPEER, ["lock", "run", "abort"])
    assert results[("leave", 1)] == ("left", ["lock"])


def test_single_rank_protocol_and_argument_check():
    import paper_2502_16631_b300 as snap
    log = []
    rc = snap.coordinate(lambda ph, st: st, lock=lambda: 0, run=lambda: snap.ENOMEM,
                         commit=lambda: log.append("c"), abort=lambda: log.append("a"))
    assert rc == snap.ENOMEM and log == ["a"]
    # a step that raises counts as a failure
    rc = snap.coordinate(lambda ph, st: st, run=lambda: 1 / 0, abort=lambda: log.append("a2"))
    assert rc == snap.ECUDA and log == ["a", "a2"]
    assert snap.lib().snap_coordinate(None, None) == snap.EINVAL
