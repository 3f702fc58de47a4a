"""GPU parity of images persisted to storage: the file written by
snap_checkpoint_file is byte-identical to the oracle's image, a restore from
the file reproduces the state, and a failed write leaves neither a file under
the caller's name nor a moved base."""
import os
import shutil

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2502_16631_b300 as snap
import workloads

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

MiB = 1 << 20
SIZES = [65536, 4096 * 3 + 16, 1, 0, 200000, 65536 * 2, 12345, 17, 65537, 3 * 65536 - 1, 5 * MiB + 48]


@pytest.fixture(scope="module", autouse=True)
def _oracle_threads():
    oracle.set_threads(min(16, len(os.sched_getaffinity(0))))
    yield
    oracle.set_threads(1)


def device_state(sizes, seed):
    ts, hs = [], []
    for k, n in enumerate(sizes):
        h = workloads.xorshift_bytes(n, seed, k)
        t = torch.empty(n, dtype=torch.uint8, device="cuda")
        if n:
            t.copy_(torch.from_numpy(h))
        ts.append(t)
        hs.append(h)
    torch.cuda.synchronize()
    return ts, hs


def make_set(ts, C=65536, **kw):
    s = snap.Set(chunk_bytes=C, **kw)
    for t in ts:
        s.register(t.data_ptr() if t.numel() else 0, t.numel())
    s.tensors = ts
    return s


def readback(ts):
    torch.cuda.synchronize()
    return [t.cpu().numpy().copy() if t.numel() else np.zeros(0, np.uint8) for t in ts]


def scribble(ts, C, chunks, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    for k, i in chunks:
        lo, hi = i * C, min((i + 1) * C, ts[k].numel())
        ts[k][lo:hi] ^= torch.randint(1, 256, (hi - lo,), dtype=torch.uint8, device="cuda", generator=g)
    torch.cuda.synchronize()


def load(path):
    return np.fromfile(path, dtype=np.uint8)


@pytest.mark.parametrize("C,ring", [(65536, 0), (4096, 1 * MiB), (65536, 2 * MiB)])
def test_file_full_incremental_restore(tmp_path, C, ring):
    ts, hs = device_state(SIZES, seed=101)
    s = make_set(ts, C, ring_bytes=ring)
    full = str(tmp_path / "full.img")
    used = s.checkpoint_file(full, snap.FULL)
    assert not os.path.exists(full + ".tmp")
    img = load(full)
    rc, exp = oracle.write_full(hs, C, generation=0)
    assert used == exp.size == img.size and np.array_equal(img, exp)
    # incremental into a second file
    nch = [oracle.n_chunks(x, C) for x in SIZES]
    dirty = [(0, 0), (4, nch[4] - 1), (8, 1), (10, 3), (10, nch[10] - 1)]
    scribble(ts, C, dirty, 102)
    cur = readback(ts)
    pfile = str(tmp_path / "gen1.patch")
    used = s.checkpoint_file(pfile, snap.INCREMENTAL, sync=True)
    patch = load(pfile)
    rc, pexp, nd = oracle.write_patch(cur, C, [oracle.chunk_hashes(h, C) for h in hs], 1, 0)
    assert nd == len(set(dirty)) and used == pexp.size == patch.size
    assert np.array_equal(patch, pexp)
    merged = img.copy()
    snap.apply_patch(merged, patch)
    assert np.array_equal(merged, oracle.write_full(cur, C, generation=1)[1])
    # restore the generation-0 file into zeroed buffers
    for t in ts:
        t.zero_()
    s.restore_file(full)
    for a, b in zip(readback(ts), hs):
        assert np.array_equal(a, b)
    n = sum(nch)
    got, gen = s.committed_hashes(n)
    assert gen == 0 and np.array_equal(got, np.concatenate([oracle.chunk_hashes(h, C) for h in hs]))
    assert s.restore_file_status(pfile) == snap.EFORMAT  # a patch must be merged first
    s.close()


def test_file_failures_leave_no_image_and_keep_the_base(tmp_path):
    ts, hs = device_state(SIZES, seed=103)
    s = make_set(ts, 65536)
    good = str(tmp_path / "a.img")
    s.checkpoint_file(good, snap.FULL)
    n = sum(oracle.n_chunks(x, 65536) for x in SIZES)
    h0, g0 = s.committed_hashes(n)
    scribble(ts, 65536, [(0, 0)], 104)
    bad = str(tmp_path / "missing-dir" / "b.img")
    rc, _ = s.checkpoint_file_status(bad, snap.INCREMENTAL)
    assert rc == snap.EIO
    assert not os.path.exists(bad) and not os.path.exists(bad + ".tmp")
    h1, g1 = s.committed_hashes(n)
    assert g1 == g0 and np.array_equal(h0, h1)  # nothing committed
    # the next incremental is still against generation 0
    p = str(tmp_path / "c.patch")
    s.checkpoint_file(p, snap.INCREMENTAL)
    rc, exp, nd = oracle.write_patch(readback(ts), 65536, [oracle.chunk_hashes(h, 65536) for h in hs], 1, 0)
    assert nd == 1 and np.array_equal(load(p), exp)
    # restore errors: no file, truncated file, wrong set, bad flags
    assert s.restore_file_status(str(tmp_path / "nope.img")) == snap.EIO
    trunc = str(tmp_path / "t.img")
    load(good)[: 100000].tofile(trunc)
    assert s.restore_file_status(trunc) == snap.EFORMAT
    short = str(tmp_path / "s.img")
    load(good)[:40].tofile(short)
    assert s.restore_file_status(short) == snap.EFORMAT
    other = make_set(ts[:-1], 65536)
    assert other.restore_file_status(good) == snap.EMISMATCH
    assert snap.lib().snap_checkpoint_file(s.h, good.encode(), snap.FULL, 2, None) == snap.EINVAL
    s.close()
    other.close()


def test_file_gpt2_state_roundtrip(tmp_path):
    """GPT-2 small training state (593 allocations, 2.26 GB) through a file:
    the file equals the oracle's image; restore from it is byte-exact."""
    spec = workloads.gpt2_state_spec()
    sizes = workloads.spec_bytes(spec)
    need = 2 * sum(sizes) + (1 << 30)
    if shutil.disk_usage(str(tmp_path)).free < need:
        pytest.skip("needs %d free bytes under %s" % (need, tmp_path))
    ts = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
    workloads.torch_fill_spec(ts, spec, seed=105)
    s = make_set(ts, 65536)
    path = str(tmp_path / "gpt2.img")
    used = s.checkpoint_file(path, snap.FULL)
    host = readback(ts)
    rc, exp = oracle.write_full(host, 65536, 0)
    img = load(path)
    assert used == exp.size and np.array_equal(img, exp)
    del exp, img
    for t in ts:
        t.zero_()
    s.restore_file(path)
    for a, b in zip(readback(ts), host):
        assert np.array_equal(a, b)
    s.close()
    os.unlink(path)


_FSIZE_CHILD = r'''
import os, resource, signal, sys
sys.path.insert(0, os.environ["SNAP_REPO"])
import numpy as np, torch
import paper_2502_16631_b300 as snap
path = sys.argv[1]
ts = [torch.ones(3 << 20, dtype=torch.uint8, device="cuda"), torch.ones(5 << 20, dtype=torch.uint8, device="cuda")]
s = snap.Set(chunk_bytes=65536)
for t in ts:
    s.register(t)
s.prepare(ring=True)
signal.signal(signal.SIGXFSZ, signal.SIG_IGN)          # a write past the limit fails with EFBIG
resource.setrlimit(resource.RLIMIT_FSIZE, (1 << 20, 1 << 20))
rc, _ = s.checkpoint_file_status(path, snap.FULL)
print(rc, os.path.exists(path), os.path.exists(path + ".tmp"))
'''


def test_file_write_failure_is_eio_and_leaves_nothing(tmp_path):
    """Storage that refuses the image (a 1 MiB file-size limit in a child
    process): SNAP_EIO, no file under the name, no temporary file left."""
    import subprocess
    import sys
    path = str(tmp_path / "big.img")
    env = dict(os.environ, SNAP_REPO=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    r = subprocess.run([sys.executable, "-c", _FSIZE_CHILD, path], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    rc, exists, tmp_exists = r.stdout.split()[-3:]
    assert int(rc) == snap.EIO and exists == "False" and tmp_exists == "False"
