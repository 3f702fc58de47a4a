"""The allocation-free chunk hasher against the allocating one.

snap_hash_chunks_noalloc exists for callers that cannot allocate GPU memory
(a checkpoint or crash handler that must leave the allocator it is saving
untouched, a process whose pool is exhausted or owned by another framework).
It must give exactly the hashes snap_hash_chunks gives buffer by buffer --
hashes are integers, so the comparison is exact -- on two calls in a row,
the second with a different buffer list, so that nothing left in the shared
static scratch by the first call leaks into the second.  Both are also held
to the CPU oracle's CRC-32C of the same bytes (read back with a plain
device-to-host copy).  This file is collected last; it passes alone in a
fresh process and after the others."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2502_16631_b300 as snap

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def reference(buffers, C):
    """The existing entry point, one buffer at a time."""
    out = []
    for t in buffers:
        n = (t.numel() + C - 1) // C
        if n == 0:
            continue
        h = torch.zeros(n, dtype=torch.int32, device="cuda")
        snap.hash_chunks(t, C, h)
        out.append(h.cpu().numpy().view(np.uint32))
    return np.concatenate(out) if out else np.zeros(0, np.uint32)


def noalloc(buffers, C):
    total = sum((t.numel() + C - 1) // C for t in buffers)
    out = torch.full((max(total, 1),), -1, dtype=torch.int32, device="cuda")
    rc = snap.hash_chunks_noalloc(buffers, C, out)
    assert rc == snap.OK, snap.strerror(rc)
    torch.cuda.synchronize()
    return out[:total].cpu().numpy().view(np.uint32)


def expected(buffers, C):
    """The oracle's chunk hashes of the buffers' bytes, in call order."""
    torch.cuda.synchronize()
    out = [oracle.chunk_hashes(t.cpu().numpy(), C) for t in buffers if t.numel()]
    return np.concatenate(out) if out else np.zeros(0, np.uint32)


def buffers_of(sizes, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return [torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda", generator=g) for n in sizes]


@pytest.mark.parametrize("C", [4096, 65536])
def test_noalloc_matches_allocating_hasher_twice(C):
    first = buffers_of([3 * C + 100, 1, 0, C, 12345, 5 * C], seed=1)
    second = buffers_of([C - 16, 2 * C + 1], seed=2)  # fewer buffers than the first call
    for bufs in (first, second):
        got = noalloc(bufs, C)
        assert np.array_equal(got, reference(bufs, C))
        assert np.array_equal(got, expected(bufs, C))


def test_noalloc_many_buffers_and_limit():
    C = 4096
    bufs = buffers_of([4096 + 16 * k for k in range(snap.NOALLOC_MAX_BUFFERS)], seed=3)
    got = noalloc(bufs, C)
    assert np.array_equal(got, reference(bufs, C))
    assert np.array_equal(got, expected(bufs, C))
    # one buffer over the static scratch's capacity is refused, nothing launched
    over = bufs + bufs[:1]
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    assert snap.hash_chunks_noalloc(over, C, out) == snap.EINVAL
    # and the entry point still works afterwards
    assert np.array_equal(noalloc(bufs[:3], C), reference(bufs[:3], C))


def test_noalloc_rejects_misaligned_buffer():
    t = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert snap.hash_chunks_noalloc([(t.data_ptr() + 8, 100)], 4096, out) == snap.EINVAL
