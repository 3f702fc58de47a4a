"""Small, fixed workloads for ncu captures of single kernels (run by hand
under `ncu`; not collected by pytest).

    python tests/profile_cases.py gather [reps]   # 8 x 64 MiB, full checkpoints
    python tests/profile_cases.py scatter [reps]  # 8 x 64 MiB, restores
    python tests/profile_cases.py hash [reps]     # 1 GiB chunk hasher
    python tests/profile_cases.py cut [reps]      # 8 x 64 MiB, asynchronous checkpoints
                                                  # (k_shadow_copy is the cut)
    python tests/profile_cases.py ring [reps]     # 8 x 256 MiB, full checkpoints through the
                                                  # 4 GiB ring into a pageable image (32 gather
                                                  # launches of one 64 MiB window each)
    python tests/profile_cases.py ringrestore [reps]  # the same state: one ring checkpoint, then
                                                  # restores through the ring (32 scatter
                                                  # launches each)
    python tests/profile_cases.py fused [reps]    # 8 x 256 MiB, one full checkpoint, then fused
                                                  # incremental checkpoints with 10 % of the
                                                  # chunks changed before each (one cooperative
                                                  # launch each; its dirty runs go to the copy
                                                  # engines, the default)
    python tests/profile_cases.py fusedsm [reps]  # the same with the dirty chunks copied by
                                                  # gather CTAs of the launch (SNAP_INCR_COPY_SM)
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

import paper_2502_16631_b300 as snap  # noqa: E402

MiB = 1 << 20


def main():
    op = sys.argv[1]
    reps = int(sys.argv[2]) if len(sys.argv) > 2 else 2
    if op == "ring":
        import numpy as np
        ts = [torch.empty(256 * MiB, dtype=torch.uint8, device="cuda") for _ in range(8)]
        for t in ts:
            t.random_(0, 256)
        s = snap.Set(chunk_bytes=65536, ring_bytes=4096 * MiB)
        for t in ts:
            s.register(t)
        img = np.empty(s.image_bytes(snap.FULL), dtype=np.uint8)
        for _ in range(reps + 1):
            s.checkpoint(img, snap.FULL)
    elif op in ("fused", "fusedsm"):
        ts = [torch.empty(256 * MiB, dtype=torch.uint8, device="cuda") for _ in range(8)]
        for t in ts:
            t.random_(0, 256)
        s = snap.Set(chunk_bytes=65536, incr_copy=snap.INCR_COPY_SM if op == "fusedsm" else snap.INCR_COPY_DMA)
        for t in ts:
            s.register(t)
        full = snap.HostBuffer(s.image_bytes(snap.FULL))
        patch = snap.HostBuffer(s.image_bytes(snap.INCREMENTAL))
        s.checkpoint(full, snap.FULL)
        g = torch.Generator(device="cuda")
        g.manual_seed(5)
        for _ in range(reps):
            for t in ts:  # every tenth 64 KiB chunk changes
                t.view(-1, 65536)[::10] ^= 0x5A
            s.checkpoint(patch, snap.INCREMENTAL)
    elif op == "ringrestore":
        import numpy as np
        ts = [torch.empty(256 * MiB, dtype=torch.uint8, device="cuda") for _ in range(8)]
        for t in ts:
            t.random_(0, 256)
        s = snap.Set(chunk_bytes=65536, ring_bytes=4096 * MiB)
        for t in ts:
            s.register(t)
        img = np.empty(s.image_bytes(snap.FULL), dtype=np.uint8)
        used = s.checkpoint(img, snap.FULL)
        for _ in range(reps + 1):
            s.restore(img, used)
    elif op == "hash":
        x = torch.empty(1024 * MiB, dtype=torch.uint8, device="cuda")
        x.random_(0, 256)
        h = torch.empty(1024 * MiB // 65536, dtype=torch.int32, device="cuda")
        for _ in range(reps):
            snap.hash_chunks(x, 65536, h)
    else:
        ts = [torch.empty(64 * MiB, dtype=torch.uint8, device="cuda") for _ in range(8)]
        for t in ts:
            t.random_(0, 256)
        s = snap.Set(chunk_bytes=65536)
        for t in ts:
            s.register(t)
        img = snap.HostBuffer(s.image_bytes(snap.FULL))
        used = s.checkpoint(img, snap.FULL)
        for _ in range(reps):
            if op == "cut":
                s.checkpoint_async(img, snap.FULL)
                s.checkpoint_wait()
            elif op == "gather":
                s.checkpoint(img, snap.FULL)
            else:
                s.restore(img, used)
    torch.cuda.synchronize()
    print("done", op)


if __name__ == "__main__":
    main()
