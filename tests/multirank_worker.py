"""Body of one rank of the world-size-2 CPU test in test_multirank.py (kept
in its own module so that spawned ranks can import it)."""
import os

import numpy as np


def run_rank(rank, ws, port, R, nsteps, out_path):
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    import sft_inputs as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w = W.model_a_64(n=[16, 16], sigma0=0.3)
        f0 = W.initial_fields(w, replicas=ws * R)  # the whole ensemble; this rank steps its share
        o = oracle.Oracle(w.d, w.n, w.dx, R, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias,
                          replica0=bench.rank_replica0(rank, R))
        for r in range(R):
            o.set_field(r, f0[rank * R + r])
        o.step(nsteps)
        mine = torch.from_numpy(np.stack([o.field(r) for r in range(R)]))
        parts = [torch.zeros_like(mine) for _ in range(ws)]
        dist.all_gather(parts, mine)
        tmax = bench.max_over_ranks(10.0 + rank, dist, device="cpu")
        if rank == 0:
            np.savez(out_path, fields=torch.cat(parts).numpy(), tmax=tmax)
    finally:
        dist.destroy_process_group()
