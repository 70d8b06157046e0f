"""Host logic of bench.py's multi-rank run, executed by `torch.distributed.run` with the gloo backend on CPU (no
GPU): the max / sum reductions over ranks, one facade component per rank, and that the components differ.  Every
rank prints one JSON line prefixed with its rank."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402
import scenes  # noqa: E402


def main():
    rank, world, _ = bench._dist()
    dist.init_process_group("gloo")
    out = {"rank": rank, "world": world,
           "max": bench._reduce(1.5 + rank, "max", world, "cpu"),
           "sum": bench._reduce(100 * (rank + 1), "sum", world, "cpu"),
           "seed": bench._facade_seed(rank)}
    sc = scenes.facade(seed=out["seed"], n_images=6, n_kp=400, n_points=3000, n_pairs=6, min_covis=5)
    sig = [float(sc.images[0].xy[:16].sum()), int(sc.images[0].desc[:4].sum())]
    sigs = [None] * world
    dist.all_gather_object(sigs, sig)
    out["signatures"] = sigs
    dist.barrier()
    dist.destroy_process_group()
    os.write(1, (f"RANK{rank} " + json.dumps(out) + "\n").encode())   # one write: the ranks share the pipe


if __name__ == "__main__":
    main()
