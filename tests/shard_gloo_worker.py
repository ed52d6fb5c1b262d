"""One rank of a sharded oracle run over torch.distributed (gloo, CPU),
launched by torchrun from tests/test_shard_host.py: the ranks exchange
their cut line ends' values after every window through
paper_1903_01081_b300.shard.run_distributed; rank 0 gathers every rank's
node voltages and prints, as one JSON line, how they compare with the
whole network run in one oracle process."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import numpy as np
import torch.distributed as dist

import oracle
from oracle_shard import OracleShard
from paper_1903_01081_b300 import netgen as g
from paper_1903_01081_b300.shard import run_distributed


def network(kind):
    base = g.multi_subsystem(77, [4, 5, 3, 6, 4, 5], n_lines=10, n_sources=3, dt=20e-6, n_series_extra=2)
    if kind == "coupled":
        return g.with_coupled_lines(base, seed=1007)
    if kind == "fd":
        return g.with_fd_lines(base, seed=1009)
    return base


def main():
    kind, n_steps, min_window = sys.argv[1], int(sys.argv[2]), int(sys.argv[3])
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    net = network(kind)
    eng = OracleShard(net, rank, world, min_window=min_window)
    run_distributed(eng, n_steps)
    parts = [None] * world
    dist.all_gather_object(parts, (eng.owned_nodes, eng.voltages(), len(eng.peers), eng.window))
    if rank == 0:
        ref = oracle.simulate(net, n_steps)
        got = np.zeros_like(ref)
        owned = np.zeros(net.n_nodes, dtype=int)
        for mask, v, _, _ in parts:
            got[:, mask] = v[:, mask]
            owned += mask
        print(json.dumps({"world": world, "window": parts[0][3], "peers": [p[2] for p in parts],
                          "each_node_once": bool(np.all(owned == 1)),
                          "bitwise": bool(np.array_equal(got, ref)),
                          "max_abs_diff": float(np.max(np.abs(got - ref))),
                          "nodes_per_rank": [int(p[0].sum()) for p in parts]}))
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
