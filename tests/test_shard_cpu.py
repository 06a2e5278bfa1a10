"""Multi-rank path on CPU: grids of a batch are split across ranks by LPT on
cell count (no collective on the data path); two gloo ranks each advance
their shard and the gathered results equal the unsplit run bit for bit."""
import os
import socket

import numpy as np
import pytest

from paper_2106_13465_gb300 import problems as pr
from paper_2106_13465_gb300.shard import lpt_split


def test_lpt_split_is_a_balanced_partition():
    costs = [50, 10, 40, 30, 30, 20, 5, 15]
    parts = lpt_split(costs, 3)
    assert sorted(i for p in parts for i in p) == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)
    assert lpt_split(costs, 3) == parts            # deterministic
    assert lpt_split(costs, 1) == [list(range(len(costs)))]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle as O
    from paper_2106_13465_gb300.shard import shard_of
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pbs = pr.batch(6, seed=17, lo=8, hi=40)
    mine = shard_of(pbs, rank, world)
    results = {g: O.run(pbs[g].U, pbs[g].h, pbs[g].bc, 4)[0] for g in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, results)
    if rank == 0:
        merged = {}
        for part in gathered:
            merged.update(part)
        np.savez(os.path.join(out_dir, "merged.npz"), **{str(k): v for k, v in merged.items()})
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_the_unsplit_run(tmp_path):
    import oracle as O
    import torch.multiprocessing as mp
    O.build()
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    merged = np.load(tmp_path / "merged.npz")
    pbs = pr.batch(6, seed=17, lo=8, hi=40)
    assert sorted(int(k) for k in merged.files) == list(range(len(pbs)))
    for g, p in enumerate(pbs):
        want, _, _ = O.run(p.U, p.h, p.bc, 4)
        assert np.array_equal(merged[str(g)], want)
