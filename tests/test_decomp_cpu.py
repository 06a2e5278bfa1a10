"""Slab decomposition of one grid across ranks (the paper's Coarse-Grain
subdomains with a ghost-row exchange, §3 and §5): host logic on the CPU.
The ranks' compute runs on the FP64 oracle here (a stand-in backend with
the library backend's interface); the owned rows of all ranks together
equal the unsplit oracle run bit for bit, with the ranks in one process and
as two gloo processes."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2106_13465_gb300 import decomp as D
from paper_2106_13465_gb300 import problems as pr

P_, T_, R_ = pr.PERIODIC, pr.TRANSMISSIVE, pr.REFLECT


class OracleBackend:
    """A rank's local grid advanced by the oracle (one step per call, dt
    given, the sweep order set by the global step count)."""

    def __init__(self, slab, nx, h, bc, U_local, step0=0):
        self.nx, self.h, self.bc = nx, h, slab.local_bc(bc)
        self.U = np.array(U_local, dtype=np.float64)
        self.k = step0

    def get_rows(self, row0, nrows):
        return self.U[:, row0:row0 + nrows].copy()

    def set_rows(self, row0, rows):
        rows = rows.numpy() if hasattr(rows, "numpy") else rows
        self.U[:, row0:row0 + rows.shape[1]] = rows

    def cfl_dt(self):
        return O.cfl_dt(self.U, self.h)

    def step(self, dt):
        self.U, _, _ = O.run(self.U, self.h, self.bc, 1, step0=self.k, dt_override=np.array([dt]))
        self.k += 1


def _make_ranks(pb, world, step0=0):
    out = []
    for s in D.slabs(pb.ny, pb.bc, world):
        U_local = pb.U[:, s.local_rows()]
        out.append(D.SlabRank(s, OracleBackend(s, pb.nx, pb.h, pb.bc, U_local, step0)))
    return out


def test_split_rows_and_halos():
    assert D.split_rows(10, 3) == [(0, 4), (4, 7), (7, 10)]
    with pytest.raises(ValueError):
        D.split_rows(5, 3)
    s = D.slabs(10, (R_, R_, R_, R_), 3)
    assert [(x.lo, x.hi) for x in s] == [(False, True), (True, True), (True, False)]
    assert [x.local_ny for x in s] == [6, 7, 5]
    assert s[0].local_bc((R_, T_, R_, T_)) == (R_, T_, R_, T_)
    assert s[1].local_bc((R_, T_, R_, T_)) == (R_, T_, T_, T_)
    assert s[2].local_bc((R_, T_, R_, T_)) == (R_, T_, T_, T_)
    p = D.slabs(10, (P_,) * 4, 2)
    assert all(x.lo and x.hi for x in p)
    assert list(p[0].local_rows()) == [8, 9, 0, 1, 2, 3, 4, 5, 6]
    assert list(p[1].local_rows()) == [3, 4, 5, 6, 7, 8, 9, 0, 1]
    one = D.slabs(10, (P_,) * 4, 1)[0]
    assert not one.lo and not one.hi and one.local_ny == 10


CASES = [
    ("modes_periodic", lambda: pr.random_modes(37, 23, seed=1)),
    ("sedov_reflect", lambda: pr.sedov(30, 26)),
    ("sod_y", lambda: pr.sod(6, 40, 1)),
    ("mixed", lambda: pr.Problem("m", pr.random_modes(29, 31, seed=2).U, 1 / 31, (P_, P_, R_, T_))),
]


@pytest.mark.parametrize("world", [2, 3, 4])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_slab_ranks_in_one_process_equal_the_unsplit_run(name, make, world):
    pb = make()
    want, _, _ = O.run(pb.U, pb.h, pb.bc, 7, step0=1)
    ranks = _make_ranks(pb, world, step0=1)
    D.step_in_process(ranks, 7)
    got = np.concatenate([rk.owned_state() for rk in ranks], axis=1)
    assert np.array_equal(got, want), name


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    results = {}
    for name, make in CASES:
        pb = make()
        s = D.slabs(pb.ny, pb.bc, world)[rank]
        rk = D.SlabRank(s, OracleBackend(s, pb.nx, pb.h, pb.bc, pb.U[:, s.local_rows()]))
        D.step_distributed(rk, 6, dist)
        results[name] = rk.owned_state()
    gathered = [None] * world
    dist.all_gather_object(gathered, results)
    if rank == 0:
        for name, _ in CASES:
            np.save(os.path.join(out_dir, name + ".npy"),
                    np.concatenate([g[name] for g in gathered], axis=1))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_the_unsplit_run(tmp_path):
    import torch.multiprocessing as mp
    O.build()
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for name, make in CASES:
        pb = make()
        want, _, _ = O.run(pb.U, pb.h, pb.bc, 6)
        assert np.array_equal(np.load(tmp_path / (name + ".npy")), want), name
