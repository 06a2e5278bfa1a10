"""Slab decomposition with the library backend: several ranks' contexts on
one GPU, advanced by the host in lockstep (messages handed over directly,
no kernel waits for another rank's), against the unsplit GPU run bit for
bit and against the oracle.  Each rank's step is an ordinary library step
of its local grid with the global dt; the exchange goes through
hydro_get_rows / hydro_set_rows."""
import numpy as np
import pytest

import oracle as O
from paper_2106_13465_gb300 import decomp as D
from paper_2106_13465_gb300 import hydro as H
from paper_2106_13465_gb300 import problems as pr

pytestmark = pytest.mark.gpu

P_, T_, R_ = pr.PERIODIC, pr.TRANSMISSIVE, pr.REFLECT


def _unsplit(pb, n, precision, fused=0):
    with H.Context([(pb.nx, pb.ny, pb.h, pb.bc)], precision=precision) as c:
        c.set_tuning(fused=fused)
        c.set_state(0, pb.U)
        c.step(n)
        return c.get_state(0)


def _split(pb, n, world, precision, fused=0):
    ranks = []
    for s in D.slabs(pb.ny, pb.bc, world):
        b = D.LibBackend(s, pb.nx, pb.h, pb.bc, pb.U[:, s.local_rows()], precision=precision)
        b.ctx.set_tuning(fused=fused)
        ranks.append(D.SlabRank(s, b))
    D.step_in_process(ranks, n)
    out = np.concatenate([rk.owned_state() for rk in ranks], axis=1)
    for rk in ranks:
        rk.b.close()
    return out


CASES = [
    ("modes_periodic", lambda: pr.random_modes(131, 97, seed=3)),
    ("sedov_reflect", lambda: pr.sedov(90, 70)),
    ("mixed", lambda: pr.Problem("m", pr.random_modes(64, 67, seed=4).U, 1 / 67, (R_, T_, P_, P_))),
]


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_slab_ranks_equal_the_unsplit_gpu_run(name, make, world, precision):
    pb = make()
    want = _unsplit(pb, 9, precision)
    got = _split(pb, 9, world, precision)
    assert np.array_equal(got, want), (name, world, precision)


def test_slab_ranks_fused_steps_and_oracle():
    pb = pr.random_modes(75, 64, seed=5)
    want, _, _ = O.run(pb.U, pb.h, pb.bc, 8)
    got = _split(pb, 8, 2, 64, fused=1)
    assert np.array_equal(got, _unsplit(pb, 8, 64))
    scale = np.abs(want).reshape(4, -1).max(axis=1)[:, None, None]
    floor = np.array([0.0, 1e-3, 1e-3, 0.0])[:, None, None] * scale
    assert float(np.max(np.abs(got - want) / np.maximum(np.abs(want), floor))) <= 1e-11


def test_rows_round_trip_and_speed_refresh():
    pb = pr.random_modes(40, 30, seed=6)
    with H.Context([(pb.nx, pb.ny, pb.h, pb.bc)], precision=64) as c:
        c.set_state(0, pb.U)
        rows = c.get_rows(0, 5, 3)
        assert np.array_equal(rows, pb.U[:, 5:8])
        fast = rows.copy()
        fast[1] *= 4.0  # faster gas in three rows: the CFL step must shrink
        dt0 = c.cfl_dt(0)
        c.set_rows(0, 5, fast)
        U = pb.U.copy()
        U[:, 5:8] = fast
        assert c.cfl_dt(0) == pytest.approx(O.cfl_dt(U, pb.h), rel=1e-14)
        assert c.cfl_dt(0) < dt0
        assert np.array_equal(c.get_state(0), U)
        assert H.hydro_set_rows(c.ctx, 0, 29, 2, fast.ctypes.data, 0) == H.HYDRO_EINVAL
