"""GPU parity at the workloads' full sizes, in the launch configuration the
benchmark times (model-default tiles, CUDA graph of 20 steps):

* the 512-grid ragged batch (sides log-uniform in [32, 512], seed 2106):
  a seeded sample of grids element-wise against the oracle, every grid
  against a single-grid run bit for bit, and FP32 against FP64 on the same
  dt sequence at a stated density error;
* the paper's 10000^2 point explosion, 10 steps: every cell beyond the
  blast's reach exactly ambient, the corner against an oracle window.
"""
import numpy as np
import pytest

import oracle as O
from paper_2106_13465_gb300 import hydro as H
from paper_2106_13465_gb300 import problems as pr

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
# FP32 batch (FP64 dt replayed, 10 steps): relative L1 density error per grid
TOL_L1_FP32_BATCH = 5e-7  # measured 1.3e-7 (worst grid)


def rel_err(a, b, floor_frac=1e-3):
    """Unfloored relative error for density and energy, floored at
    floor_frac of the plane's largest magnitude for the momenta."""
    worst = 0.0
    for q in range(a.shape[0]):
        den = np.abs(b[q])
        if q in (1, 2):
            den = np.maximum(den, floor_frac * den.max())
        den = np.where(den > 0, den, 1.0)
        worst = max(worst, float((np.abs(a[q] - b[q]) / den).max()))
    return worst


@pytest.fixture(scope="module")
def batch_run():
    pbs = pr.batch(512)
    grids = [(p.nx, p.ny, p.h, p.bc) for p in pbs]
    with H.Context(grids, precision=64) as c:
        for g, p in enumerate(pbs):
            c.set_state(g, p.U)
        dts = c.step(10, record_dt=True)
        out64 = [c.get_state(g) for g in range(len(pbs))]
    with H.Context(grids, precision=32) as c:
        for g, p in enumerate(pbs):
            c.set_state(g, p.U)
        c.step(10, dt_override=dts)
        out32 = [c.get_state(g) for g in range(len(pbs))]
    return pbs, dts, out64, out32


def test_batch512_sample_matches_oracle(batch_run):
    pbs, dts, out64, _ = batch_run
    rng = np.random.default_rng(2106)
    sample = rng.choice(len(pbs), size=16, replace=False)
    kinds = {pbs[g].meta["kind"] for g in sample}
    assert len(kinds) >= 3
    for g in sample:
        p = pbs[g]
        want, odts, _ = O.run(p.U, p.h, p.bc, 10, threads=0)
        assert rel_err(out64[g], want) <= TOL64, (g, p.name)
        np.testing.assert_allclose(dts[:, g], odts, rtol=1e-12)


def test_batch512_every_grid_equals_its_single_grid_run(batch_run):
    pbs, dts, out64, _ = batch_run
    for g, p in enumerate(pbs):
        with H.Context([(p.nx, p.ny, p.h, p.bc)], precision=64) as c:
            c.set_state(0, p.U)
            c.step(10)
            single = c.get_state(0)
        assert np.array_equal(single, out64[g]), (g, p.name)


def test_batch512_fp32_density_error_against_fp64(batch_run):
    pbs, _dts, out64, out32 = batch_run
    worst = 0.0
    for g in range(len(pbs)):
        l1 = np.abs(out32[g][0] - out64[g][0]).sum() / np.abs(out64[g][0]).sum()
        worst = max(worst, float(l1))
    assert worst <= TOL_L1_FP32_BATCH, worst


def test_explosion_10000_sampled_against_oracle_window():
    """The paper's 10000^2 point explosion, 10 steps, in FP64: after k steps
    the blast has reached at most 2k cells along each axis (two per sweep),
    so every cell outside that corner square is exactly ambient, and the
    corner equals what the oracle computes on a 256^2 window with the same h
    (its artificial far walls reach only the last 2k cells of the window)."""
    k = 10
    pb = pr.sedov(10000)
    with H.Context([(pb.nx, pb.ny, pb.h, pb.bc)], precision=64) as c:
        c.set_state(0, pb.U)
        gdts = c.step(k, record_dt=True)[:, 0]
        got = c.get_state(0)
    reach = 2 * k + 1
    amb = pb.U[:, -1, -1]
    for q in range(4):
        plane = got[q]
        assert np.all(plane[reach:, :] == amb[q])
        assert np.all(plane[:reach, reach:] == amb[q])
    win = pb.U[:, :256, :256].copy()
    want, odts, _ = O.run(win, pb.h, pb.bc, k, threads=0)
    np.testing.assert_allclose(gdts, odts, rtol=1e-12)
    m = 256 - reach
    assert rel_err(got[:, :m, :m], want[:, :m, :m]) <= TOL64
