"""The fused step kernel (hydro_tuning.fused = 1: both sweeps of a step on a
tile held in shared memory, one HBM pass per step) gives the same bits as
the split sweeps, for both precisions, both sweep orders, every boundary
condition, ragged and small grids, batches, CUDA graphs, the FP32
near-vacuum second pass, checkpoint/resume across the buffer it leaves the
state in, and the bounded-wait failure path."""
import numpy as np
import pytest

import oracle as O
from paper_2106_13465_gb300 import hydro as H
from paper_2106_13465_gb300 import problems as pr

pytestmark = pytest.mark.gpu

P_, T_, R_ = pr.PERIODIC, pr.TRANSMISSIVE, pr.REFLECT
TOL64 = 1e-11


def run(pbs, nsteps, precision, fused, graph_steps=20, dt_override=None, step0=0, **kw):
    grids = [(p.nx, p.ny, p.h, p.bc) for p in pbs]
    with H.Context(grids, precision=precision, **kw) as c:
        c.set_tuning(graph_steps=graph_steps, fused=fused)
        for g, p in enumerate(pbs):
            c.set_state(g, p.U)
        if step0:
            c.set_step(step0)
        dts = c.step(nsteps, dt_override=dt_override, record_dt=dt_override is None and graph_steps == 0)
        out = [c.get_state(g) for g in range(len(pbs))]
        stats = c.stats()
    return out, dts, stats


def _modes(nx, ny, bc, seed):
    pb = pr.random_modes(nx, ny, seed=seed)
    pb.bc = bc
    return pb


CASES = [
    ("modes_periodic", lambda: _modes(150, 97, (P_,) * 4, 1)),
    ("modes_mixed", lambda: _modes(121, 66, (R_, T_, P_, P_), 2)),
    ("modes_mixed2", lambda: _modes(61, 35, (P_, P_, T_, R_), 3)),
    ("sedov", lambda: pr.sedov(130, 70)),
    ("sod_x", lambda: pr.sod(300, 9, 0)),
    ("sod_y", lambda: pr.sod(9, 300, 1)),
    ("tiny_periodic", lambda: _modes(2, 3, (P_,) * 4, 4)),
    ("tiny_reflect", lambda: _modes(3, 2, (R_,) * 4, 5)),
    ("edge_widths", lambda: _modes(62, 33, (T_, T_, P_, P_), 6)),
]


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fused_step_bit_identical_to_split_sweeps(name, make, precision):
    pb = make()
    for step0 in (0, 1):  # both sweep orders first
        split, _, _ = run([pb], 7, precision, fused=0, graph_steps=0, step0=step0)
        fused, _, st = run([pb], 7, precision, fused=1, graph_steps=0, step0=step0)
        assert np.array_equal(fused[0], split[0]), (name, step0)
        assert st["status_flags"] == 0


def test_fused_fp64_matches_oracle_and_dt():
    pb = _modes(130, 90, (R_, R_, P_, P_), 9)
    want, odts, _ = O.run(pb.U, pb.h, pb.bc, 10)
    got, dts, _ = run([pb], 10, 64, fused=1, graph_steps=0)
    np.testing.assert_allclose(dts[:, 0], odts, rtol=1e-12)
    d = np.abs(got[0] - want)
    scale = np.abs(want).reshape(4, -1).max(axis=1)[:, None, None]
    floor = np.array([0.0, 1e-3, 1e-3, 0.0])[:, None, None] * scale
    assert float(np.max(d / np.maximum(np.abs(want), floor))) <= TOL64


@pytest.mark.parametrize("precision", [64, 32])
def test_fused_batch_graph_and_odd_step_counts(precision):
    """A ragged batch through CUDA graphs and single steps (the state moves
    between the two buffers every fused step)."""
    pbs = pr.batch(9, seed=5, lo=8, hi=130)
    ref, _, _ = run(pbs, 23, precision, fused=0, graph_steps=0)
    for gs in (0, 2, 20):
        got, _, st = run(pbs, 23, precision, fused=1, graph_steps=gs)
        for g in range(len(pbs)):
            assert np.array_equal(got[g], ref[g]), (gs, g)
        assert st["status_flags"] == 0


def test_fused_switching_and_checkpoint_resume():
    """Fused and split steps interleaved on one context, and a resume from
    a state taken after an odd number of fused steps."""
    pb = _modes(97, 64, (P_, P_, R_, R_), 11)
    ref, _, _ = run([pb], 12, 64, fused=0, graph_steps=0)
    with H.Context([(pb.nx, pb.ny, pb.h, pb.bc)], precision=64) as c:
        c.set_state(0, pb.U)
        c.set_tuning(graph_steps=0, fused=1)
        c.step(3)
        c.set_tuning(graph_steps=20, fused=0)
        c.step(4)
        c.set_tuning(graph_steps=2, fused=1)
        c.step(5)
        assert np.array_equal(c.get_state(0), ref[0])
        s = c.conservation(0)
    assert np.allclose(s, O.conservation(ref[0], pb.h), rtol=1e-14, atol=1e-16)
    with H.Context([(pb.nx, pb.ny, pb.h, pb.bc)], precision=64) as c:
        c.set_tuning(graph_steps=0, fused=1)
        c.set_state(0, pb.U)
        c.step(5)
        snap, step, t = c.get_state(0), c.get_step(), c.time(0)
    with H.Context([(pb.nx, pb.ny, pb.h, pb.bc)], precision=64) as c:
        c.set_tuning(graph_steps=0, fused=1)
        c.set_state(0, snap)
        c.set_step(step)
        c.set_time(0, t)
        c.step(7)
        assert np.array_equal(c.get_state(0), ref[0])


def test_fused_fp32_near_vacuum_second_pass():
    x = (np.arange(64) + 0.5) / 64
    u = np.where(x < 0.5, -2.0, 2.0)
    U = pr.conserved(np.ones((40, 64)), np.tile(u, (40, 1)), 0.0, 0.4)
    pb = pr.Problem("123", U, 1.0 / 64, (T_,) * 4)
    dts = np.full((5, 1), 0.2 / 64)
    split, _, s1 = run([pb], 5, 32, fused=0, graph_steps=0, dt_override=dts)
    fused, _, s2 = run([pb], 5, 32, fused=1, graph_steps=0, dt_override=dts)
    assert s1["riemann_fp64"] > 0 and s2["riemann_fp64"] > 0
    assert np.array_equal(fused[0], split[0])


@pytest.mark.parametrize("precision,per_step", [(64, 3), (32, 3)])
def test_fused_launch_count(precision, per_step):
    pb = pr.sedov(64, 48)
    with H.Context([(pb.nx, pb.ny, pb.h, pb.bc)], precision=precision) as c:
        c.set_tuning(fused=1)
        c.set_state(0, pb.U)
        n0 = c.stats()["kernel_launches"]
        c.step(3)
        c.step(40)
        assert c.stats()["kernel_launches"] - n0 == 43 * per_step


def test_fused_timeout_status():
    pb = _modes(96, 64, (P_,) * 4, 12)
    ref, _, _ = run([pb], 4, 64, fused=0, graph_steps=0)
    with H.Context([(pb.nx, pb.ny, pb.h, pb.bc)], precision=64) as c:
        c.set_tuning(graph_steps=0, fused=1)
        c.set_state(0, pb.U)
        c.set_wait_limit(0)
        with pytest.raises(H.HydroError) as e:
            c.step(1)
        assert e.value.status == H.HYDRO_ETIMEOUT
        c.set_wait_limit(-1)
        c.set_state(0, pb.U)
        c.step(4)
        assert np.array_equal(c.get_state(0), ref[0])
