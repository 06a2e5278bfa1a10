"""Scheme variants on the GPU (hydro_params.riemann_solver, slope_type,
trace_type): the two-shock approximate Riemann solver, the monotonized
central and first-order slopes and characteristic tracing, each against the oracle run with the same variant, in
FP64 to the parity tolerance, and FP32 to a stated density error; the fused
step kernel gives the split sweeps' bits with a variant too."""
import numpy as np
import pytest

import oracle as O
from paper_2106_13465_gb300 import hydro as H
from paper_2106_13465_gb300 import problems as pr

pytestmark = pytest.mark.gpu

T_ = pr.TRANSMISSIVE
TOL64 = 1e-11
VARIANTS = [
    ("two_shock", H.RIEMANN_TWO_SHOCK, H.SLOPE_MINMOD, H.TRACE_MUSCL_HANCOCK),
    ("mc", H.RIEMANN_EXACT, H.SLOPE_MC, H.TRACE_MUSCL_HANCOCK),
    ("first_order", H.RIEMANN_EXACT, H.SLOPE_NONE, H.TRACE_MUSCL_HANCOCK),
    ("two_shock_mc", H.RIEMANN_TWO_SHOCK, H.SLOPE_MC, H.TRACE_MUSCL_HANCOCK),
    ("characteristic", H.RIEMANN_EXACT, H.SLOPE_MINMOD, H.TRACE_CHARACTERISTIC),
    ("characteristic_mc", H.RIEMANN_EXACT, H.SLOPE_MC, H.TRACE_CHARACTERISTIC),
]


def rel_err(a, b):
    worst = 0.0
    for q in range(4):
        den = np.abs(b[q])
        if q in (1, 2):
            den = np.maximum(den, 1e-3 * den.max())
        den = np.where(den > 0, den, 1.0)
        worst = max(worst, float((np.abs(a[q] - b[q]) / den).max()))
    return worst


def _vacuum_pair(n=64, ny=4):
    x = (np.arange(n) + 0.5) / n
    u = np.where(x < 0.5, -1.5, 1.5)
    U = pr.conserved(np.ones((ny, n)), np.tile(u, (ny, 1)), 0.0, 0.4)
    return pr.Problem("separating", U, 1.0 / n, (T_,) * 4)


CASES = [lambda: pr.sedov(96, 80), lambda: pr.random_modes(128, 90, seed=7), lambda: pr.sod(200, 4, 0),
         lambda: _vacuum_pair()]


@pytest.mark.parametrize("name,riemann,slope,trace", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_variant_fp64_matches_oracle(name, riemann, slope, trace):
    for make in CASES:
        pb = make()
        want, odts, _ = O.run(pb.U, pb.h, pb.bc, 10, P=O.params(riemann=riemann, slope=slope, trace=trace))
        with H.Context([(pb.nx, pb.ny, pb.h, pb.bc)], precision=64, riemann=riemann, slope=slope,
                       trace=trace) as c:
            c.set_state(0, pb.U)
            dts = c.step(10, record_dt=True)
            got = c.get_state(0)
        assert rel_err(got, want) <= TOL64, (name, pb.name)
        np.testing.assert_allclose(dts[:, 0], odts, rtol=1e-12)
        # the variant is active: the default scheme gives another state
        base, _, _ = O.run(pb.U, pb.h, pb.bc, 10, dt_override=odts)
        assert not np.array_equal(base, want), (name, pb.name)


@pytest.mark.parametrize("name,riemann,slope,trace", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_variant_fp32_density_error_and_fused(name, riemann, slope, trace):
    pb = pr.random_modes(128, 90, seed=7)
    ref, dts, _ = O.run(pb.U, pb.h, pb.bc, 10, P=O.params(riemann=riemann, slope=slope, trace=trace))
    outs = {}
    for fused in (0, 1):
        with H.Context([(pb.nx, pb.ny, pb.h, pb.bc)], precision=32, riemann=riemann, slope=slope,
                       trace=trace) as c:
            c.set_tuning(fused=fused, graph_steps=0)
            c.set_state(0, pb.U)
            c.step(10, dt_override=dts)
            outs[fused] = c.get_state(0)
    assert np.array_equal(outs[0], outs[1])
    l1 = np.abs(outs[0][0] - ref[0]).sum() / np.abs(ref[0]).sum()
    assert l1 < 5e-7, (name, l1)


def test_variant_arguments_checked():
    p, _arr = H.make_params([(16, 16, 1 / 16, (0, 0, 0, 0))], riemann=2)
    assert H.hydro_init(p)[0] == H.HYDRO_EINVAL
    p, _arr = H.make_params([(16, 16, 1 / 16, (0, 0, 0, 0))], slope=3)
    assert H.hydro_init(p)[0] == H.HYDRO_EINVAL
    p, _arr = H.make_params([(16, 16, 1 / 16, (0, 0, 0, 0))], trace=2)
    assert H.hydro_init(p)[0] == H.HYDRO_EINVAL
