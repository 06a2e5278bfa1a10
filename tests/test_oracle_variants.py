"""Pins of the scheme variants (the HYDRO options the paper leaves to its
ref. [5]): the two-shock approximate Riemann solver and the monotonized
central and first-order (no) slopes.  Each is pinned to a closed form or a
textbook scheme, not to a copy of its own formula."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2106_13465_gb300 import problems as pr

G = 1.4
TS = O.params(riemann=O.RIEMANN_TWO_SHOCK)


@pytest.mark.parametrize("rho,p0,U", [(1.0, 1.0, 0.5), (0.3, 2.0, 1.0), (2.0, 0.01, 0.02)])
def test_two_shock_separating_streams_closed_form(rho, p0, U):
    """Separating equal states (rho, -U, p0) | (rho, +U, p0) under the
    two-shock approximation: both waves follow the shock relation, so
    f(p*) = -U with f = (p - p0) sqrt(A/(p + B)): the negative root
    x = (U^2 - sqrt(U^4 + 4 A U^2 (B + p0)))/(2A) of A x^2 - U^2 x -
    U^2 (B + p0) = 0, x = p* - p0, A = 2/((g+1) rho), B = (g-1)/(g+1) p0;
    u* = 0.  The exact solver's two-rarefaction p* differs."""
    A = 2 / ((G + 1) * rho)
    B = (G - 1) / (G + 1) * p0
    x = (U * U - math.sqrt(U ** 4 + 4 * A * U * U * (B + p0))) / (2 * A)
    wl, wr = [rho, -U, 0.0, p0], [rho, U, 0.0, p0]
    ps, us = O.riemann_star(wl, wr, TS)
    assert ps == pytest.approx(p0 + x, rel=1e-13)
    assert us == 0.0
    pe, _ = O.riemann_star(wl, wr)
    assert abs(pe - ps) > 1e-6 * p0


@pytest.mark.parametrize("wl,wr", [
    ([1.0, 1.0, 0.0, 1.0], [1.0, -1.0, 0.0, 1.0]),
    ([2.0, 0.7, 0.3, 0.5], [0.4, -0.9, -0.2, 0.8]),
])
def test_two_shock_equals_exact_when_both_waves_are_shocks(wl, wr):
    ps, us = O.riemann_star(wl, wr)
    assert ps > max(wl[3], wr[3])
    assert O.riemann_star(wl, wr, TS) == (ps, us)
    np.testing.assert_array_equal(O.interface_flux(wl, wr, TS), O.interface_flux(wl, wr))


def test_two_shock_galilean_invariance_and_mirror_symmetry():
    wl, wr = [1.0, 0.0, 0.1, 1.0], [0.125, 0.0, -0.3, 0.1]   # Sod: a left rarefaction
    ps, us = O.riemann_star(wl, wr, TS)
    pe, _ = O.riemann_star(wl, wr)
    assert abs(ps - pe) > 1e-4                       # the approximation is active
    s = 0.37
    ps2, us2 = O.riemann_star([1.0, s, 0.1, 1.0], [0.125, s, -0.3, 0.1], TS)
    assert ps2 == pytest.approx(ps, rel=1e-12) and us2 == pytest.approx(us + s, rel=1e-12)
    pm, um = O.riemann_star([0.125, 0.0, -0.3, 0.1], [1.0, 0.0, 0.1, 1.0], TS)
    assert pm == pytest.approx(ps, rel=1e-14) and um == pytest.approx(-us, rel=1e-14)


@pytest.mark.parametrize("a,b,want", [
    (1.0, 3.0, 2.0),      # 2a
    (1.0, 1.5, 1.25),     # (a + b)/2
    (3.0, 1.0, 2.0),      # 2b
    (-1.0, -5.0, -2.0),
    (2.0, 2.0, 2.0),      # a linear profile keeps its exact slope
    (1.0, -1.0, 0.0),     # an extremum
    (0.0, 4.0, 0.0),
])
def test_mc_slope_values(a, b, want):
    """Monotonized central slope: the smallest in magnitude of 2a, 2b and
    (a + b)/2 when a and b share a sign, else 0.  Seen through the trace at
    u = 0 (no predictor): the face difference WR - WL is the slope."""
    P = O.params(slope=O.SLOPE_MC)
    wm, w0, wp = [10.0, 0.0, 0.0, 1.0], [10.0 + a, 0.0, 0.0, 1.0], [10.0 + a + b, 0.0, 0.0, 1.0]
    wl, wr = O.trace(0.3, wm, w0, wp, P)
    assert wr[0] - wl[0] == pytest.approx(want, abs=1e-15)


def test_no_slope_faces_are_the_cell():
    P = O.params(slope=O.SLOPE_NONE)
    wl, wr = O.trace(0.3, [1.0, 0.2, 0.1, 1.0], [1.2, 0.3, 0.1, 1.1], [1.5, 0.1, 0.0, 0.7], P)
    np.testing.assert_array_equal(wl, [1.2, 0.3, 0.1, 1.1])
    np.testing.assert_array_equal(wr, [1.2, 0.3, 0.1, 1.1])


def _scalar_scheme(q, nu, nsteps, slope):
    """Textbook scalar MUSCL-Hancock for q_t + a q_x = 0, a > 0, periodic:
    face q + (1 - nu)/2 s with s the limited slope (mc, or 0: the
    first-order upwind scheme q_i - nu (q_i - q_{i-1}))."""
    for _ in range(nsteps):
        dm = q - np.roll(q, 1)
        dp = np.roll(q, -1) - q
        if slope == "none":
            s = np.zeros_like(q)
        else:
            c = 0.5 * (dm + dp)
            m = np.minimum(np.minimum(np.abs(2 * dm), np.abs(2 * dp)), np.abs(c))
            s = np.where(dm * dp > 0, np.sign(dm) * m, 0.0)
        face = q + 0.5 * (1.0 - nu) * s
        q = q - nu * (face - np.roll(face, 1))
    return q


@pytest.mark.parametrize("slope,code,rtol", [("mc", O.SLOPE_MC, 2e-14), ("none", O.SLOPE_NONE, 2e-14)])
def test_contact_advection_reduces_to_the_scalar_scheme(slope, code, rtol):
    n, a, p0 = 64, 0.6, 1.0
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x) + 0.2 * (np.abs(x - 0.3) < 0.1)
    U = pr.conserved(np.tile(rho, (2, 1)), a, 0.0, p0)
    h = 1.0 / n
    dt = 0.8 * h / (a + math.sqrt(G * p0 / rho.min()))
    nu = a * dt / h
    out, _, _ = O.run(U, h, (pr.PERIODIC,) * 4, 20, dt_override=[dt] * 20, P=O.params(slope=code))
    assert np.allclose(out[0, 0], _scalar_scheme(rho, nu, 20, slope), rtol=rtol, atol=0)


def test_first_order_scheme_converges_at_first_order_on_smooth_flow():
    """Self-convergence of a smooth periodic flow: errors against the next
    finer grid fall by ~2 per refinement with no slopes (first order) and by
    ~4 with MC slopes (second order)."""
    def solve(n, slope, t=0.05):
        x = (np.arange(n) + 0.5) / n
        rho = 1.0 + 0.2 * np.sin(2 * np.pi * x)
        U = pr.conserved(np.tile(rho, (2, 1)), 0.5, 0.0, 1.0)
        h = 1.0 / n
        steps = 4 * n // 32
        dt = t / steps
        out, _, _ = O.run(U, h, (pr.PERIODIC,) * 4, steps, dt_override=[dt] * steps, P=O.params(slope=slope))
        return out[0, 0]

    for slope, lo, hi in [(O.SLOPE_NONE, 1.7, 2.3), (O.SLOPE_MC, 3.2, 5.0)]:
        errs = []
        for n in (64, 128, 256):
            c, f = solve(n, slope), solve(2 * n, slope)
            errs.append(np.abs(c - 0.5 * (f[0::2] + f[1::2])).mean())
        ratios = [errs[i] / errs[i + 1] for i in range(2)]
        assert all(lo < r < hi for r in ratios), (slope, ratios)


# ---- characteristic tracing ----------------------------------------------
CH = O.params(trace=O.TRACE_CHARACTERISTIC)


def _c_of(w):
    return math.sqrt(G * w[3] / w[0])


@pytest.mark.parametrize("sgn", [1.0, -1.0])
def test_characteristic_trace_supersonic_keeps_all_waves_on_one_face(sgn):
    """Flow faster than sound: every wave moves the same way, so the downwind
    face is the full MUSCL-Hancock face and the upwind face is the cell
    state itself (the wave split of the slopes recombines them)."""
    c = _c_of([1.0, 0.0, 0.0, 1.0])
    u = sgn * 2.5 * c
    wm, w0, wp = [0.9, u - 0.02, 0.1, 0.95], [1.0, u, 0.12, 1.0], [1.08, u + 0.03, 0.15, 1.07]
    wl, wr = O.trace(0.2, wm, w0, wp, CH)
    ml, mr = O.trace(0.2, wm, w0, wp)
    if sgn > 0:
        np.testing.assert_array_equal(wl, w0)
        np.testing.assert_allclose(wr, mr, rtol=1e-13, atol=1e-15)
    else:
        np.testing.assert_array_equal(wr, w0)
        np.testing.assert_allclose(wl, ml, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("wave", [1, 4])
def test_characteristic_trace_of_a_simple_acoustic_slope(wave):
    """Subsonic flow (0 < u < c) with the slope along one acoustic
    eigenvector r = (1, -+c/rho, 0, c^2) of amplitude e: the u + c wave reaches
    only the right face, W + (1 - (u + c) dt/dx)/2 e r4; the u - c wave only
    the left one, W - (1 + (u - c) dt/dx)/2 e r1."""
    rho, u, p = 1.0, 0.3, 1.0
    c = math.sqrt(G * p / rho)
    e, dtdx = 1e-3, 0.25
    s = 1.0 if wave == 4 else -1.0
    r = np.array([1.0, s * c / rho, 0.0, c * c])
    w0 = np.array([rho, u, 0.0, p])
    wl, wr = O.trace(dtdx, w0 - e * r, w0, w0 + e * r, CH)
    lam = u + s * c
    if wave == 4:
        np.testing.assert_allclose(wr, w0 + 0.5 * (1 - lam * dtdx) * e * r, rtol=1e-13)
        np.testing.assert_allclose(wl, w0, rtol=1e-13)
    else:
        np.testing.assert_allclose(wl, w0 - 0.5 * (1 + lam * dtdx) * e * r, rtol=1e-13)
        np.testing.assert_allclose(wr, w0, rtol=1e-13)


def test_characteristic_trace_contact_reduces_to_the_scalar_scheme():
    """A contact carried at u > 0 through uniform pressure: only the entropy
    wave moves, toward the right face, so the scheme is the textbook scalar
    minmod MUSCL-Hancock scheme again."""
    n, a, p0 = 64, 0.6, 1.0
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x) + 0.2 * (np.abs(x - 0.3) < 0.1)
    U = pr.conserved(np.tile(rho, (2, 1)), a, 0.0, p0)
    h = 1.0 / n
    dt = 0.8 * h / (a + math.sqrt(G * p0 / rho.min()))
    nu = a * dt / h
    out, _, _ = O.run(U, h, (pr.PERIODIC,) * 4, 20, dt_override=[dt] * 20, P=CH)

    q = rho.copy()
    for _ in range(20):
        dm = q - np.roll(q, 1)
        dp = np.roll(q, -1) - q
        s = np.where(dm * dp > 0, np.where(np.abs(dm) < np.abs(dp), dm, dp), 0.0)
        face = q + 0.5 * (1.0 - nu) * s
        q = q - nu * (face - np.roll(face, 1))
    assert np.allclose(out[0, 0], q, rtol=2e-14, atol=0)


def test_characteristic_trace_sod_converges():
    """The Sod problem with characteristic tracing approaches the exact
    profile as the grid is refined (L1 error of density falls)."""
    wl, wr = [1.0, 0.0, 0.0, 1.0], [0.125, 0.0, 0.0, 0.1]
    errs = []
    for n in (64, 128, 256):
        pb = pr.sod(n, 2, 0)
        t, k, U = 0.0, 0, pb.U.copy()
        while t < 0.2 * (1 - 1e-14):
            dt = min(O.cfl_dt(U, pb.h, CH), 0.2 - t)
            U, _, _ = O.run(U, pb.h, pb.bc, 1, step0=k, dt_override=[dt], P=CH)
            t += dt
            k += 1
        x = (np.arange(n) + 0.5) / n - 0.5
        ps, us = O.riemann_star(wl, wr)
        exact = np.array([O.sample(wl, wr, ps, us, xi / 0.2)[0] for xi in x])
        errs.append(np.abs(U[0, 0] - exact).mean())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.012
