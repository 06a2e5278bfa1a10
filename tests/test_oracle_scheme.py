"""Pins of the oracle's full scheme (§1, Figs. 1-2, Fig. 5) against properties
the mathematics fixes: uniform states are preserved exactly, periodic runs
conserve mass/momentum/energy, reflective walls equal a mirrored periodic
domain, the result commutes with transposition and with periodic shifts, one
sweep reaches exactly two cells along its axis, a pure contact reduces to the
scalar minmod MUSCL-Hancock scheme, and the Sod tube converges to the exact
solution while smooth flow converges at second order."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2106_13465_gb300 import problems as pr

G = 1.4
P, T, R = pr.PERIODIC, pr.TRANSMISSIVE, pr.REFLECT


@pytest.mark.parametrize("bc,u,v", [((P,) * 4, 0.3, -0.7), ((T,) * 4, -0.4, 0.2),
                                    ((R,) * 4, 0.0, 0.0), ((P, P, T, T), 0.5, 0.0),
                                    ((R, R, P, P), 0.0, 0.6)])
def test_uniform_state_preserved_bit_exact(bc, u, v):
    pb = pr.uniform(13, 7, rho=0.8, u=u, v=v, p=1.7, bc=bc)
    U, dts, _ = O.run(pb.U, pb.h, pb.bc, 6)
    assert np.array_equal(U, pb.U)
    c = math.sqrt(G * 1.7 / 0.8)
    assert dts[0] == pytest.approx(0.8 * pb.h / (max(abs(u), abs(v)) + c), rel=1e-15)


def test_conservation_periodic_random_modes():
    pb = pr.random_modes(48, 40)
    s0 = O.conservation(pb.U, pb.h)
    U, _, _ = O.run(pb.U, pb.h, pb.bc, 12)
    s1 = O.conservation(U, pb.h)
    scale = np.abs(pb.U).sum(axis=(1, 2)) * pb.h * pb.h
    assert np.all(np.abs(s1 - s0) <= 1e-14 * scale)


def test_conservation_reflective_sedov_mass_and_energy():
    pb = pr.sedov(32)
    s0 = O.conservation(pb.U, pb.h)
    U, _, _ = O.run(pb.U, pb.h, pb.bc, 25)
    s1 = O.conservation(U, pb.h)
    tol = 25 * 8 * np.finfo(float).eps           # round-off of 25 steps
    assert abs(s1[0] - s0[0]) <= tol * s0[0]
    assert abs(s1[3] - s0[3]) <= tol * s0[3]
    assert not np.array_equal(U, pb.U)


def test_reflective_wall_equals_mirrored_periodic_domain():
    """A box with reflective x walls evolves exactly like the periodic box of
    twice the width that holds the state and its mirror image (normal
    momentum negated)."""
    rng = np.random.default_rng(7)
    nx, ny = 10, 6
    rho = 1 + 0.3 * rng.random((ny, nx))
    u = 0.4 * rng.standard_normal((ny, nx))
    v = 0.4 * rng.standard_normal((ny, nx))
    p = 1 + 0.5 * rng.random((ny, nx))
    U = pr.conserved(rho, u, v, p)
    M = np.concatenate([U, U[:, :, ::-1]], axis=2).copy()
    M[1, :, nx:] *= -1.0
    h = 1.0 / 20
    a, _, _ = O.run(U, h, (R, R, P, P), 8)
    b, _, _ = O.run(M, h, (P, P, P, P), 8)
    assert np.array_equal(a, b[:, :, :nx])


def test_transmissive_ends_do_not_disturb_the_interior_early_on():
    """Before any wave reaches an end, a Sod tube in a short transmissive
    domain equals the same tube embedded in a longer one."""
    short = pr.sod(64, 2, 0)
    long_U = np.concatenate([np.repeat(short.U[:, :, :1], 32, axis=2), short.U,
                             np.repeat(short.U[:, :, -1:], 32, axis=2)], axis=2)
    dt = 0.2 * short.h
    a, _, _ = O.run(short.U, short.h, short.bc, 6, dt_override=[dt] * 6)
    b, _, _ = O.run(long_U, short.h, short.bc, 6, dt_override=[dt] * 6)
    assert np.array_equal(a, b[:, :, 32:96])


def test_transpose_symmetry_bit_exact():
    pb = pr.random_modes(20, 14, seed=11)
    pb.bc = (P, P, R, R)
    t = pr.transpose(pb)
    a, da, _ = O.run(pb.U, pb.h, pb.bc, 7, step0=0)
    b, db, _ = O.run(t.U, t.h, t.bc, 7, step0=1)
    assert np.array_equal(da, db)
    at = pr.transpose(pr.Problem("a", a, pb.h, pb.bc)).U
    assert np.array_equal(at, b)


def test_periodic_shift_invariance_bit_exact():
    pb = pr.random_modes(16, 12, seed=5)
    a, _, _ = O.run(pb.U, pb.h, pb.bc, 5)
    s = np.roll(np.roll(pb.U, 5, axis=2), -3, axis=1)
    b, _, _ = O.run(s, pb.h, pb.bc, 5)
    assert np.array_equal(np.roll(np.roll(a, 5, axis=2), -3, axis=1), b)


@pytest.mark.parametrize("direction", [0, 1])
def test_single_sweep_footprint_is_two_cells(direction):
    """Figs. 1-2: after one sweep a cell depends on cells i-2..i+2 of its line
    only; a one-cell perturbation changes nothing further away."""
    pb = pr.random_modes(24, 24, seed=3)
    dt = 0.3 * pb.h
    base = O.sweep(pb.U, pb.h, pb.bc, direction, dt)
    U = pb.U.copy()
    i0, j0 = 11, 9
    U[0, j0, i0] *= 1.05
    U[3, j0, i0] *= 1.03
    pert = O.sweep(U, pb.h, pb.bc, direction, dt)
    diff = np.any(pert != base, axis=0)
    jj, ii = np.nonzero(diff)
    along, across, c0, c1 = (ii, jj, i0, j0) if direction == 0 else (jj, ii, j0, i0)
    assert set(across) == {c1}
    assert set(along) <= set(range(c0 - 2, c0 + 3))
    assert {c0 - 1, c0, c0 + 1} <= set(along)


def _scalar_muscl_hancock(q, nu, nsteps):
    """Textbook MUSCL-Hancock for q_t + a q_x = 0, a > 0, periodic, minmod
    slopes, Courant number nu: face value q_i + (1 - nu)/2 * minmod(...)."""
    q = q.copy()
    for _ in range(nsteps):
        dm = q - np.roll(q, 1)
        dp = np.roll(q, -1) - q
        s = np.where(dm * dp > 0, np.where(np.abs(dm) < np.abs(dp), dm, dp), 0.0)
        face = q + 0.5 * (1.0 - nu) * s
        q = q - nu * (face - np.roll(face, 1))
    return q


def test_contact_advection_reduces_to_scalar_muscl_hancock():
    n, a, p0 = 64, 0.6, 1.0
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x) + 0.2 * (np.abs(x - 0.3) < 0.1)
    U = pr.conserved(np.tile(rho, (2, 1)), a, 0.0, p0)
    h = 1.0 / n
    cmax = math.sqrt(G * p0 / rho.min())
    dt = 0.8 * h / (a + cmax)                   # acoustic CFL limit
    nu = a * dt / h
    out, _, _ = O.run(U, h, (P,) * 4, 20, dt_override=[dt] * 20)
    want = _scalar_muscl_hancock(rho, nu, 20)
    assert np.allclose(out[0, 0], want, rtol=2e-14, atol=0)
    assert np.allclose(out[1, 0] / out[0, 0], a, rtol=1e-13)
    pr_ = (G - 1) * (out[3, 0] - 0.5 * out[1, 0] ** 2 / out[0, 0])
    assert np.allclose(pr_, p0, rtol=1e-12)


def _advance_to(U, h, bc, t_end):
    """CFL steps with the last one shortened to land on t_end exactly."""
    t, k = 0.0, 0
    while t < t_end * (1 - 1e-14):
        dt = O.cfl_dt(U, h)
        if t + dt > t_end:
            dt = t_end - t
        U, _, _ = O.run(U, h, bc, 1, step0=k, dt_override=[dt])
        t += dt
        k += 1
    return U


def test_sod_converges_to_exact_solution():
    wl, wr = [1.0, 0.0, 0.0, 1.0], [0.125, 0.0, 0.0, 0.1]
    ps, us = O.riemann_star(wl, wr)
    errs = []
    for n in (64, 128, 256, 512):
        pb = pr.sod(n, 2, 0)
        U = _advance_to(pb.U, pb.h, pb.bc, 0.2)
        x = (np.arange(n) + 0.5) / n
        exact = np.array([O.sample(wl, wr, ps, us, (xi - 0.5) / 0.2)[0] for xi in x])
        errs.append(np.sum(np.abs(U[0, 0] - exact)) / n)
        assert np.array_equal(U[:, 0], U[:, 1])          # the y sweep is a no-op
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert errs[0] < 0.02
    assert all(r > 0.55 for r in rates), (errs, rates)


def test_smooth_flow_self_convergence_second_order():
    """Smooth periodic 1D flow before any shock forms: the difference between
    successive resolutions falls by about 4x per refinement."""
    sols = []
    for n in (32, 64, 128, 256):
        x = (np.arange(n) + 0.5) / n
        rho = 1 + 0.2 * np.sin(2 * np.pi * x)
        u = 0.3 + 0.05 * np.sin(2 * np.pi * x)
        p = 1 + 0.1 * np.cos(2 * np.pi * x)
        U = pr.conserved(np.tile(rho, (2, 1)), np.tile(u, (2, 1)), 0.0, np.tile(p, (2, 1)))
        sols.append(_advance_to(U, 1.0 / n, (P,) * 4, 0.1)[:, 0])
    diffs = []
    for a, b in zip(sols[:-1], sols[1:]):
        coarse = 0.5 * (b[:, 0::2] + b[:, 1::2])
        diffs.append(np.abs(a - coarse).mean())
    orders = [math.log2(diffs[i] / diffs[i + 1]) for i in range(len(diffs) - 1)]
    assert all(o > 1.6 for o in orders), (diffs, orders)


def test_cfl_dt_takes_the_fastest_cell():
    U = pr.conserved(np.ones((3, 4)), 0.0, 0.0, 1.0)
    U2 = U.copy()
    U2[:, 1, 2] = pr.conserved(np.array([[0.5]]), 0.0, -2.0, 3.0)[:, 0, 0]
    h = 0.25
    fast = 2.0 + math.sqrt(G * 3.0 / 0.5)
    assert O.cfl_dt(U2, h) == pytest.approx(0.8 * h / fast, rel=1e-15)
    assert O.cfl_dt(U, h) == pytest.approx(0.8 * h / math.sqrt(G), rel=1e-15)


def test_conservation_sums_of_uniform_state():
    pb = pr.uniform(8, 4, rho=2.0, u=0.5, v=-1.0, p=3.0)
    s = O.conservation(pb.U, pb.h)
    area = 8 * 4 * pb.h * pb.h
    E = 3.0 / (G - 1) + 0.5 * 2.0 * (0.25 + 1.0)
    assert np.allclose(s, [2.0 * area, 1.0 * area, -2.0 * area, E * area], rtol=1e-15)


def test_negative_density_reported():
    pb = pr.sod(16, 2, 0)
    U = pb.U.copy()
    U[0, 0, 3] = np.nan
    _, _, rc = O.run(U, pb.h, pb.bc, 1, check=False)
    assert rc == 4


def test_even_steps_sweep_x_first_odd_steps_y_first():
    """Sweep order alternates: step k even runs x then y, odd runs y then x;
    both sweeps of a step use the dt of the state at the start of the step."""
    pb = pr.random_modes(12, 10, seed=9)
    dt = O.cfl_dt(pb.U, pb.h)
    want = O.sweep(O.sweep(pb.U, pb.h, pb.bc, 0, dt), pb.h, pb.bc, 1, dt)
    got, dts, _ = O.run(pb.U, pb.h, pb.bc, 1, step0=0)
    assert dts[0] == dt and np.array_equal(got, want)
    want = O.sweep(O.sweep(pb.U, pb.h, pb.bc, 1, dt), pb.h, pb.bc, 0, dt)
    got, _, _ = O.run(pb.U, pb.h, pb.bc, 1, step0=1)
    assert np.array_equal(got, want)
