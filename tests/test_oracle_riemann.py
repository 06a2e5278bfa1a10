"""Pins of the oracle's exact Riemann solver and sampler (§1: fluxes from a
Riemann solver at every interface) against facts that do not come from the
oracle's own code: the tabulated Sod star state, closed forms of the pressure
equation for two rarefactions and for two symmetric shocks, the
Rankine-Hugoniot jump conditions, the fan invariants and exact symmetries."""
import math
import os

import numpy as np
import pytest

import oracle as O

G = 1.4
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sod_star.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def _c(w):
    return math.sqrt(G * w[3] / w[0])


def test_sod_star_state_matches_tabulated_values():
    g = _golden()
    ps, us = O.riemann_star([1.0, 0.0, 0.0, 1.0], [0.125, 0.0, 0.0, 0.1])
    assert abs(ps - g["pstar"]) <= 5e-6
    assert abs(us - g["ustar"]) <= 5e-6


@pytest.mark.parametrize("wl,wr", [
    ([1.0, -0.5, 0.0, 1.0], [1.0, 0.5, 0.0, 1.0]),
    ([1.0, -0.8, 0.2, 2.0], [0.5, 0.9, -0.1, 0.7]),
    ([3.0, 0.1, 0.0, 5.0], [2.0, 0.9, 1.0, 4.0]),
])
def test_two_rarefaction_closed_form(wl, wr):
    """With p* below both p_L and p_R, f_L + f_R + du = 0 has the closed form
    p* = [(c_L + c_R - (g-1)/2 du) / (c_L p_L^-z + c_R p_R^-z)]^(1/z),
    z = (g-1)/(2g)."""
    z = (G - 1) / (2 * G)
    cl, cr = _c(wl), _c(wr)
    du = wr[1] - wl[1]
    p_tr = ((cl + cr - 0.5 * (G - 1) * du) / (cl / wl[3] ** z + cr / wr[3] ** z)) ** (1 / z)
    assert p_tr < min(wl[3], wr[3])          # really a two-rarefaction case
    ps, us = O.riemann_star(wl, wr)
    assert ps == pytest.approx(p_tr, rel=1e-13)
    # u* from the left rarefaction's Riemann invariant (independent of f_R)
    u_left = wl[1] - 2 * cl / (G - 1) * ((p_tr / wl[3]) ** z - 1)
    assert us == pytest.approx(u_left, rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("rho,p0,U", [(1.0, 1.0, 1.0), (0.3, 2.0, 4.0), (2.0, 0.01, 0.05)])
def test_symmetric_two_shock_closed_form(rho, p0, U):
    """Colliding equal states (rho, +U, p0) | (rho, -U, p0): both waves are
    shocks with f(p*) = U, i.e. A x^2 - U^2 x - U^2 (B + p0) = 0 for
    x = p* - p0, A = 2/((g+1) rho), B = (g-1)/(g+1) p0; and u* = 0."""
    A = 2 / ((G + 1) * rho)
    B = (G - 1) / (G + 1) * p0
    x = (U * U + math.sqrt(U ** 4 + 4 * A * U * U * (B + p0))) / (2 * A)
    ps, us = O.riemann_star([rho, U, 0.0, p0], [rho, -U, 0.0, p0])
    assert ps == pytest.approx(p0 + x, rel=1e-13)
    assert us == 0.0


def test_equal_states_are_a_fixed_point():
    w = [0.7, 0.3, -0.2, 1.9]
    ps, us = O.riemann_star(w, w)
    assert ps == w[3] and us == w[1]
    s = O.sample(w, w, ps, us, 0.0)
    assert np.array_equal(s, np.array(w))


def test_mirror_states_give_zero_contact_speed():
    wl = [0.9, 0.4, 0.1, 1.3]
    wr = [0.9, -0.4, 0.1, 1.3]
    ps, us = O.riemann_star(wl, wr)
    assert us == 0.0
    wl = [0.9, -0.6, 0.1, 1.3]
    wr = [0.9, 0.6, 0.3, 1.3]
    assert O.riemann_star(wl, wr)[1] == 0.0


@pytest.mark.parametrize("shift", [-1.7, 0.25, 3.0])
def test_galilean_invariance(shift):
    wl, wr = [1.0, 0.0, 0.0, 1.0], [0.125, 0.0, 0.0, 0.1]
    p0, u0 = O.riemann_star(wl, wr)
    p1, u1 = O.riemann_star([1.0, shift, 0.0, 1.0], [0.125, shift, 0.0, 0.1])
    assert p1 == pytest.approx(p0, rel=1e-13)
    assert u1 == pytest.approx(u0 + shift, rel=1e-13)


def _cons_flux_frame(w, S):
    """Mass, momentum and energy fluxes through a surface moving at speed S."""
    rho, u, p = w[0], w[1], w[3]
    E = p / (G - 1) + 0.5 * rho * u * u
    return np.array([rho * (u - S), rho * u * (u - S) + p, E * (u - S) + p * u])


def test_mirrored_sod_is_the_mirror_image():
    """Swapping the two states and reversing the velocities mirrors the
    solution: W(xi) of the swapped problem is W(-xi) of the original with
    the normal velocity negated (exercises the left-shock and right-fan
    branches)."""
    wl, wr = [1.0, 0.0, 0.0, 1.0], [0.125, 0.0, 0.0, 0.1]
    ps, us = O.riemann_star(wl, wr)
    ps2, us2 = O.riemann_star(wr, wl)
    assert ps2 == pytest.approx(ps, rel=1e-14) and us2 == pytest.approx(-us, rel=1e-14)
    for xi in np.linspace(-1.9, 1.9, 77):
        a = O.sample(wl, wr, ps, us, xi)
        b = O.sample(wr, wl, ps2, us2, -xi)
        assert np.allclose([b[0], -b[1], b[3]], [a[0], a[1], a[3]], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("mirror", [False, True])
def test_sod_solution_satisfies_jump_conditions_and_fan_invariants(mirror):
    wl, wr = [1.0, 0.0, 0.0, 1.0], [0.125, 0.0, 0.0, 0.1]
    if mirror:
        # check the left-shock / right-fan branches through the mirror image
        wl, wr = wr, wl
    ps, us = O.riemann_star(wl, wr)
    if mirror:
        # map the mirrored solution back to the original orientation
        def sample_o(a, b, p, u, x, ml=wl, mr=wr, mp=ps, mu=us):
            w = O.sample(ml, mr, mp, mu, -x)
            return np.array([w[0], -w[1], w[2], w[3]])
        wl, wr = wr, wl
        ps, us = ps, -us
    else:
        sample_o = O.sample
    xs = np.linspace(-2.0, 2.0, 40001)
    S = np.array([sample_o(wl, wr, ps, us, x) for x in xs])
    rho = S[:, 0]
    # the right shock: the largest density jump right of the contact
    right = xs > us + 1e-9
    jumps = np.abs(np.diff(rho))
    k = int(np.argmax(np.where(right[1:], jumps, 0.0)))
    a, b = S[k], S[k + 1]                      # behind / ahead of the shock
    s_shock = (a[0] * a[1] - b[0] * b[1]) / (a[0] - b[0])   # from the mass jump
    fa, fb = _cons_flux_frame(a, s_shock), _cons_flux_frame(b, s_shock)
    assert np.allclose(fa, fb, rtol=1e-12, atol=1e-12)
    # across the contact: pressure and normal velocity continuous
    c = int(np.argmin(np.abs(xs - us)))
    lo, hi = S[c - 2], S[c + 2]
    assert lo[3] == pytest.approx(ps, rel=1e-14) and hi[3] == pytest.approx(ps, rel=1e-14)
    assert lo[1] == pytest.approx(us, rel=1e-14) and hi[1] == pytest.approx(us, rel=1e-14)
    assert lo[0] != hi[0]
    # left fan: entropy and the Riemann invariant u + 2c/(g-1) are constant,
    # and on the characteristic x/t = u - c
    cl = _c(wl)
    fan = (xs > -cl + 1e-6) & (xs < us - _c([lo[0], 0, 0, ps]) - 1e-6)
    assert fan.sum() > 100
    for row, x in zip(S[fan][::50], xs[fan][::50]):
        c = _c(row)
        assert row[3] / row[0] ** G == pytest.approx(wl[3] / wl[0] ** G, rel=1e-12)
        assert row[1] + 2 * c / (G - 1) == pytest.approx(2 * cl / (G - 1), rel=1e-12)
        assert row[1] - c == pytest.approx(x, abs=1e-12)


def test_transonic_fan_sampled_at_sonic_point():
    """A left rarefaction straddling x/t = 0: the sampled state is sonic
    (u = c) and isentropic with the left state."""
    wl, wr = [1.0, 0.75, 0.0, 1.0], [0.125, 0.0, 0.0, 0.1]
    ps, us = O.riemann_star(wl, wr)
    cl = _c(wl)
    assert wl[1] - cl < 0 < us - _c([1.0, 0, 0, 1.0]) * (ps / wl[3]) ** ((G - 1) / (2 * G))
    w = O.sample(wl, wr, ps, us, 0.0)
    c = _c(w)
    assert w[1] == pytest.approx(c, rel=1e-13)
    assert w[3] / w[0] ** G == pytest.approx(wl[3] / wl[0] ** G, rel=1e-12)
    assert w[1] + 2 * c / (G - 1) == pytest.approx(wl[1] + 2 * cl / (G - 1), rel=1e-13)


def test_tangential_velocity_follows_the_contact():
    wl, wr = [1.0, 0.2, 0.7, 1.0], [1.0, 0.2, -0.4, 1.0]
    ps, us = O.riemann_star(wl, wr)
    assert us > 0
    assert O.sample(wl, wr, ps, us, 0.0)[2] == 0.7
    wl, wr = [1.0, -0.2, 0.7, 1.0], [1.0, -0.2, -0.4, 1.0]
    ps, us = O.riemann_star(wl, wr)
    assert us < 0
    assert O.sample(wl, wr, ps, us, 0.0)[2] == -0.4


def test_interface_flux_of_a_supersonic_state_is_its_physical_flux():
    """Flow supersonic to the right: the Godunov flux is the left state's
    physical flux (rho u, rho u^2 + p, rho u v, u (E + p))."""
    w = [1.0, 3.0, 0.5, 1.0]
    f = O.interface_flux(w, [0.9, 3.1, 0.4, 1.05])
    E = w[3] / (G - 1) + 0.5 * w[0] * (w[1] ** 2 + w[2] ** 2)
    want = [w[0] * w[1], w[0] * w[1] ** 2 + w[3], w[0] * w[1] * w[2], w[1] * (E + w[3])]
    assert np.allclose(f, want, rtol=1e-15, atol=0)


# ---- floors (density floor, pressure floor p >= rho c_floor^2 / gamma) -----
# Floors of 1e-3 (density) and 0.1 (sound speed) with gamma = 1.4: the
# pressure floor of a state at the density floor is 1e-3 * 0.01 / 1.4.
_FLOORS = dict(rho_floor=1e-3, c_floor=0.1)
_PFLOOR = 7.142857142857143e-06


def test_floors_clamp_the_primitive_state_to_their_magnitudes():
    P = O.params(**_FLOORS)
    # density below its floor, internal energy negative
    W = O.cons_to_prim([1e-4, 2e-4, -3e-4, 1e-9], P)
    assert W[0] == 1e-3
    assert W[1] == pytest.approx(0.2, rel=1e-15) and W[2] == pytest.approx(-0.3, rel=1e-15)
    assert W[3] == pytest.approx(_PFLOOR, rel=1e-15)
    # a pressure above the floor of its density is kept
    W = O.cons_to_prim([2.0, 0.0, 0.0, 1.0], P)
    assert W[3] == pytest.approx(0.4, rel=1e-15)
    # at density 0.5 the floor is 0.5 * 0.01 / 1.4
    W = O.cons_to_prim([0.5, 0.0, 0.0, 1e-12], P)
    assert W[3] == pytest.approx(0.5 * 0.01 / 1.4, rel=1e-15)


def test_trace_faces_clamped_to_the_floors():
    """A steep density drop swept by a fast inflow: the predictor drives both
    face densities negative (rho 1 -+ 0.4995 - 2.4975), so both take the
    density floor and then the pressure floor of that density."""
    P = O.params(**_FLOORS)
    wl, wr = O.trace(0.5, [2.0, -10.0, 0.0, 1e-12], [1.0, -10.0, 0.0, 1e-12],
                     [0.001, -10.0, 0.0, 1e-12], P)
    for w in (wl, wr):
        assert w[0] == 1e-3
        assert w[1] == -10.0 and w[2] == 0.0
        assert w[3] == pytest.approx(_PFLOOR, rel=1e-15)


def test_vacuum_generating_pair_drives_pstar_to_the_floor():
    """Streams leaving each other faster than 2 (cL + cR)/(gamma - 1) open a
    vacuum; the iteration is clamped at the smallest admissible pressure,
    rho_floor c_floor^2 / gamma, and no vacuum state is formed."""
    P = O.params(**_FLOORS)
    c = math.sqrt(1.4)
    assert 20.0 > 2 * (2 * c) / 0.4
    ps, us = O.riemann_star([1.0, -10.0, 0.0, 1.0], [1.0, 10.0, 0.0, 1.0], P)
    assert ps == pytest.approx(_PFLOOR, rel=1e-15)
    assert us == 0.0
