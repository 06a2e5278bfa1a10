"""Pin of the Sedov-blast workload on the oracle: the blast front against the
Sedov-Taylor similarity solution of a point explosion in a cold uniform gas.

In d dimensions (d = 2 here: a cylindrical blast) the front of a blast of
energy E in a gas of density rho0 is at R(t) = xi0 (E t^2 / rho0)^(1/(d+2)).
The constant xi0 = alpha^(-1/(d+2)) follows from the self-similar flow behind
the strong shock.  With lambda = r / R(t), delta = 2/(d+2) (R grows like
t^delta), and
    u = (r/t) V(lambda),  rho = rho0 G(lambda),  c^2 = (r/t)^2 Z(lambda),
the Euler equations (mass, momentum, entropy; p = rho c^2 / g) become, in
x = ln lambda, with w = V - delta and primes d/dx,
    w G'/G + V' + d V = 0
    (Z/g) G'/G + w V' + Z'/g + V (V - 1) + 2 Z/g = 0
    (1 - g) w G'/G + w Z'/Z + 2 (V - 1) = 0,
a linear system in (G'/G, V', Z'/Z) whose determinant is proportional to
Z - w^2 (the flow behind the shock is subsonic relative to the similarity
lines, so it stays positive).  At the shock (lambda = 1) the strong-shock
jump conditions give V = 2 delta/(g+1), G = (g+1)/(g-1) and
Z = 2 g (g-1) delta^2/(g+1)^2.  The energy of the flow is
    E = S_d rho0 R^(d+2) / t^2 * int_0^1 lambda^(d+1) G (V^2/2 + Z/(g(g-1))) d lambda
(S_d = 2 pi for d = 2), so alpha = S_d * integral.  Near the centre the
pressure is uniform, which forces V -> delta / g: the integration is checked
against that limit.

The workload (problems.sedov) puts E = 1 into the corner cell of a grid with
reflective walls on every side, a quarter of a blast of 4E centred on the
corner point.  The oracle's front is a few cells wide; the exact radius must
lie between its density peak and its outer half-peak point, and their mean
must follow R(t) within 2 % at both times and its growth the t^(1/2) law
within 3 %.  Planted mistakes move the front by far more: the scheme run with
g = 5/3 on this state puts it at 1.15 R, a blast of half the energy at 0.84 R."""
import numpy as np
import pytest

import oracle as O
from paper_2106_13465_gb300 import problems as pr

scipy_integrate = pytest.importorskip("scipy.integrate")


def _similarity(g: float, d: int, x_end: float):
    delta = 2.0 / (d + 2)

    def rhs(x, y):
        V, lnG, lnZ = y
        Z = np.exp(lnZ)
        w = V - delta
        gl = (-V * (V - 1) - 2 * Z / g + d * V * w + 2 * Z * (V - 1) / (g * w)) / (Z - w * w)
        dV = -d * V - w * gl
        zl = (-2 * (V - 1) - (1 - g) * w * gl) / w
        return [dV, gl, zl]

    y0 = [2 * delta / (g + 1), np.log((g + 1) / (g - 1)), np.log(2 * g * (g - 1) * delta ** 2 / (g + 1) ** 2)]
    x = np.linspace(0.0, x_end, 40001)
    sol = scipy_integrate.solve_ivp(rhs, (0.0, x_end), y0, method="DOP853", rtol=1e-11, atol=1e-12, t_eval=x)
    assert sol.status == 0
    return x, sol.y, delta


def sedov_alpha(g: float, d: int = 2, x_end: float = -8.0) -> float:
    x, (V, lnG, lnZ), _ = _similarity(g, d, x_end)
    lam = np.exp(x)
    # d lambda = lambda dx; x runs from 0 down to x_end
    f = lam ** (d + 2) * np.exp(lnG) * (V ** 2 / 2 + np.exp(lnZ) / (g * (g - 1)))
    S = {1: 2.0, 2: 2.0 * np.pi, 3: 4.0 * np.pi}[d]
    return S * float(-np.trapezoid(f, x))


def test_similarity_solution_is_consistent():
    g = pr.GAMMA
    x, (V, _, _), delta = _similarity(g, 2, -8.0)
    assert abs(V[-1] - delta / g) < 1e-4            # uniform central pressure
    a8, a10 = sedov_alpha(g, 2, -8.0), sedov_alpha(g, 2, -10.0)
    assert abs(a8 - a10) < 1e-6 * a8                # the centre holds no energy to speak of
    assert sedov_alpha(5.0 / 3.0) < 0.7 * a8        # larger gamma: less energy for the same front


def _front(U: np.ndarray, h: float):
    """Density peak radius and outer half-peak radius of the azimuthally
    averaged density, r measured from the corner point."""
    ny, nx = U.shape[1:]
    yc = (np.arange(ny) + 0.5) * h
    xc = (np.arange(nx) + 0.5) * h
    r = np.hypot(xc[None, :], yc[:, None])
    bins = np.floor(r / h).astype(int)
    nb = int(bins.max()) + 1
    prof = np.bincount(bins.ravel(), U[0].ravel(), nb) / np.maximum(np.bincount(bins.ravel(), None, nb), 1)
    k = int(np.argmax(prof))
    mid = 0.5 * (1.0 + prof[k])
    kout = int(np.nonzero(prof > mid)[0].max())
    return (k + 0.5) * h, (kout + 1) * h


def test_oracle_blast_front_follows_sedov_taylor():
    pb = pr.sedov(128)
    assert pb.bc == (pr.REFLECT,) * 4
    rho0 = float(pb.U[0, 1, 1])
    assert float(pb.U[3, 0, 0]) * pb.h * pb.h == 1.0   # the deposited energy
    E = 4.0                                          # the corner cell's energy, mirrored four ways
    xi0 = sedov_alpha(pr.GAMMA) ** -0.25
    U, t, steps = pb.U.copy(), 0.0, 0
    mids = []
    for t_target in (0.05, 0.1):
        while t < t_target:
            U, dts, rc = O.run(U, pb.h, pb.bc, 5, step0=steps, threads=0)
            assert rc == 0
            t += float(dts.sum())
            steps += 5
        R = xi0 * (E * t * t / rho0) ** 0.25
        r_peak, r_out = _front(U, pb.h)
        assert r_peak <= R <= r_out, (t, r_peak, R, r_out)
        mid = 0.5 * (r_peak + r_out)
        assert abs(mid / R - 1.0) < 0.02, (t, mid, R)
        mids.append((t, mid))
    (t1, m1), (t2, m2) = mids
    assert abs((m2 / m1) / np.sqrt(t2 / t1) - 1.0) < 0.03
