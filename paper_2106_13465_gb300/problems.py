"""Seeded synthetic initial states for the HYDRO workloads.

This module only *states* initial data.  It holds none of the scheme's
arithmetic (no slope, trace, Riemann or update step) and imports neither the
CUDA binding nor the oracle, so the CUDA path and the oracle consume the same
arrays without sharing any code.  Each state is returned as conserved
variables U[4, ny, nx] in FP64, planes (rho, rho*u, rho*v, E), x fastest; the
ideal-gas energy E = p/(gamma-1) + rho (u^2 + v^2)/2 is the definition of the
initial data, not a step of the method.

Workloads (the paper runs a "point explosion" on a 10000^2 grid, §7; the
shapes below restate it as a Sedov blast and add the standard shock-tube,
random-mode, batch and shear-layer cases):
  * sedov(n)          reflective box, rho=1, u=v=0, p=1e-5, total energy 1 in
                      corner cell (0,0): E(0,0) = 1/h^2
  * sod(nx, ny, axis) transmissive tube, (rho,p) = (1,1) | (0.125,0.1) split at
                      mid-length along `axis`, u=v=0
  * random_modes(n)   periodic, rho = 1 + 0.1 sum_8 cos(2 pi k.x + phi), p = 1,
                      (u, v) = 0.2 sum_8 (cos, sin)(2 pi k'.x + phi')
  * kelvin_helmholtz  periodic shear layer (rho 2|1, u +-0.5 tanh-smoothed,
                      p = 2.5, v = 0.01 sin(4 pi x) + U(-1e-3, 1e-3))
  * batch(ngrids)     ragged list of the above with log-uniform sides in [32,512]
Mesh: h = dx = dy = 1/max(nx, ny); cell centres ((i+1/2)h, (j+1/2)h).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED = 2106
GAMMA = 1.4

REFLECT, TRANSMISSIVE, PERIODIC = 0, 1, 2


@dataclass
class Problem:
    name: str
    U: np.ndarray            # [4, ny, nx] float64
    h: float
    bc: tuple                # (xlo, xhi, ylo, yhi)
    meta: dict = field(default_factory=dict)

    @property
    def nx(self) -> int:
        return int(self.U.shape[2])

    @property
    def ny(self) -> int:
        return int(self.U.shape[1])


def _rng(seed: int, purpose: int) -> np.random.Generator:
    """Independent sub-stream per purpose (SeedSequence spawn key)."""
    return np.random.default_rng(np.random.SeedSequence(seed, spawn_key=(purpose,)))


def conserved(rho, u, v, p, gamma: float = GAMMA) -> np.ndarray:
    """Stack initial primitive fields into U = (rho, rho u, rho v, E)."""
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), shape)
    v = np.broadcast_to(np.asarray(v, dtype=np.float64), shape)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), shape)
    U = np.empty((4,) + shape, dtype=np.float64)
    U[0] = rho
    U[1] = rho * u
    U[2] = rho * v
    U[3] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return U


def mesh_h(nx: int, ny: int) -> float:
    return 1.0 / max(nx, ny)


def uniform(nx: int, ny: int, rho=1.0, u=0.0, v=0.0, p=1.0, bc=(PERIODIC,) * 4,
            gamma: float = GAMMA) -> Problem:
    U = conserved(np.full((ny, nx), rho), u, v, p, gamma)
    return Problem("uniform", U, mesh_h(nx, ny), tuple(bc))


def sedov(nx: int, ny: int | None = None, gamma: float = GAMMA, p_ambient: float = 1e-5,
          energy: float = 1.0) -> Problem:
    ny = nx if ny is None else ny
    h = mesh_h(nx, ny)
    U = conserved(np.ones((ny, nx)), 0.0, 0.0, p_ambient, gamma)
    U[3, 0, 0] = energy / (h * h)
    return Problem(f"sedov{nx}x{ny}", U, h, (REFLECT,) * 4)


def sod(nx: int, ny: int, axis: int = 0, gamma: float = GAMMA) -> Problem:
    """Sod tube along axis 0 (x) or 1 (y); the left state fills the first half."""
    n = nx if axis == 0 else ny
    k = np.arange(n)
    left = k < n // 2
    prof_r = np.where(left, 1.0, 0.125)
    prof_p = np.where(left, 1.0, 0.1)
    if axis == 0:
        rho = np.broadcast_to(prof_r[None, :], (ny, nx)).copy()
        p = np.broadcast_to(prof_p[None, :], (ny, nx)).copy()
    else:
        rho = np.broadcast_to(prof_r[:, None], (ny, nx)).copy()
        p = np.broadcast_to(prof_p[:, None], (ny, nx)).copy()
    U = conserved(rho, 0.0, 0.0, p, gamma)
    return Problem(f"sod{'xy'[axis]}{nx}x{ny}", U, mesh_h(nx, ny), (TRANSMISSIVE,) * 4)


def _modes(rng: np.random.Generator, count: int, kmax: int):
    """`count` integer wave vectors k != 0 with |k| <= kmax and phases in [0, 2 pi)."""
    ks = []
    while len(ks) < count:
        k = rng.integers(-kmax, kmax + 1, size=2)
        if (k[0] or k[1]) and k[0] * k[0] + k[1] * k[1] <= kmax * kmax:
            ks.append((int(k[0]), int(k[1])))
    phases = rng.uniform(0.0, 2.0 * np.pi, size=count)
    return np.array(ks, dtype=np.float64), phases


def random_modes(nx: int, ny: int | None = None, seed: int = SEED, gamma: float = GAMMA,
                 nmodes: int = 8, kmax: int = 8, rows: slice | None = None) -> Problem:
    """Periodic random-mode field.  `rows` restricts generation to a band of rows
    (same values as the full field there), for bounded samples of big grids."""
    ny = nx if ny is None else ny
    h = mesh_h(nx, ny)
    rng = _rng(seed, 3)
    kr, phr = _modes(rng, nmodes, kmax)
    kv, phv = _modes(rng, nmodes, kmax)
    j = np.arange(ny)[rows] if rows is not None else np.arange(ny)
    x = (np.arange(nx) + 0.5) * h
    y = (j + 0.5) * h
    # each mode cos(2 pi (k0 x + k1 y) + phi) = cos(a + b) with a = 2 pi k0 x
    # and b = 2 pi k1 y + phi, expanded by the angle-sum identities into
    # outer products of row and column vectors (a band of rows gets the same
    # values as inside the full field)
    two_pi = 2.0 * np.pi
    rho = np.ones((len(j), nx))
    for (k, ph) in zip(kr, phr):
        a, b = two_pi * k[0] * x, two_pi * k[1] * y + ph
        rho += 0.1 * (np.outer(np.cos(b), np.cos(a)) - np.outer(np.sin(b), np.sin(a)))
    u = np.zeros_like(rho)
    v = np.zeros_like(rho)
    for (k, ph) in zip(kv, phv):
        a, b = two_pi * k[0] * x, two_pi * k[1] * y + ph
        ca, sa, cb, sb = np.cos(a), np.sin(a), np.cos(b), np.sin(b)
        u += 0.2 * (np.outer(cb, ca) - np.outer(sb, sa))
        v += 0.2 * (np.outer(cb, sa) + np.outer(sb, ca))
    U = conserved(rho, u, v, 1.0, gamma)
    return Problem(f"modes{nx}x{ny}", U, h, (PERIODIC,) * 4,
                   {"k_rho": kr.tolist(), "k_vel": kv.tolist()})


def kelvin_helmholtz(nx: int, ny: int | None = None, seed: int = SEED, gamma: float = GAMMA,
                     rows: slice | None = None) -> Problem:
    ny = nx if ny is None else ny
    h = mesh_h(nx, ny)
    j = np.arange(ny)[rows] if rows is not None else np.arange(ny)
    x = (np.arange(nx) + 0.5) * h
    y = (j + 0.5) * h
    X, Y = np.meshgrid(x, y)
    rho = np.where(np.abs(Y - 0.5) < 0.25, 2.0, 1.0)
    u = 0.5 * (np.tanh((Y - 0.25) / 0.01) - np.tanh((Y - 0.75) / 0.01)) - 0.5
    # the noise is drawn for the whole grid row by row, so a band of rows gets
    # the same values it has inside the full field
    rng = _rng(seed, 5)
    noise = np.empty((len(j), nx))
    row0 = int(j[0]) if len(j) else 0
    if row0:
        rng.uniform(-1e-3, 1e-3, size=(row0, nx))
    noise[:] = rng.uniform(-1e-3, 1e-3, size=(len(j), nx))
    v = 0.01 * np.sin(4.0 * np.pi * X) + noise
    U = conserved(rho, u, v, 2.5, gamma)
    return Problem(f"kh{nx}x{ny}", U, h, (PERIODIC,) * 4)


BATCH_KINDS = ("sedov", "sod_x", "sod_y", "modes")


def batch_shapes(ngrids: int = 512, seed: int = SEED, lo: int = 32, hi: int = 512):
    """Side lengths round(exp(U[ln lo, ln hi])) per axis and a kind per grid."""
    rng = _rng(seed, 4)
    nx = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=ngrids))).astype(int)
    ny = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=ngrids))).astype(int)
    kind = rng.integers(0, len(BATCH_KINDS), size=ngrids)
    return [(int(a), int(b), BATCH_KINDS[int(c)]) for a, b, c in zip(nx, ny, kind)]


def batch(ngrids: int = 512, seed: int = SEED, lo: int = 32, hi: int = 512,
          gamma: float = GAMMA) -> list[Problem]:
    out = []
    for g, (nx, ny, kind) in enumerate(batch_shapes(ngrids, seed, lo, hi)):
        if kind == "sedov":
            pb = sedov(nx, ny, gamma)
        elif kind == "sod_x":
            pb = sod(nx, ny, 0, gamma)
        elif kind == "sod_y":
            pb = sod(nx, ny, 1, gamma)
        else:
            pb = random_modes(nx, ny, seed=seed + 1 + g, gamma=gamma)
        pb.meta["kind"] = kind
        out.append(pb)
    return out


def transpose(pb: Problem) -> Problem:
    """Mirror the state about the diagonal: swap x/y, swap rho*u/rho*v, swap the
    x and y boundary conditions."""
    U = pb.U
    T = np.empty((4, U.shape[2], U.shape[1]), dtype=np.float64)
    T[0] = U[0].T
    T[1] = U[2].T
    T[2] = U[1].T
    T[3] = U[3].T
    bc = (pb.bc[2], pb.bc[3], pb.bc[0], pb.bc[1])
    return Problem(pb.name + "_T", T, pb.h, bc, dict(pb.meta))
