"""Langevin dynamics of a slab electrolyte (oracle).

ORACLE: test infrastructure (see oracle/__init__.py). Plain numpy, FP64.

Section 4.3 evolves the particles by Langevin dynamics,
  dr_i = p_i/m dt,  dp_i = [F_i - gamma p_i/m] dt + sqrt(2 gamma/beta) dW_i,
with F_i the (random-batch) Coulomb force plus the short-range model of
Section 5.2: a purely repulsive shifted-truncated Lennard-Jones potential
between particles,
  U_LJ(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6 + 1/4]  for r < 2^(1/6) sigma,
and the same form in the distance to each wall (z and Lz - z) with its own
eps_wall and sigma_wall. Periodic images in x and y; the walls keep the
particles inside [0, Lz].

Time stepping: the BAOAB splitting of Leimkuhler and Matthews (2013), in
velocities v = p/m: half kick, half drift, the exact Ornstein-Uhlenbeck
step v <- c v + sqrt((1 - c^2) kT/m) xi with c = e^{-gamma dt/m}, half
drift, new forces, half kick. x and y are wrapped into [0, L) after each
drift (x - L floor(x/L)).

Noise: xi of particle i at step n from Philox4x64-10 with counter
(i, n, 0, MD_TAG) and key (seed, 0): words (0, 1) and (2, 3) give two
Box-Muller pairs (u1 = 1 - uniform53, u2 = uniform53, r = sqrt(-2 ln u1),
(r cos 2 pi u2, r sin 2 pi u2)); xi = (first pair, first of the second).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .lattice import philox4x64_10, uniform53

PI = math.pi
MD_TAG = 0x4D445331
TWO16 = 2.0 ** (1.0 / 6.0)


@dataclasses.dataclass
class MDParams:
    dt: float
    mass: float = 1.0
    gamma: float = 1.0
    kT: float = 1.0
    lj_eps: float = 1.0
    lj_sigma: float = 1.0
    wall_eps: float = 1.0
    wall_sigma: float = 0.5
    seed: int = 0


def lj_pairs(pos, box, eps, sigma):
    """Shifted-truncated LJ energy and forces over all pairs (minimum image
    in x, y; the cut-off 2^(1/6) sigma must be below L/2)."""
    pos = np.asarray(pos, float)
    Lx, Ly, _ = box
    d = pos[:, None, :] - pos[None, :, :]
    d[..., 0] -= Lx * np.round(d[..., 0] / Lx)
    d[..., 1] -= Ly * np.round(d[..., 1] / Ly)
    r2 = (d * d).sum(-1)
    np.fill_diagonal(r2, np.inf)
    rc2 = (TWO16 * sigma) ** 2
    on = r2 < rc2
    s6 = np.where(on, (sigma * sigma / np.where(on, r2, 1.0)) ** 3, 0.0)
    e = np.where(on, 4 * eps * (s6 * s6 - s6 + 0.25), 0.0)
    # -dU/dr / r
    fr = np.where(on, 24 * eps * (2 * s6 * s6 - s6) / np.where(on, r2, 1.0), 0.0)
    F = (fr[..., None] * d).sum(1)
    return {"E": 0.5 * float(e.sum()), "F": F}


def lj_walls(pos, box, eps, sigma):
    """Shifted-truncated LJ of the distance to each wall (z and Lz - z)."""
    z = np.asarray(pos, float)[:, 2]
    Lz = box[2]
    E = np.zeros(z.size)
    Fz = np.zeros(z.size)
    for d, sgn in ((z, 1.0), (Lz - z, -1.0)):
        on = d < TWO16 * sigma
        dd = np.where(on, d, 1.0)
        s6 = (sigma / dd) ** 6
        E += np.where(on, 4 * eps * (s6 * s6 - s6 + 0.25), 0.0)
        Fz += sgn * np.where(on, 24 * eps * (2 * s6 * s6 - s6) / dd, 0.0)
    F = np.zeros((z.size, 3))
    F[:, 2] = Fz
    return {"E": float(E.sum()), "F": F}


def noise(N, step, seed):
    """Standard normal xi (N x 3) of one step."""
    ctr = np.zeros((N, 4), np.uint64)
    ctr[:, 0] = np.arange(N, dtype=np.uint64)
    ctr[:, 1] = np.uint64(step)
    ctr[:, 3] = np.uint64(MD_TAG)
    key = np.zeros((N, 2), np.uint64)
    key[:, 0] = np.uint64(seed)
    w = philox4x64_10(ctr, key)
    out = np.empty((N, 3))
    for j, (a, b) in enumerate(((0, 1), (2, 3))):
        u1 = 1.0 - uniform53(w[:, a])
        u2 = uniform53(w[:, b])
        r = np.sqrt(-2.0 * np.log(u1))
        th = 2.0 * PI * u2
        out[:, 2 * j] = r * np.cos(th)
        if j == 0:
            out[:, 1] = r * np.sin(th)
    return out


def wrap_xy(pos, box):
    pos = pos.copy()
    for a in (0, 1):
        pos[:, a] = pos[:, a] - box[a] * np.floor(pos[:, a] / box[a])
    return pos


def baoab_step(pos, vel, F, box, p: MDParams, step, force_fn):
    """One BAOAB step from (pos, vel) with the force F at pos; force_fn(pos)
    returns the force at the new positions. Returns (pos, vel, F)."""
    h = 0.5 * p.dt
    vel = vel + h * F / p.mass
    pos = wrap_xy(pos + h * vel, box)
    c = math.exp(-p.gamma * p.dt / p.mass)
    vel = c * vel + math.sqrt((1.0 - c * c) * p.kT / p.mass) * noise(len(pos), step, p.seed)
    pos = wrap_xy(pos + h * vel, box)
    F = force_fn(pos)
    vel = vel + h * F / p.mass
    return pos, vel, F
