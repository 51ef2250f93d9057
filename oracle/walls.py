"""Charged walls at z = 0 and z = Lz: the particle-slab potential (oracle).

ORACLE: test infrastructure (see oracle/__init__.py). Plain numpy, FP64.

Section 2.4 adds two walls with doubly periodic surface charge densities
sigma_bot(rho) at z = 0 and sigma_top(rho) at z = Lz. The potential at a
particle is phi_p-p + phi_p-s, where phi_p-p is the Ewald2D potential of the
particles alone (which need not be neutral; the particles and walls together
must be: the neutrality condition of Section 2.4) and phi_p-s the potential
of the walls (Thm 2.4):

  phi_p-s(r) = (2 pi / A) sum_{k != 0} e^{i k.rho}/k
                 [sig^_bot(k) e^{-k|z|} + sig^_top(k) e^{-k|z - Lz|}]
               - (2 pi / A) [sig^_bot(0) |z| + sig^_top(0) |z - Lz|]

with A = Lx Ly and sig^(k) the integral of sigma(rho) e^{-i k.rho} over one
cell [0, Lx] x [0, Ly]. With uniform densities only the k = 0 term remains
(the uniform-density case stated after Thm 2.4).

Densities are given by their Fourier series per unit area,

  sigma(rho) = sigma0 + sum_w 2 Re[ sigma_w e^{i k_w . rho} ],

so that sig^(0) = A sigma0, sig^(k_w) = A sigma_w, sig^(-k_w) = A conj(sigma_w):
``modes`` lists each pair (m, -m) once, (mx, my) != (0, 0).

Energy: the walls are fixed external charges, so each particle-wall pair is
counted once, U_p-s = sum_i q_i phi_p-s(r_i) (no factor 1/2); then
F_i = -dU_p-s/dr_i = -q_i grad phi_p-s(r_i) and phi_p-s = dU_p-s/dq_i.
"""
from __future__ import annotations

import math

import numpy as np

from .lattice import kvec

PI = math.pi


def _full_set(box, modes, sb, st):
    """The modes k and -k of the listed pairs with their cell integrals."""
    Lx, Ly, _ = box
    A = Lx * Ly
    modes = np.asarray(modes, dtype=np.int64).reshape(-1, 2)
    sb = np.asarray(sb, dtype=complex).reshape(-1)
    st = np.asarray(st, dtype=complex).reshape(-1)
    mx = np.concatenate([modes[:, 0], -modes[:, 0]])
    my = np.concatenate([modes[:, 1], -modes[:, 1]])
    hb = A * np.concatenate([sb, np.conj(sb)])
    ht = A * np.concatenate([st, np.conj(st)])
    return mx, my, hb, ht


def wall_potential(pos, q, box, sigma_bot0, sigma_top0, modes=(), sb=(), st=()):
    """phi_p-s and F_p-s at every particle and U_p-s (Thm 2.4).

    For z inside [0, Lz]; on a wall (z = 0 or z = Lz) the z-derivative is
    the one-sided limit from inside the slab."""
    pos = np.asarray(pos, float)
    q = np.asarray(q, float)
    Lx, Ly, Lz = box
    A = Lx * Ly
    x, y, z = pos[:, 0], pos[:, 1], pos[:, 2]
    zb = np.abs(z)                 # distance to the bottom wall
    zt = np.abs(z - Lz)            # distance to the top wall
    sgb = np.where(z >= 0, 1.0, -1.0)    # d|z|/dz, +1 on the wall itself
    sgt = np.where(z > Lz, 1.0, -1.0)    # d|z - Lz|/dz, -1 on the wall itself
    # zero mode of Thm 2.4
    phi = -(2 * PI / A) * (A * sigma_bot0 * zb + A * sigma_top0 * zt)
    dphi_dz = -(2 * PI / A) * (A * sigma_bot0 * sgb + A * sigma_top0 * sgt)
    dphi_dx = np.zeros_like(x)
    dphi_dy = np.zeros_like(x)
    if len(modes):
        mx, my, hb, ht = _full_set(box, modes, sb, st)
        kx, ky, kk = kvec(mx, my, Lx, Ly)
        for j in range(mx.size):
            ph = np.exp(1j * (kx[j] * x + ky[j] * y))
            eb = np.exp(-kk[j] * zb)
            et = np.exp(-kk[j] * zt)
            term = (2 * PI / A) * ph / kk[j] * (hb[j] * eb + ht[j] * et)
            phi = phi + term.real
            dphi_dx = dphi_dx + (1j * kx[j] * term).real
            dphi_dy = dphi_dy + (1j * ky[j] * term).real
            dz = (2 * PI / A) * ph / kk[j] * (hb[j] * (-kk[j] * sgb) * eb
                                              + ht[j] * (-kk[j] * sgt) * et)
            dphi_dz = dphi_dz + dz.real
    F = -q[:, None] * np.stack([dphi_dx, dphi_dy, dphi_dz], axis=1)
    return {"E": float(q @ phi), "phi": phi, "F": F}


def wall_charge(box, sigma_bot0, sigma_top0):
    """Net charge of the two walls per cell: sig^_bot(0) + sig^_top(0)."""
    Lx, Ly, _ = box
    return Lx * Ly * (sigma_bot0 + sigma_top0)


def discretise_wall(box, z0, sigma0, modes=(), sw=(), n=16):
    """Point charges on an n x n grid at height z0 (cell midpoints) carrying
    sigma(rho) A / n^2: the trapezoid rule, exact for the Fourier modes with
    |mx|, |my| < n; its aliases sit at wave numbers >= 2 pi (n - |m|)/L."""
    Lx, Ly, _ = box
    A = Lx * Ly
    g = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(g * Lx, g * Ly, indexing="ij")
    X, Y = X.ravel(), Y.ravel()
    sig = np.full(X.size, float(sigma0))
    modes = np.asarray(modes, dtype=np.int64).reshape(-1, 2)
    sw = np.asarray(sw, dtype=complex).reshape(-1)
    for (m1, m2), c in zip(modes, sw):
        sig += 2 * (c * np.exp(1j * (2 * PI * m1 / Lx * X + 2 * PI * m2 / Ly * Y))).real
    pos = np.stack([X, Y, np.full(X.size, float(z0))], axis=1)
    return pos, sig * A / (n * n)
