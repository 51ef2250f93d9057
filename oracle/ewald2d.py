"""Direct FP64 evaluations of quasi-2D Coulomb sums (oracle).

ORACLE: test infrastructure (see oracle/__init__.py). Plain numpy/scipy, FP64,
O(N^2) per mode; meant for N up to a few thousand.

Everything is in Gaussian units with the pair energy U = 1/2 sum' q_i q_j/|r_ij|
(Eq. 2.8). Conventions: A = Lx*Ly; E = 1/2 sum_i q_i phi_i; F_i = -dE/dr_i.

  ewald2d_longrange   Lemma 2.1 (Eqs. 2.14-2.16) plus the self term
                      (Eq. 2.12): the exact long-range part with the erfc
                      z-kernel, every pair (i,j) including i = j.
  realspace           Eq. 2.10, the screened short-range sum within r_c,
                      explicit periodic images in x,y.
  image_sum           Eq. 2.3 / 2.8 summed directly over images inside a
                      growing disc (the symmetric shape of Thm 2.1), with
                      extrapolation in 1/R.
  soe_pair_direct     the SOE pair kernels of Eqs. 3.21 and 3.26 summed over
                      all pairs directly (no recursion), for small N.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf, erfc, erfcx

from .lattice import kvec

PI = math.pi
SQPI = math.sqrt(PI)


# ------------------------------------------------------------------ kernels


def xi_plus(k, z, alpha):
    """xi+(k,z) = e^{kz} erfc(k/(2 alpha) + alpha z) (Eq. 2.15), z >= 0.

    Written as erfcx(t) e^{-k^2/(4 alpha^2) - alpha^2 z^2} with
    t = k/(2 alpha) + alpha z, which never forms e^{kz}.
    """
    t = k / (2 * alpha) + alpha * z
    return erfcx(t) * np.exp(-(k / (2 * alpha)) ** 2 - (alpha * z) ** 2)


def xi_minus(k, z, alpha):
    """xi-(k,z) = e^{-kz} erfc(k/(2 alpha) - alpha z) (Eq. 2.15), z >= 0."""
    t = k / (2 * alpha) - alpha * z
    pos = erfcx(np.maximum(t, 0.0)) * np.exp(-(k / (2 * alpha)) ** 2 - (alpha * z) ** 2)
    neg = np.exp(-k * z) * erfc(np.minimum(t, 0.0))
    return np.where(t >= 0, pos, neg)


def g0_exact(z, alpha):
    """z erf(alpha z) + e^{-alpha^2 z^2}/(alpha sqrt(pi)) (Eq. 2.16), z >= 0."""
    return z * erf(alpha * z) + np.exp(-(alpha * z) ** 2) / (alpha * SQPI)


# ------------------------------------------------------------------ Ewald2D


def ewald2d_longrange(pos, q, box, alpha, mx, my, with_kzero=True, with_self=True):
    """Exact Ewald2D long-range part (Lemma 2.1) over the given k modes.

    The modes (mx, my) must be closed under k -> -k or be a half-plane whose
    weight is doubled by the caller; this routine sums exactly the modes it
    is given. Returns dict(E, phi, F) where phi and F include every term
    requested and E = 1/2 sum q phi.
    """
    pos = np.asarray(pos, float)
    q = np.asarray(q, float)
    Lx, Ly, _ = box
    A = Lx * Ly
    N = q.size
    x, y, z = pos[:, 0], pos[:, 1], pos[:, 2]
    dz = z[:, None] - z[None, :]
    adz = np.abs(dz)
    sgn = np.sign(dz)
    phi = np.zeros(N)
    F = np.zeros((N, 3))
    kx, ky, kk = kvec(mx, my, Lx, Ly)
    # group modes by |k| so the z-kernels are evaluated once per |k|
    order = np.argsort(kk, kind="stable")
    kk_s = kk[order]
    splits = np.flatnonzero(np.diff(kk_s) > 1e-12 * kk_s[1:]) + 1
    for grp in np.split(order, splits):
        k = kk[grp[0]]
        xp = xi_plus(k, adz, alpha)
        xm = xi_minus(k, adz, alpha)
        G = (xp + xm) / k                   # (1/k)(xi+ + xi-), symmetric in i,j
        Gd = (xp - xm) * sgn                # d/dz_i of (1/k)(xi+ + xi-)(|z_ij|)
        for m in grp:
            th = kx[m] * x + ky[m] * y
            c, s = np.cos(th), np.sin(th)
            # cos(k.rho_ij) = c_i c_j + s_i s_j ; sin(k.rho_ij) = s_i c_j - c_i s_j
            Gc, Gs = G @ (q * c), G @ (q * s)
            phi += (PI / A) * (c * Gc + s * Gs)
            sinsum = s * Gc - c * Gs               # sum_j q_j sin(k.rho_ij) G_ij
            F[:, 0] += (PI / A) * q * kx[m] * sinsum
            F[:, 1] += (PI / A) * q * ky[m] * sinsum
            Dc, Ds = Gd @ (q * c), Gd @ (q * s)
            F[:, 2] -= (PI / A) * q * (c * Dc + s * Ds)
    if with_kzero:
        g0 = g0_exact(adz, alpha)
        phi += -(2 * PI / A) * (g0 @ q)
        F[:, 2] += (2 * PI / A) * q * (erf(alpha * dz) @ q)
    if with_self:
        phi -= 2 * alpha / SQPI * q
    E = 0.5 * float(q @ phi)
    return {"E": E, "phi": phi, "F": F}


def realspace(pos, q, box, alpha, rc):
    """Short-range part phi_s (Eq. 2.10) within |r_ij + M| <= rc, images in x,y."""
    pos = np.asarray(pos, float)
    q = np.asarray(q, float)
    Lx, Ly, _ = box
    N = q.size
    phi = np.zeros(N)
    F = np.zeros((N, 3))
    nx = int(math.ceil(rc / Lx)) + 1
    ny = int(math.ceil(rc / Ly)) + 1
    d0 = pos[:, None, :] - pos[None, :, :]
    for ix in range(-nx, nx + 1):
        for iy in range(-ny, ny + 1):
            d = d0.copy()
            d[..., 0] += ix * Lx
            d[..., 1] += iy * Ly
            r = np.sqrt((d * d).sum(-1))
            mask = r <= rc
            if ix == 0 and iy == 0:
                np.fill_diagonal(mask, False)
            if not mask.any():
                continue
            rr = np.where(mask, r, 1.0)
            e = np.where(mask, erfc(alpha * rr) / rr, 0.0)
            phi += e @ q
            # -d/dr [erfc(a r)/r] = erfc(a r)/r^2 + 2a/sqrt(pi) e^{-a^2 r^2}/r
            fr = np.where(mask, (erfc(alpha * rr) / rr
                                 + 2 * alpha / SQPI * np.exp(-(alpha * rr) ** 2)) / (rr * rr), 0.0)
            F += q[:, None] * np.einsum("ij,ijc,j->ic", fr, d, q)
    return {"E": 0.5 * float(q @ phi), "phi": phi, "F": F}


def realspace_at(pos, q, box, alpha, rc, idx):
    """phi_s and F_s (Eq. 2.10, |r_ij + M| <= rc, images in x,y) of the
    particles idx only, each summed over every j: the same sum as realspace()
    restricted to a sample of targets, for systems too large for all pairs."""
    pos = np.asarray(pos, float)
    q = np.asarray(q, float)
    Lx, Ly, _ = box
    idx = np.asarray(idx, int)
    nx = int(math.ceil(rc / Lx)) + 1
    ny = int(math.ceil(rc / Ly)) + 1
    phi = np.zeros(idx.size)
    F = np.zeros((idx.size, 3))
    for a, i in enumerate(idx):
        d0 = pos[i][None, :] - pos
        for ix in range(-nx, nx + 1):
            for iy in range(-ny, ny + 1):
                d = d0.copy()
                d[:, 0] += ix * Lx
                d[:, 1] += iy * Ly
                r = np.sqrt((d * d).sum(-1))
                mask = r <= rc
                if ix == 0 and iy == 0:
                    mask[i] = False
                if not mask.any():
                    continue
                rr = r[mask]
                e = erfc(alpha * rr) / rr
                phi[a] += e @ q[mask]
                fr = (e + 2 * alpha / SQPI * np.exp(-(alpha * rr) ** 2)) / (rr * rr)
                F[a] += q[i] * ((fr * q[mask])[:, None] * d[mask]).sum(0)
    return {"phi": phi, "F": F}


def image_sum_energy(pos, q, box, R, chunk=200_000):
    """U(R) = 1/2 sum_{|M| <= R} sum'_{i,j} q_i q_j/|r_ij + M| (Eq. 2.8) with the
    images M = (mx Lx, my Ly, 0) inside the disc of radius R."""
    pos = np.asarray(pos, float)
    q = np.asarray(q, float)
    Lx, Ly, _ = box
    mxm = int(R / Lx) + 1
    mym = int(R / Ly) + 1
    mx, my = np.meshgrid(np.arange(-mxm, mxm + 1), np.arange(-mym, mym + 1), indexing="ij")
    Mx = (mx * Lx).ravel()
    My = (my * Ly).ravel()
    keep = Mx * Mx + My * My <= R * R
    Mx, My = Mx[keep], My[keep]
    N = q.size
    total = 0.0
    for i in range(N):
        for j in range(N):
            dx = pos[i, 0] - pos[j, 0]
            dy = pos[i, 1] - pos[j, 1]
            dzz = pos[i, 2] - pos[j, 2]
            acc = 0.0
            for c0 in range(0, Mx.size, chunk):
                ex = dx + Mx[c0:c0 + chunk]
                ey = dy + My[c0:c0 + chunk]
                r2 = ex * ex + ey * ey + dzz * dzz
                if i == j:
                    r2 = np.where(r2 == 0.0, np.inf, r2)
                acc += float(np.sort(1.0 / np.sqrt(r2)).sum())
            total += q[i] * q[j] * acc
    return 0.5 * total


def image_sum_extrapolated(pos, q, box, Rs):
    """Fit U(R) = U_inf + a/R + b/R^2 through the given radii (least squares)."""
    Rs = np.asarray(Rs, float)
    U = np.array([image_sum_energy(pos, q, box, R) for R in Rs])
    A = np.stack([np.ones_like(Rs), 1 / Rs, 1 / Rs ** 2], axis=1)
    coef, *_ = np.linalg.lstsq(A, U, rcond=None)
    return float(coef[0]), U


# ------------------------------------------------------------------ SOE direct


def soe_kernel_k(k, z, alpha, s, w):
    """(1/k)(xi+_M + xi-_M)(k, z) of Eq. 3.21 without the e^{ik.rho} factor."""
    a = alpha * np.asarray(s)
    C = 2 * alpha * math.exp(-k * k / (4 * alpha * alpha)) / (SQPI * k)
    out = 0.0
    for al, wl in zip(a, w):
        out = out + wl / (al * al - k * k) * (2 * al * np.exp(-k * z) - 2 * k * np.exp(-al * z))
    return C * np.real(out)


def soe_kernel_k_dz(k, z, alpha, s, w):
    """d/dz of soe_kernel_k (Eq. E.5 form)."""
    a = alpha * np.asarray(s)
    C = 2 * alpha * math.exp(-k * k / (4 * alpha * alpha)) / (SQPI * k)
    out = 0.0
    for al, wl in zip(a, w):
        out = out + wl / (al * al - k * k) * (-2 * al * k * np.exp(-k * z) + 2 * k * al * np.exp(-al * z))
    return C * np.real(out)


def soe_kernel_0(z, alpha, s, w):
    """g0_SOE(z) of Eq. 3.26."""
    out = 0.0
    for sl, wl in zip(s, w):
        out = out + wl / SQPI * (2 * z / sl + (1 / alpha - 2 * z / sl) * np.exp(-alpha * sl * z))
    return np.real(out)


def soe_kernel_0_dz(z, alpha, s, w):
    """g0_SOE'(z) of Eq. E.6."""
    out = 0.0
    for sl, wl in zip(s, w):
        out = out + wl / SQPI * (2 / sl - (sl + 2 / sl - 2 * alpha * z) * np.exp(-alpha * sl * z))
    return np.real(out)


def soe_pair_direct(pos, q, box, alpha, s, w, mx, my, gam):
    """Direct O(N^2 K M) evaluation of the SOE pair sums (j != i only).

    For each mode k with prefactor gam[k] (pi/A C_k and the mode weight, see
    oracle.soe_longrange) and for k = 0, returns phi and F of the pair parts.
    The SOE kernel is written so that gam * C_k^{-1} appears; here gam is the
    full prefactor of (pi/A)(1/k)(xi+_M + xi-_M), i.e. gam_k / ((pi/A) C_k)
    is the mode weight.
    """
    pos = np.asarray(pos, float)
    q = np.asarray(q, float)
    Lx, Ly, _ = box
    A = Lx * Ly
    N = q.size
    x, y, z = pos[:, 0], pos[:, 1], pos[:, 2]
    dz = z[:, None] - z[None, :]
    adz = np.abs(dz)
    sgn = np.sign(dz)
    off = ~np.eye(N, dtype=bool)
    phi = np.zeros(N)
    F = np.zeros((N, 3))
    kx, ky, kk = kvec(mx, my, Lx, Ly)
    for m in range(len(kk)):
        k = kk[m]
        C = 2 * alpha * math.exp(-k * k / (4 * alpha * alpha)) / (SQPI * k)
        wmode = gam[m] / ((PI / A) * C)         # mode weight
        G = soe_kernel_k(k, adz, alpha, s, w) * off
        Gd = soe_kernel_k_dz(k, adz, alpha, s, w) * sgn * off
        dth = kx[m] * (x[:, None] - x[None, :]) + ky[m] * (y[:, None] - y[None, :])
        cs, sn = np.cos(dth), np.sin(dth)
        pref = wmode * PI / A
        phi += pref * ((cs * G) @ q)
        F[:, 0] += pref * q * kx[m] * ((sn * G) @ q)
        F[:, 1] += pref * q * ky[m] * ((sn * G) @ q)
        F[:, 2] -= pref * q * ((cs * Gd) @ q)
    g0 = soe_kernel_0(adz, alpha, s, w) * off
    g0d = soe_kernel_0_dz(adz, alpha, s, w) * sgn * off
    phi0 = -(2 * PI / A) * (g0 @ q)
    fz0 = (2 * PI / A) * q * (g0d @ q)
    return {"phi_k": phi, "F_k": F, "phi_0": phi0, "fz_0": fz0}
