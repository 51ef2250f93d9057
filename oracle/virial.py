"""Virial tensor of the Ewald2D energy of a slab (oracle).

ORACLE: test infrastructure (see oracle/__init__.py). Plain numpy + the C
recursion of soe_recursion.c, FP64.

The paper notes that the random-batch dynamics extends to the NPT ensemble
once the virial tensor is approximated as well (Section 4.3 and its
discussion of other ensembles), and that the L_z-dependent constant of the
particle-slab potential (Section 2.4, uniform-density case of Thm 2.4) is
what makes pressures come out right. This module computes that virial.

Definition. A strain eps maps every particle r -> (I + eps) r, the two
lattice vectors (Lx, 0, 0), (0, Ly, 0) -> (I + eps) a, and every element of
the two charged walls with the box, keeping its charge. The lattice stays in
the plane z = 0, so eps_zx = eps_zy = 0; the virial is

    W_ab = -dE/d eps_ab  at eps = 0,   ab in {xx, yy, xy, zz, xz, yz},

W_xy = W_yx by rotation invariance in the plane. For the components that
leave the lattice alone (zz, xz, yz) this is W_ab = sum_i F_i,a r_i,b plus
the explicit terms of the top wall, which moves with the box.

Lateral part of the long-range energy (Lemma 2.1). Under a lateral strain the
phases k.rho_ij do not change, the area scales as A (1 + tr eps) and
|k| -> |k| - k_a eps_ab k_b/|k|. Every term of E except U_self carries 1/A,
so with U^k = (pi/(2A)) sum_{i,j} q_i q_j cos(k.rho_ij) G(|k|, |z_ij|),
G = (xi+ + xi-)/k (j = i included),

    W_ab = delta_ab (E + U_self) + sum_k (k_a k_b/|k|) D_k,
    D_k = (pi/(2A)) sum_{i,j} q_i q_j cos(k.rho_ij) dG/dk(|k|, |z_ij|),
    dG/dk = -G/k + [z (xi+ - xi-) - (2/(alpha sqrt(pi))) e^{-k^2/(4 alpha^2)
             - alpha^2 z^2}]/k       (exact kernel; from Eq. 2.15),

and for the SOE kernel of Eq. 3.21 the k-derivative of its SOE form (the
recursion of soe_recursion.c). The j = i part of D_k uses the exact
G(k, 0) = 2 erfc(k/(2 alpha))/k, as the energy's constants do. For a
random-batch sample each mode's D_k gets the weight (H/P) e^{k^2/(4 alpha^2)}
of Eq. 4.7 (an unbiased estimator of the full sum); the j = i part is summed
over the whole lattice.

Walls (Thm 2.4). The walls keep their charge per cell, so sigma and its
per-area Fourier coefficients scale as 1/A, and the wall modes' wave vectors
move like k. The top wall sits at z = L_z, which scales with eps_zz and
shifts by eps_xz L_z, eps_yz L_z in x and y.

Real space (Eq. 2.10 within r_c): the pair virial
W_ab = (1/2) sum_{i,j,M} (F_ij)_a (r_ij)_b with r_ij = r_i - r_j + M.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
from scipy.special import erfc

from . import soe_ewald2d as _se
from .ewald2d import ewald2d_longrange, g0_exact, realspace, xi_minus, xi_plus
from .lattice import H_direct, full_modes, kvec, self_energy_coef
from .soe_ewald2d import soe_full, soe_rbe

PI = math.pi
SQPI = math.sqrt(PI)
KEYS = ("xx", "yy", "xy", "zz", "xz", "yz")


def _lib():
    lib = _se._load()
    if not hasattr(lib, "_dk_ready"):
        P = ctypes.POINTER(ctypes.c_double)
        lib.oracle_kspace_soe_dk.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_int64,
                                             P, P, ctypes.c_double, ctypes.c_int,
                                             P, P, P, P, P]
        lib.oracle_kspace_soe_dk.restype = None
        lib._dk_ready = True
    return lib


def _zero():
    return {k: 0.0 for k in KEYS}


def _add(a, b, scale=1.0):
    return {k: a[k] + scale * b[k] for k in KEYS}


def force_part(pos, F):
    """The terms sum_i F_i,a r_i,b of the components that leave the lattice
    alone (zz, xz, yz)."""
    pos = np.asarray(pos, float)
    F = np.asarray(F, float)
    W = _zero()
    W["zz"] = float(F[:, 2] @ pos[:, 2])
    W["xz"] = float(F[:, 0] @ pos[:, 2])
    W["yz"] = float(F[:, 1] @ pos[:, 2])
    return W


def lateral_from_modes(box, mx, my, D):
    """sum over modes of (k_a k_b/|k|) D_k for ab in {xx, yy, xy}."""
    Lx, Ly, _ = box
    kx, ky, kk = kvec(mx, my, Lx, Ly)
    D = np.asarray(D, float)
    W = _zero()
    W["xx"] = float((kx * kx / kk * D).sum())
    W["yy"] = float((ky * ky / kk * D).sum())
    W["xy"] = float((kx * ky / kk * D).sum())
    return W


def dG_exact(k, z, alpha):
    """dG/dk of G(k, z) = (xi+ + xi-)(k, z)/k (Eq. 2.15), z >= 0."""
    xp = xi_plus(k, z, alpha)
    xm = xi_minus(k, z, alpha)
    gauss = np.exp(-(k / (2 * alpha)) ** 2 - (alpha * z) ** 2)
    return -(xp + xm) / (k * k) + (z * (xp - xm) - 2.0 / (alpha * SQPI) * gauss) / k


def dG0_exact(k, alpha):
    """dG/dk at z = 0: d/dk [2 erfc(k/(2 alpha))/k]."""
    return -2 * erfc(k / (2 * alpha)) / (k * k) - 2 * np.exp(-(k / (2 * alpha)) ** 2) / (alpha * SQPI * k)


def diag_dk(alpha, box, mx, my):
    """(pi/(2A)) dG/dk(k, 0) per mode: the j = i part of D_k per unit Q."""
    Lx, Ly, _ = box
    _, _, kk = kvec(mx, my, Lx, Ly)
    return PI / (2 * Lx * Ly) * dG0_exact(kk, alpha)


# ------------------------------------------------------------------ exact


def longrange_virial_exact(pos, q, box, alpha, mx, my):
    """Virial of the exact Ewald2D long-range energy (Lemma 2.1, every pair
    including j = i, the k = 0 term and U_self) over the given modes, which
    must be closed under k -> -k. O(N^2 K)."""
    pos = np.asarray(pos, float)
    q = np.asarray(q, float)
    Lx, Ly, _ = box
    A = Lx * Ly
    out = ewald2d_longrange(pos, q, box, alpha, mx, my)
    x, y, z = pos[:, 0], pos[:, 1], pos[:, 2]
    adz = np.abs(z[:, None] - z[None, :])
    kx, ky, kk = kvec(mx, my, Lx, Ly)
    D = np.zeros(len(kk))
    order = np.argsort(kk, kind="stable")
    kk_s = kk[order]
    splits = np.flatnonzero(np.diff(kk_s) > 1e-12 * kk_s[1:]) + 1
    for grp in np.split(order, splits):
        dG = dG_exact(kk[grp[0]], adz, alpha)
        for m in grp:
            th = kx[m] * x + ky[m] * y
            c, s = q * np.cos(th), q * np.sin(th)
            D[m] = PI / (2 * A) * float(c @ dG @ c + s @ dG @ s)
    W = lateral_from_modes(box, mx, my, D)
    Uself = self_energy_coef(alpha) * float(q @ q)
    W["xx"] += out["E"] + Uself
    W["yy"] += out["E"] + Uself
    W = _add(W, force_part(pos, out["F"]))
    return {"W": W, "E": out["E"], "F": out["F"]}


def longrange_energy_lattice(frac, z, q, h, alpha, m, with_kzero=True, with_self=True):
    """Exact Ewald2D long-range energy (Lemma 2.1) for an oblique lattice.

    h: 2 x 2 matrix whose columns are the lattice vectors; frac: N x 2
    fractional coordinates (rho = h frac); m: K x 2 integer modes (closed
    under m -> -m), k = 2 pi h^{-T} m, A = |det h|. The rectangular box is
    h = diag(Lx, Ly). Used to differentiate the energy under a shear.
    """
    frac = np.asarray(frac, float)
    z = np.asarray(z, float)
    q = np.asarray(q, float)
    h = np.asarray(h, float)
    m = np.asarray(m, float).reshape(-1, 2)
    A = abs(float(np.linalg.det(h)))
    kvecs = 2 * PI * m @ np.linalg.inv(h)       # rows: k = 2 pi h^{-T} m
    kk = np.sqrt((kvecs ** 2).sum(1))
    adz = np.abs(z[:, None] - z[None, :])
    E = 0.0
    for j in range(len(kk)):
        th = 2 * PI * (frac @ m[j])
        c, s = q * np.cos(th), q * np.sin(th)
        G = (xi_plus(kk[j], adz, alpha) + xi_minus(kk[j], adz, alpha)) / kk[j]
        E += PI / (2 * A) * float(c @ G @ c + s @ G @ s)
    if with_kzero:
        E += -(PI / A) * float(q @ g0_exact(adz, alpha) @ q)
    if with_self:
        E -= self_energy_coef(alpha) * float(q @ q)
    return E


# ------------------------------------------------------------------ SOE


def soe_dk(pos, q, box, alpha, s, w, mx, my):
    """R_k = sum_{i != j} q_i q_j cos(k.rho_ij) dG_SOE/dk(k, |z_ij|) per mode,
    by the sorted recursion (soe_recursion.c)."""
    lib = _lib()
    pos = np.asarray(pos, float)
    N = pos.shape[0]
    c = _se._c
    x, y, z, qq = c(pos[:, 0]), c(pos[:, 1]), c(pos[:, 2]), c(q)
    Lx, Ly, _ = box
    kx, ky, _ = kvec(mx, my, Lx, Ly)
    kx, ky = c(kx), c(ky)
    s = np.asarray(s, complex)
    w = np.asarray(w, complex)
    R = np.zeros(len(kx))
    p = _se._p
    lib.oracle_kspace_soe_dk(N, p(x), p(y), p(z), p(qq), len(kx), p(kx), p(ky), alpha,
                             len(s), p(c(s.real)), p(c(s.imag)), p(c(w.real)), p(c(w.imag)),
                             p(R))
    return R


def soe_dk_direct(pos, q, box, alpha, s, w, mx, my):
    """The same R_k by direct O(N^2) pair sums of the k-derivative of the
    SOE kernel of Eq. 3.21 (no recursion), for small N."""
    pos = np.asarray(pos, float)
    q = np.asarray(q, float)
    Lx, Ly, _ = box
    x, y, z = pos[:, 0], pos[:, 1], pos[:, 2]
    adz = np.abs(z[:, None] - z[None, :])
    off = ~np.eye(q.size, dtype=bool)
    a = alpha * np.asarray(s, complex)
    w = np.asarray(w, complex)
    kx, ky, kk = kvec(mx, my, Lx, Ly)
    R = np.zeros(len(kk))
    for j in range(len(kk)):
        k = kk[j]
        # analytic derivative of each factor, written out term by term
        C = 2 * alpha * math.exp(-k * k / (4 * alpha * alpha)) / (SQPI * k)
        dC = C * (-k / (2 * alpha * alpha) - 1 / k)
        dG = 0.0
        for al, wl in zip(a, w):
            den = al * al - k * k
            f = 2 * al * np.exp(-k * adz) - 2 * k * np.exp(-al * adz)
            df = -2 * al * adz * np.exp(-k * adz) - 2 * np.exp(-al * adz)
            dG = dG + wl * (dC * f / den + C * df / den + C * f * 2 * k / (den * den))
        dG = np.real(dG) * off
        th = kx[j] * x + ky[j] * y
        cq, sq = q * np.cos(th), q * np.sin(th)
        R[j] = float(cq @ dG @ cq + sq @ dG @ sq)
    return R


def _assemble_lateral(box, alpha, q, E, mx, my, D, diag_mx, diag_my):
    q = np.asarray(q, float)
    Q = float(q @ q)
    W = lateral_from_modes(box, mx, my, D)
    Wd = lateral_from_modes(box, diag_mx, diag_my, Q * diag_dk(alpha, box, diag_mx, diag_my))
    W = _add(W, Wd)
    Uself = self_energy_coef(alpha) * Q
    W["xx"] += E + Uself
    W["yy"] += E + Uself
    return W


def soe_full_virial(pos, q, box, alpha, s, w, kc=None, tail=1e-8, modes=None):
    """Virial of the SOEwald2D long-range energy, full k-sum (soe_full)."""
    Lx, Ly, _ = box
    if modes is None:
        from .lattice import kcut_for_tail
        if kc is None:
            kc = kcut_for_tail(alpha, tail)
        mx, my = full_modes(Lx, Ly, kc)
    else:
        mx, my = modes
    out = soe_full(pos, q, box, alpha, s, w, modes=(mx, my))
    R = soe_dk(pos, q, box, alpha, s, w, mx, my)
    D = PI / (2 * Lx * Ly) * R
    W = _assemble_lateral(box, alpha, q, out["E"], mx, my, D, mx, my)
    W = _add(W, force_part(pos, out["F"]))
    out["W"] = W
    return out


def soe_rbe_virial(pos, q, box, alpha, s, w, mx, my, P=None):
    """Random-batch estimator of the virial on a given sample (soe_rbe)."""
    Lx, Ly, _ = box
    P = len(mx) if P is None else P
    out = soe_rbe(pos, q, box, alpha, s, w, mx, my, P)
    H = out["H"]
    _, _, kk = kvec(mx, my, Lx, Ly)
    R = soe_dk(pos, q, box, alpha, s, w, mx, my)
    D = PI / (2 * Lx * Ly) * (H / P) * np.exp(kk * kk / (4 * alpha * alpha)) * R
    dmx, dmy = full_modes(Lx, Ly, 14.0 * alpha)    # the j = i part over the whole lattice
    W = _assemble_lateral(box, alpha, q, out["E"], mx, my, D, dmx, dmy)
    W = _add(W, force_part(pos, out["F"]))
    out["W"] = W
    return out


# ------------------------------------------------------------------ walls


def wall_virial(pos, q, box, sigma_bot0, sigma_top0, modes=(), sb=(), st=()):
    """Virial of U_p-s = sum_i q_i phi_p-s(r_i) (Thm 2.4), particles inside
    the slab. Returns the W dict (force terms included) and U_p-s."""
    from .walls import _full_set, wall_potential
    pos = np.asarray(pos, float)
    q = np.asarray(q, float)
    Lx, Ly, Lz = box
    A = Lx * Ly
    out = wall_potential(pos, q, box, sigma_bot0, sigma_top0, modes, sb, st)
    U = out["E"]
    x, y, z = pos[:, 0], pos[:, 1], pos[:, 2]
    zb, zt = z, Lz - z
    W = force_part(pos, out["F"])
    W["xx"] += U
    W["yy"] += U
    # explicit L_z dependence of the top wall (zero mode): d phi/d Lz = -2 pi sigma_top0
    dU_dLz = float(q.sum()) * (-2 * PI * sigma_top0)
    shift = np.zeros(2)      # dU/d(shift of the top wall in x, y)
    if len(modes):
        mx, my, hb, ht = _full_set(box, modes, sb, st)
        kx, ky, kk = kvec(mx, my, Lx, Ly)
        D = np.zeros(mx.size)
        for j in range(mx.size):
            ph = np.exp(1j * (kx[j] * x + ky[j] * y))
            k = kk[j]
            eb, et = np.exp(-k * zb), np.exp(-k * zt)
            # d/dk of (2 pi/A)(1/k)(hb e^{-k zb} + ht e^{-k zt})
            dterm = (2 * PI / A) * ph * (-(hb[j] * eb + ht[j] * et) / (k * k)
                                         - (hb[j] * zb * eb + ht[j] * zt * et) / k)
            D[j] = float(q @ dterm.real)
            top = (2 * PI / A) * ph / k * ht[j] * et
            dU_dLz += float(q @ (-k * top).real)
            # the top wall's pattern shifted by d: its phase gains e^{-i k.d}
            shift[0] += float(q @ (-1j * kx[j] * top).real)
            shift[1] += float(q @ (-1j * ky[j] * top).real)
        W = _add(W, lateral_from_modes(box, mx, my, D))
    W["zz"] -= Lz * dU_dLz
    W["xz"] -= Lz * shift[0]
    W["yz"] -= Lz * shift[1]
    return {"W": W, "E": U, "F": out["F"], "phi": out["phi"]}


# ------------------------------------------------------------------ real space


def realspace_virial(pos, q, box, alpha, rc):
    """Pair virial of the real-space sum (Eq. 2.10 within |r_ij + M| <= rc)."""
    pos = np.asarray(pos, float)
    q = np.asarray(q, float)
    Lx, Ly, _ = box
    nx = int(math.ceil(rc / Lx)) + 1
    ny = int(math.ceil(rc / Ly)) + 1
    d0 = pos[:, None, :] - pos[None, :, :]
    S = np.zeros((3, 3))
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
            fr = np.where(mask, (erfc(alpha * rr) / rr
                                 + 2 * alpha / SQPI * np.exp(-(alpha * rr) ** 2)) / (rr * rr), 0.0)
            qq = q[:, None] * q[None, :] * fr
            S += 0.5 * np.einsum("ij,ija,ijb->ab", qq, d, d)
    out = realspace(pos, q, box, alpha, rc)
    W = {"xx": S[0, 0], "yy": S[1, 1], "xy": S[0, 1], "zz": S[2, 2], "xz": S[0, 2], "yz": S[1, 2]}
    return {"W": {k: float(v) for k, v in W.items()}, "E": out["E"], "F": out["F"]}
