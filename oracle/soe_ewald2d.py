"""SOE-Ewald2D long-range energy, potentials and forces by the sorted
recursion (oracle), for the full k-sum and for the random-batch estimator.

ORACLE: test infrastructure (see oracle/__init__.py).

  full k-sum (Algorithm 1, steps 4-5 and 7-9, long-range part):
      E = sum_{0<|k|<=kc} U^k_SOE + U^0_SOE - U_self
  random batch (Algorithm 2, steps 4-7 and 9, long-range part):
      E* = (H/P) sum_eta phi~^RB(k_eta) + [j = i constants] + U^0_SOE - U_self

The per-mode recursion and the k = 0 term run in oracle/soe_recursion.c;
this module chooses the modes and their weights and adds the j = i
constants of Eqs. 3.20 and 3.25 and the self term of Eq. 2.12:

  phi_i += q_i [2 D_k + 2 D_0 - 2 alpha/sqrt(pi)],   E = 1/2 sum_i q_i phi_i,

with D_k = sum_k (pi/A) erfc(k/(2 alpha))/k over the modes summed (over the
whole lattice for the random batch, whose sample covers every k) and
D_0 = -(pi/A)/(alpha sqrt(pi)).

Mode weights. Every lattice vector appears once in the full k-sum (k and -k
both listed, weight 1). A random-batch sample k_eta gets weight
(H/P) e^{k^2/(4 alpha^2)} (Eq. 4.7 with Eq. 4.9); the Gaussian cancels the one
inside C_k = 2 alpha e^{-k^2/(4 alpha^2)}/(sqrt(pi) k), so the per-mode
prefactor is (pi/A) (H/P) 2 alpha/(sqrt(pi) k).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import build as _build
from .lattice import (H_direct, diag_kspace, diag_kspace_all, diag_kzero,
                      full_modes, kcut_for_tail, kvec, sample_modes)

PI = math.pi
SQPI = math.sqrt(PI)
_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        P = ctypes.POINTER(ctypes.c_double)
        _lib.oracle_kspace_soe.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_int64,
                                           P, P, P, ctypes.c_double, ctypes.c_int,
                                           P, P, P, P, P, P, P, P]
        _lib.oracle_kspace_soe.restype = None
        _lib.oracle_kzero_soe.argtypes = [ctypes.c_int64, P, P, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, P, P, P, P, P, P]
        _lib.oracle_kzero_soe.restype = None
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def mode_prefactor(alpha, Lx, Ly, mx, my, weight):
    """gam_k = (pi/A) C_k * weight_k."""
    _, _, k = kvec(mx, my, Lx, Ly)
    C = 2 * alpha * np.exp(-k * k / (4 * alpha * alpha)) / (SQPI * k)
    return PI / (Lx * Ly) * C * weight


def rbe_prefactor(alpha, Lx, Ly, mx, my, H, P):
    """gam_k for a random-batch sample: (pi/A) (H/P) 2 alpha/(sqrt(pi) k)."""
    _, _, k = kvec(mx, my, Lx, Ly)
    return PI / (Lx * Ly) * (H / P) * 2 * alpha / (SQPI * k)


def kspace_pairs(pos, q, box, alpha, s, w, mx, my, gam):
    """k != 0 pair sums (j != i) over the modes with prefactors gam."""
    lib = _load()
    pos = np.asarray(pos, float)
    N = pos.shape[0]
    x, y, z, qq = _c(pos[:, 0]), _c(pos[:, 1]), _c(pos[:, 2]), _c(q)
    Lx, Ly, _ = box
    kx, ky, _ = kvec(mx, my, Lx, Ly)
    kx, ky, gam = _c(kx), _c(ky), _c(gam)
    s = np.asarray(s, complex)
    w = np.asarray(w, complex)
    sr, si, wr, wi = _c(s.real), _c(s.imag), _c(w.real), _c(w.imag)
    phi = np.zeros(N)
    fx, fy, fz = np.zeros(N), np.zeros(N), np.zeros(N)
    lib.oracle_kspace_soe(N, _p(x), _p(y), _p(z), _p(qq), len(kx), _p(kx), _p(ky),
                          _p(gam), alpha, len(s), _p(sr), _p(si), _p(wr), _p(wi),
                          _p(phi), _p(fx), _p(fy), _p(fz))
    return phi, np.stack([fx, fy, fz], axis=1)


def kzero_pairs(pos, q, box, alpha, s, w):
    """k = 0 pair sums (j != i): phi0 and F0_z."""
    lib = _load()
    pos = np.asarray(pos, float)
    N = pos.shape[0]
    z, qq = _c(pos[:, 2]), _c(q)
    Lx, Ly, _ = box
    s = np.asarray(s, complex)
    w = np.asarray(w, complex)
    sr, si, wr, wi = _c(s.real), _c(s.imag), _c(w.real), _c(w.imag)
    phi0 = np.zeros(N)
    fz0 = np.zeros(N)
    lib.oracle_kzero_soe(N, _p(z), _p(qq), Lx * Ly, alpha, len(s), _p(sr), _p(si),
                         _p(wr), _p(wi), _p(phi0), _p(fz0))
    return phi0, fz0


def _assemble(q, box, alpha, phik, Fk, phi0, fz0, Dk):
    Lx, Ly, _ = box
    q = np.asarray(q, float)
    diag = 2 * Dk + 2 * diag_kzero(alpha, Lx, Ly) - 2 * alpha / SQPI
    phi = phik + phi0 + q * diag
    F = Fk.copy()
    F[:, 2] += fz0
    # the three parts of E: k != 0 pairs, k = 0 pairs, j = i constants and self
    parts = (0.5 * float(q @ phik), 0.5 * float(q @ phi0), 0.5 * diag * float(q @ q))
    return {"E": 0.5 * float(q @ phi), "phi": phi, "F": F, "E_parts": parts}


def soe_full(pos, q, box, alpha, s, w, kc=None, tail=1e-8, modes=None):
    """SOEwald2D long-range part, full k-sum over 0 < |k| <= kc (or over the
    given integer modes (mx, my), which must be closed under k -> -k)."""
    Lx, Ly, _ = box
    if modes is not None:
        mx, my = (np.asarray(v, dtype=np.int64) for v in modes)
    else:
        if kc is None:
            kc = kcut_for_tail(alpha, tail)
        mx, my = full_modes(Lx, Ly, kc)
    gam = mode_prefactor(alpha, Lx, Ly, mx, my, 1.0)
    phik, Fk = kspace_pairs(pos, q, box, alpha, s, w, mx, my, gam)
    phi0, fz0 = kzero_pairs(pos, q, box, alpha, s, w)
    Dk = diag_kspace(alpha, Lx, Ly, mx, my)
    out = _assemble(q, box, alpha, phik, Fk, phi0, fz0, Dk)
    out["modes"] = (mx, my)
    return out


def soe_rbe(pos, q, box, alpha, s, w, mx, my, P=None):
    """RBSE2D long-range estimator on a given sample of modes (mx, my)."""
    Lx, Ly, _ = box
    P = len(mx) if P is None else P
    H = H_direct(alpha, Lx, Ly)
    gam = rbe_prefactor(alpha, Lx, Ly, mx, my, H, P)
    phik, Fk = kspace_pairs(pos, q, box, alpha, s, w, mx, my, gam)
    phi0, fz0 = kzero_pairs(pos, q, box, alpha, s, w)
    Dk = diag_kspace_all(alpha, Lx, Ly)
    out = _assemble(q, box, alpha, phik, Fk, phi0, fz0, Dk)
    out["H"] = H
    return out


def soe_rbe_seeded(pos, q, box, alpha, s, w, P, seed, call):
    """RBSE2D estimator with the modes drawn by the oracle's own sampler."""
    Lx, Ly, _ = box
    mx, my = sample_modes(P, seed, call, alpha, Lx, Ly)
    out = soe_rbe(pos, q, box, alpha, s, w, mx, my, P)
    out["modes"] = (mx, my)
    return out


def per_mode_energies(pos, q, box, alpha, s, w, mx, my):
    """phi~(k) for each listed mode: the j != i part of U^k_SOE (Eq. 3.20),
    one pass per mode. Used by the variance check of Prop. 4.1."""
    Lx, Ly, _ = box
    q = np.asarray(q, float)
    gam1 = mode_prefactor(alpha, Lx, Ly, mx, my, 1.0)
    out = np.zeros(len(mx))
    for m in range(len(mx)):
        phik, _ = kspace_pairs(pos, q, box, alpha, s, w, mx[m:m + 1], my[m:m + 1], gam1[m:m + 1])
        out[m] = 0.5 * float(q @ phik)
    return out
