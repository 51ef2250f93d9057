"""Checks of an SOE table against the Gaussian and against the paper's
error bounds (oracle).

ORACLE: test infrastructure (see oracle/__init__.py).

  sup_error         |e^{-x^2} - sum_l w_l e^{-s_l x}| on [0, xmax] (Eq. 3.1)
  xi_errors         |xi^{+-} - xi^{+-}_M| and the z-derivatives against the
                    bounds of Theorem 3.2 (Eqs. 3.14-3.17 give xi_M; the exact
                    xi come from erfcx)
  erf_error         |erf(alpha z) - (2/sqrt(pi)) sum (w_l/s_l)(1 - e^{-alpha s_l z})|
                    against the bound of Eq. 3.24
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from .ewald2d import xi_minus, xi_plus

SQPI = math.sqrt(math.pi)


def sup_error(s, w, xmax=60.0, n=200001):
    x = np.linspace(0.0, xmax, n)
    approx = np.zeros(n, complex)
    for sl, wl in zip(s, w):
        approx += wl * np.exp(-sl * x)
    return float(np.abs(np.exp(-x * x) - approx.real).max()), float(np.abs(approx.imag).max())


def xi_M(k, z, alpha, s, w):
    """xi+_M and xi-_M (Eqs. 3.14, 3.15) and their z-derivatives (3.16, 3.17)."""
    pre = 2 * alpha / SQPI * math.exp(-k * k / (4 * alpha * alpha))
    xp = xm = dxp = dxm = 0.0
    for sl, wl in zip(s, w):
        a = alpha * sl
        e = np.exp(-a * z)
        xp = xp + wl * e / (a + k)
        xm = xm + wl * (-e / (a - k) + 2 * a * np.exp(-k * z) / (a * a - k * k))
        dxp = dxp + wl * sl * e / (a + k)
        dxm = dxm + wl * sl * (-e / (a - k) + 2 * k * np.exp(-k * z) / (a * a - k * k))
    d = -2 * alpha * alpha / SQPI * math.exp(-k * k / (4 * alpha * alpha))
    return (pre * np.real(xp), pre * np.real(xm), d * np.real(dxp), d * np.real(dxm))


def xi_errors(k, z, alpha, s, w):
    """Max errors of xi+-_M and d/dz xi+-_M on the grid z, and the Thm 3.2 bounds
    for the table's own eps (its sup error)."""
    eps, _ = sup_error(s, w)
    xp, xm, dxp, dxm = xi_M(k, z, alpha, s, w)
    ep = xi_plus(k, z, alpha)
    em = xi_minus(k, z, alpha)
    # exact derivatives: d/dz xi+ = k xi+ - (2 alpha/sqrt(pi)) e^{-k^2/4a^2 - a^2 z^2},
    #                    d/dz xi- = -k xi- + (2 alpha/sqrt(pi)) e^{-k^2/4a^2 - a^2 z^2}
    gau = 2 * alpha / SQPI * np.exp(-k * k / (4 * alpha * alpha) - (alpha * z) ** 2)
    dep = k * ep - gau
    dem = -k * em + gau
    bound = 2 * alpha * math.exp(-k * k / (4 * alpha * alpha)) / (SQPI * k) * eps
    dbound = 4 * alpha * math.exp(-k * k / (4 * alpha * alpha)) / SQPI * eps
    return {"xi_plus": float(np.abs(xp - ep).max()), "xi_minus": float(np.abs(xm - em).max()),
            "dxi_plus": float(np.abs(dxp - dep).max()), "dxi_minus": float(np.abs(dxm - dem).max()),
            "bound": bound, "dbound": dbound, "eps": eps}


def erf_error(alpha, Lz, s, w, n=20001):
    eps, _ = sup_error(s, w)
    z = np.linspace(0.0, Lz, n)
    approx = 0.0
    for sl, wl in zip(s, w):
        approx = approx + wl / sl * (1 - np.exp(-alpha * sl * z))
    approx = 2 / SQPI * np.real(approx)
    return float(np.abs(erf(alpha * z) - approx).max()), 2 * alpha * Lz / SQPI * eps
