"""Sum-of-exponentials (SOE) tables for the Gaussian, e^{-x^2} ~ sum_l w_l e^{-s_l|x|}.

The method needs, for a precision eps, weights w_l and exponents s_l with
Re s_l > 0 such that |e^{-x^2} - sum_l w_l e^{-s_l |x|}| <= eps for all real x
(Eq. 3.1; the Gaussian factor of Eq. 3.18 is approximated in the variable
x = alpha*t, Eq. 3.6). The paper builds them with the VPMR method, which it does
not describe; this module builds them with the matrix-pencil method
(Hua & Sarkar, IEEE Trans. ASSP 38 (1990)) instead:

  1. sample f(x)=e^{-x^2} at x_n = n h, n = 0..S-1, on [0, X];
  2. form the Hankel matrix Y[i, j] = f(x_{i+j}) and take its SVD;
  3. keep the M dominant right singular vectors V; the eigenvalues z_l of the
     pencil pinv(V[:, :-1]^T) V[:, 1:]^T are e^{-s_l h}, so s_l = -log(z_l)/h;
  4. solve the least-squares problem f(x_n) = sum_l w_l z_l^n for w.

Steps 2-4 run in 50-digit arithmetic (mpmath) because the Hankel matrix is
numerically rank-deficient in double precision. All exponents come out in
complex-conjugate pairs with Re s_l > 3, so every e^{-alpha s_l z} decays.

The fitted tables are shipped as JSON in data/; ``python -m
paper_2403_01521_gb300.soe`` rewrites them (needs mpmath, which only the
build machine has). Each table records its measured sup-norm error on
[0, 60] (200001 points).
"""
from __future__ import annotations

import json
import os

import numpy as np

_DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")

# (M, X, samples) chosen by a sweep of the interval length X.
FIT_PLAN = {4: (3.5, 81), 8: (5.0, 121), 12: (6.5, 121), 16: (8.0, 121),
            20: (8.5, 161), 24: (9.0, 161)}


def fit_gaussian_soe(M: int, X: float, samples: int, dps: int = 50):
    """Matrix-pencil SOE fit of e^{-x^2} on [0, X]; returns complex s, w."""
    import mpmath as mp

    mp.mp.dps = dps
    h = mp.mpf(X) / (samples - 1)
    f = [mp.exp(-(n * h) ** 2) for n in range(samples)]
    L = samples // 2
    rows = samples - L
    Y = mp.matrix(rows, L + 1)
    for i in range(rows):
        for j in range(L + 1):
            Y[i, j] = f[i + j]
    _, _, V = mp.svd_r(Y)
    V1 = mp.matrix(M, L)
    V2 = mp.matrix(M, L)
    for i in range(M):
        for j in range(L):
            V1[i, j] = V[i, j]
            V2[i, j] = V[i, j + 1]
    A = V1.T
    B = V2.T
    pencil = mp.inverse(A.T * A) * A.T * B
    z, _ = mp.eig(pencil)
    z = list(z)
    Vd = mp.matrix(samples, M)
    for n in range(samples):
        for l in range(M):
            Vd[n, l] = z[l] ** n
    w = mp.lu_solve(Vd.H * Vd, Vd.H * mp.matrix(f))
    s = np.array([complex(-mp.log(zz) / h) for zz in z])
    w = np.array([complex(x) for x in w])
    return _conjugate_pairs(s, w)


def _conjugate_pairs(s, w):
    """Order nodes as (pair, pair, ...) with exact conjugate symmetry."""
    order = np.lexsort((s.imag, s.real))
    s, w = s[order], w[order]
    used = np.zeros(len(s), bool)
    out_s, out_w = [], []
    for i in range(len(s)):
        if used[i]:
            continue
        used[i] = True
        if abs(s[i].imag) < 1e-12 * abs(s[i]):
            out_s.append(complex(s[i].real, 0.0))
            out_w.append(complex(w[i].real, 0.0))
            continue
        d = np.abs(s - np.conj(s[i]))
        d[used] = np.inf
        j = int(np.argmin(d))
        used[j] = True
        sp = s[i] if s[i].imag > 0 else s[j]
        wp = w[i] if s[i].imag > 0 else w[j]
        ws = 0.5 * (wp + np.conj(w[j] if s[i].imag > 0 else w[i]))
        ss = 0.5 * (sp + np.conj(s[j] if s[i].imag > 0 else s[i]))
        out_s += [ss, np.conj(ss)]
        out_w += [ws, np.conj(ws)]
    return np.array(out_s), np.array(out_w)


def sup_error(s, w, xmax: float = 60.0, n: int = 200001) -> float:
    x = np.linspace(0.0, xmax, n)
    approx = np.zeros_like(x)
    for sl, wl in zip(s, w):
        approx += (wl * np.exp(-sl * x)).real
    return float(np.abs(np.exp(-x * x) - approx).max())


def load_soe(M: int):
    """Load the shipped table for M terms: (s, w) complex arrays."""
    path = os.path.join(_DATA, f"soe_gauss_M{M}.json")
    with open(path) as fh:
        d = json.load(fh)
    s = np.array(d["s_re"]) + 1j * np.array(d["s_im"])
    w = np.array(d["w_re"]) + 1j * np.array(d["w_im"])
    return s, w


def table_error(M: int) -> float:
    path = os.path.join(_DATA, f"soe_gauss_M{M}.json")
    with open(path) as fh:
        return float(json.load(fh)["sup_error"])


def write_tables(Ms=None):
    os.makedirs(_DATA, exist_ok=True)
    for M in (Ms or sorted(FIT_PLAN)):
        X, S = FIT_PLAN[M]
        s, w = fit_gaussian_soe(M, X, S)
        err = sup_error(s, w)
        d = {"M": M, "X": X, "samples": S, "method": "matrix pencil",
             "sup_error": err,
             "s_re": [float(v.real) for v in s], "s_im": [float(v.imag) for v in s],
             "w_re": [float(v.real) for v in w], "w_im": [float(v.imag) for v in w]}
        with open(os.path.join(_DATA, f"soe_gauss_M{M}.json"), "w") as fh:
            json.dump(d, fh, indent=1)
        print(f"M={M:2d} X={X} samples={S} sup error {err:.3e} "
              f"min Re s {s.real.min():.3f}")


if __name__ == "__main__":
    write_tables()
