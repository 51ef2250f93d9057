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
complex-conjugate pairs with Re s_l > 2, so every e^{-alpha s_l z} decays.

The fitted tables are shipped as JSON in data/; ``python -m
paper_2403_01521_gb300.soe`` rewrites them (needs mpmath, which only the
build machine has). Each table records its measured sup-norm error on
[0, 60] (200001 points) and sum |w_l|, the factor by which rounding errors of
the M exponential sums can be amplified when they are combined.
"""
from __future__ import annotations

import json
import os

import numpy as np

_DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")

# (M, X, samples) per table family, chosen by sweeps of the interval X.
# "conditioned": the shortest interval whose sup error still meets 1e-7
#   (M=8) / 1e-9 (M>=12); it keeps sum |w_l| small (8 to 31), which bounds
#   how much rounding in FP32 recurrences is amplified when the M terms are
#   summed. This is the default family.
# "accurate": the interval with the smallest sup error, which reaches the
#   accuracies the paper quotes for its VPMR tables (M=8: 1e-8, M=16: 1e-14)
#   at the price of sum |w_l| of several hundred.
FIT_PLAN = {
    "conditioned": {4: (3.5, 81), 8: (4.5, 121), 12: (4.0, 121), 16: (4.0, 121),
                    20: (3.75, 161), 24: (3.5, 161)},
    "accurate": {4: (3.5, 81), 8: (5.0, 121), 12: (6.5, 121), 16: (6.0, 121),
                 20: (8.5, 161), 24: (5.0, 161)},
}


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


def _path(M: int, kind: str) -> str:
    suffix = "" if kind == "conditioned" else "_" + kind
    return os.path.join(_DATA, f"soe_gauss_M{M}{suffix}.json")


def load_soe(M: int, kind: str = "conditioned"):
    """Load a shipped table: (s, w) complex arrays of length M."""
    with open(_path(M, kind)) as fh:
        d = json.load(fh)
    s = np.array(d["s_re"]) + 1j * np.array(d["s_im"])
    w = np.array(d["w_re"]) + 1j * np.array(d["w_im"])
    return s, w


def table_info(M: int, kind: str = "conditioned") -> dict:
    with open(_path(M, kind)) as fh:
        d = json.load(fh)
    return {k: d[k] for k in ("M", "X", "samples", "sup_error", "sum_abs_w")}


def table_error(M: int, kind: str = "conditioned") -> float:
    return float(table_info(M, kind)["sup_error"])


def write_tables():
    os.makedirs(_DATA, exist_ok=True)
    for kind, plan in FIT_PLAN.items():
        for M in sorted(plan):
            X, S = plan[M]
            s, w = fit_gaussian_soe(M, X, S)
            err = sup_error(s, w)
            d = {"M": M, "X": X, "samples": S, "method": "matrix pencil", "family": kind,
                 "sup_error": err, "sum_abs_w": float(np.abs(w).sum()),
                 "s_re": [float(v.real) for v in s], "s_im": [float(v.imag) for v in s],
                 "w_re": [float(v.real) for v in w], "w_im": [float(v.imag) for v in w]}
            with open(_path(M, kind), "w") as fh:
                json.dump(d, fh, indent=1)
            print(f"{kind:11s} M={M:2d} X={X} samples={S} sup error {err:.3e} "
                  f"sum|w| {np.abs(w).sum():8.1f} min Re s {s.real.min():.3f}")


if __name__ == "__main__":
    write_tables()
