"""Coefficients of the FP32 erfc used by the real-space kernel.

erfc(x) = e^{-x^2} erfcx(x), and for x >= 0 erfcx(x) = t P(2t - 1) with
t = 1/(1 + x/2), P a polynomial. t runs over (0, 1] as x runs over
[0, inf) and erfcx(x)/t tends to 1/(2 sqrt(pi)) as x -> inf, so P is
smooth on [-1, 1]. P is fitted by least squares in the relative error on
Chebyshev nodes in t, with erfcx from scipy in FP64.

Run: python paper_2403_01521_gb300/fit_erfcx.py   (prints the coefficients
of P, constant term first, and the maximum relative error on x in [0, 12]
in FP64 and in an FP32 Horner evaluation with t within 2 ulp)
"""
import numpy as np
from scipy.special import erfcx

P_SCALE = 0.5
DEGREE = 10


def fit(degree=DEGREE, nodes=6000):
    k = np.arange(nodes)
    t = 0.5 * (1 - np.cos(np.pi * (k + 0.5) / nodes))
    t = t[t > 1e-7]
    y = erfcx((1.0 / t - 1.0) / P_SCALE) / t
    s = 2 * t - 1
    V = np.vander(s, degree + 1, increasing=True)
    coef, *_ = np.linalg.lstsq(V / y[:, None], np.ones_like(y), rcond=None)
    return coef


def check(coef, t_ulps=0):
    """Maximum relative error of t P(2t - 1) against erfcx on x in [0, 12]:
    in FP64, and in an FP32 Horner evaluation whose t = 1/(1 + x/2) is off
    by -t_ulps, 0 and +t_ulps units in the last place (the worst of the
    three; the kernel's approximate reciprocal is within 2 ulp)."""
    x = np.linspace(0, 12, 400001)
    t = 1 / (1 + P_SCALE * x)
    rel64 = np.abs(np.polyval(coef[::-1], 2 * t - 1) * t / erfcx(x) - 1).max()
    x32 = x.astype(np.float32)
    t32 = (np.float32(1) / (np.float32(1) + np.float32(P_SCALE) * x32)).astype(np.float32)
    c32 = coef.astype(np.float32)
    rel32 = 0.0
    for u in sorted({-t_ulps, 0, t_ulps}):
        tu = (t32 + np.float32(u) * np.spacing(t32)).astype(np.float32)
        s32 = (np.float32(2) * tu - np.float32(1)).astype(np.float32)
        acc = c32[-1]
        for c in c32[::-1][1:]:
            acc = (acc * s32 + c).astype(np.float32)
        ref = erfcx(x32.astype(np.float64))
        rel32 = max(rel32, np.abs((acc * tu).astype(np.float64) / ref - 1).max())
    return rel64, rel32


if __name__ == "__main__":
    c = fit()
    r64, r32 = check(c, t_ulps=2)
    print("coefficients:", ", ".join("%.9e" % v for v in c))
    print("max relative error: FP64 %.2e, FP32 (t within 2 ulp) %.2e" % (r64, r32))
