"""The FP32 erfc of the real-space kernel: its coefficients are the ones the
committed fit produces, and the fit meets its stated error bound against
scipy's erfcx, in FP64 and in FP32 arithmetic with the reciprocal
t = 1/(1 + x/2) off by up to 2 units in the last place."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _kernel_coefficients():
    src = open(os.path.join(ROOT, "paper_2403_01521_gb300", "csrc", "qslab_real.cu")).read()
    body = src[src.index("rs_erfcx(float x)"):src.index("return t * p;")]
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    return np.array(vals[::-1])   # Horner order in the source: highest degree first


def test_erfc_fit_matches_kernel_and_bound():
    pytest.importorskip("scipy")
    from paper_2403_01521_gb300 import fit_erfcx
    coef = fit_erfcx.fit()
    ker = _kernel_coefficients()
    assert ker.shape == coef.shape
    assert np.allclose(ker, coef, rtol=1e-8, atol=1e-12)
    rel64, rel32 = fit_erfcx.check(ker, t_ulps=2)
    assert rel64 < 2e-8
    assert rel32 < 7e-7
