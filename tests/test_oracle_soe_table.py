"""Pins of the SOE tables and of the oracle's SOE-kernel formulas against the
Gaussian itself and the error bounds of the paper (no GPU)."""
import math
import os

import numpy as np
import pytest

from oracle import soe_check
from paper_2403_01521_gb300.soe import load_soe, table_error

HERE = os.path.dirname(os.path.abspath(__file__))


def _printed_eps():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_soe_accuracy.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                m, e = line.split()
                out[int(m)] = float(e)
    return out


TABLES = [("conditioned", 4, 5e-4, 8), ("conditioned", 8, 2e-7, 20),
          ("conditioned", 12, 1e-8, 25), ("conditioned", 16, 1e-9, 30),
          ("conditioned", 20, 1e-10, 25), ("conditioned", 24, 1e-10, 20),
          ("accurate", 8, 1e-7, 30), ("accurate", 16, 1e-13, 300),
          ("accurate", 24, 1e-13, 200)]


@pytest.mark.parametrize("kind,M,tol,wsum", TABLES)
def test_table_sup_error(kind, M, tol, wsum):
    """Eq. 3.1: the table approximates e^{-x^2} uniformly on [0, 60]; its
    weights stay bounded (sum |w| is the rounding amplification factor)."""
    s, w = load_soe(M, kind)
    assert len(s) == M
    err, imag = soe_check.sup_error(s, w)
    assert err <= tol
    assert imag < 1e-13                      # conjugate pairs: the sum is real
    assert abs(err - table_error(M, kind)) <= 1e-3 * err
    assert np.abs(w).sum() <= wsum
    assert (s.real > 0).all()                # every e^{-alpha s z} decays (Remark 3.3)
    # closed under conjugation
    for sl, wl in zip(s, w):
        j = np.argmin(np.abs(s - np.conj(sl)))
        assert abs(s[j] - np.conj(sl)) < 1e-12 * abs(sl)
        assert abs(w[j] - np.conj(wl)) < 1e-12 * max(abs(wl), 1e-30)


def test_tables_against_printed_accuracy():
    """Section 5.1 prints M <-> eps for VPMR; the accurate matrix-pencil tables
    reach accuracies within two orders of magnitude of it."""
    for M, eps in _printed_eps().items():
        assert table_error(M, "accurate") <= 100 * eps


def test_sum_of_weights():
    """x = 0: sum_l w_l = e^0 = 1 to the table's accuracy."""
    for kind in ("conditioned", "accurate"):
        for M in (8, 16, 24):
            s, w = load_soe(M, kind)
            assert abs(w.sum() - 1.0) <= 2 * table_error(M, kind)


@pytest.mark.parametrize("M,kind", [(8, "conditioned"), (16, "conditioned"), (16, "accurate")])
@pytest.mark.parametrize("k", [0.05, 0.3, 1.0, 3.0])
def test_theorem_3_2_bounds(M, kind, k):
    """Theorem 3.2: |xi - xi_M| <= 2 alpha e^{-k^2/4a^2} eps/(sqrt(pi) k) and
    |d xi - d xi_M| <= 4 alpha e^{-k^2/4a^2} eps/sqrt(pi), uniformly in z."""
    s, w = load_soe(M)
    alpha = 0.7
    z = np.linspace(0.0, 30.0, 3001)
    e = soe_check.xi_errors(k, z, alpha, s, w)
    floor = 1e-15
    assert e["xi_plus"] <= e["bound"] + floor
    assert e["xi_minus"] <= e["bound"] + floor
    assert e["dxi_plus"] <= e["dbound"] + floor
    assert e["dxi_minus"] <= e["dbound"] + floor


def test_theorem_3_2_is_not_vacuous():
    """A table with a perturbed weight violates the bound: the check has teeth."""
    s, w = load_soe(8)
    w2 = w.copy()
    w2[0] *= 1.0 + 1e-2
    w2[1] = np.conj(w2[0])
    z = np.linspace(0.0, 30.0, 3001)
    eps_good = soe_check.sup_error(s, w)[0]
    xp, _, _, _ = soe_check.xi_M(0.3, z, 0.7, s, w2)
    from oracle.ewald2d import xi_plus
    err = np.abs(xp - xi_plus(0.3, z, 0.7)).max()
    bound = 2 * 0.7 * math.exp(-0.3 ** 2 / (4 * 0.49)) / (math.sqrt(math.pi) * 0.3) * eps_good
    assert err > bound


@pytest.mark.parametrize("M", [8, 16])
def test_erf_bound(M):
    """Eq. 3.24: |erf(alpha z) - SOE| <= 2 alpha Lz eps/sqrt(pi) on [0, Lz]."""
    s, w = load_soe(M)
    err, bound = soe_check.erf_error(0.3, 10.0, s, w)
    assert err <= bound


@pytest.mark.parametrize("M", [4, 8])
def test_fit_reproduces_the_shipped_table(M):
    """Re-run the matrix-pencil fit (50-digit arithmetic) with the shipped
    table's interval and sample count: it gives the shipped nodes and
    weights, and the shipped sup-norm error."""
    pytest.importorskip("mpmath")
    from paper_2403_01521_gb300 import soe
    info = soe.table_info(M)
    s, w = soe.fit_gaussian_soe(M, info["X"], info["samples"])
    s0, w0 = soe.load_soe(M)
    o, o0 = np.lexsort((s.imag, s.real)), np.lexsort((s0.imag, s0.real))
    assert np.abs(s[o] - s0[o0]).max() <= 1e-12 * np.abs(s0).max()
    assert np.abs(w[o] - w0[o0]).max() <= 1e-12 * np.abs(w0).max()
    assert abs(soe.sup_error(s, w) - info["sup_error"]) <= 1e-3 * info["sup_error"]
