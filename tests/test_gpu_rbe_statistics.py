"""GPU: the random-batch estimator's statistics (Section 4, Prop. 4.1).

On the unbiasedness workload (N = 1e4 charges +-1 in 40 x 40 x 50,
alpha = 0.1, P = 200; the density of the N = 1e6 workload), 1000 GPU calls
with fresh samples (the counter advances per call) must average to the full
k-sum energy of the oracle within 4 standard errors, and their variance must
equal Prop. 4.1's exact variance
  Var = (1/P) [H sum_k e^{k^2/(4 alpha^2)} phi~(k)^2 - (sum_k phi~(k))^2],
computed from the oracle's per-mode energies: a sample variance of 1000
draws has a relative standard deviation of sqrt(2/999) = 4.5 %, so the ratio
must lie in [0.8, 1.25].
"""
import math

import numpy as np
import pytest

import workloads
from oracle import lattice, soe_ewald2d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NCALL = 1000


@pytest.fixture(scope="module")
def qslab():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01521_gb300 as q
    q.load()
    return q


@pytest.fixture(scope="module")
def reference(soe16):
    """Full k-sum energy (tail 1e-12) and the exact variance of one sample."""
    sl = workloads.rbe_unbiased()
    s, w = soe16
    Lx, Ly, _ = sl.box
    kc = lattice.kcut_for_tail(sl.alpha, 1e-12)
    full = soe_ewald2d.soe_full(sl.pos, sl.q, sl.box, sl.alpha, s, w, kc=kc)
    mx, my = lattice.full_modes(Lx, Ly, kc)
    half = (mx > 0) | ((mx == 0) & (my > 0))
    pm = soe_ewald2d.per_mode_energies(sl.pos, sl.q, sl.box, sl.alpha, s, w, mx[half], my[half])
    _, _, k = lattice.kvec(mx[half], my[half], Lx, Ly)
    H = lattice.H_direct(sl.alpha, Lx, Ly)
    second = 2 * H * float((np.exp(k * k / (4 * sl.alpha ** 2)) * pm ** 2).sum())
    first = 2 * float(pm.sum())
    var1 = second - first ** 2          # variance of a single-mode sample (P = 1)
    return sl, full["E"], var1


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_unbiased_and_exact_variance(qslab, soe16, reference, prec):
    sl, E_full, var1 = reference
    P = sl.P
    dt = torch.float64 if prec == "fp64" else torch.float32
    slab = qslab.QSlab(0, prec).configure(sl.box, sl.alpha, soe16, rbe=(P, 2024))
    pos = torch.tensor(sl.pos, device="cuda", dtype=dt)
    q = torch.tensor(sl.q, device="cuda", dtype=dt)
    outs = slab.compute(pos, q, want_phi=False, want_force=False)
    E = torch.empty(NCALL, dtype=torch.float64, device="cuda")
    qslab.qslab_set_rng_state(slab.h, 2024, 0)
    for i in range(NCALL):
        slab.compute(pos, q, E[i:i + 1], None, None, want_phi=False, want_force=False)
    assert slab.status() == 0
    Es = E.cpu().numpy()
    assert len(set(Es.tolist())) > NCALL // 2          # fresh samples
    mean, sd = Es.mean(), Es.std(ddof=1)
    var_exact = var1 / P
    ratio = sd ** 2 / var_exact
    print(f"\n{prec}: mean {mean:.6f} full-k {E_full:.6f} (diff {(mean - E_full) / (sd / math.sqrt(NCALL)):+.2f} "
          f"standard errors); sample variance {sd ** 2:.6f}, Prop. 4.1 {var_exact:.6f}, ratio {ratio:.3f}")
    assert abs(mean - E_full) < 4 * sd / math.sqrt(NCALL)
    assert 0.8 < ratio < 1.25
    slab.close()
