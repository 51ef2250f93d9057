"""Pins of the oracle's lattice helpers, RNG, k-sampler and random-batch
estimator (no GPU)."""
import math

import numpy as np
import pytest

import workloads
from oracle import lattice, soe_ewald2d


def test_full_modes_definition():
    """Every lattice vector with 0 < |k| <= kc, closed under k -> -k."""
    Lx, Ly, kc = 30.0, 23.0, 1.7
    mx, my = lattice.full_modes(Lx, Ly, kc)
    got = set(zip(mx.tolist(), my.tolist()))
    want = set()
    for a in range(-40, 41):
        for b in range(-40, 41):
            if (a, b) != (0, 0) and (2 * math.pi * a / Lx) ** 2 + (2 * math.pi * b / Ly) ** 2 <= kc * kc:
                want.add((a, b))
    assert got == want
    assert all((-a, -b) in got for a, b in got)


def test_mode_counts_of_workloads():
    """k_c = 2 alpha sqrt(ln 1e8) (Gaussian tail 1e-8) gives 'a few hundred'
    modes for the N = 1000 workload."""
    for sl, n in ((workloads.small_full(), 480),):
        kc = lattice.kcut_for_tail(sl.alpha, sl.tail)
        assert abs(math.exp(-kc * kc / (4 * sl.alpha ** 2)) - sl.tail) < 1e-20
        assert len(lattice.full_modes(sl.box[0], sl.box[1], kc)[0]) == n


@pytest.mark.parametrize("alpha,L", [(0.3, 30.0), (0.25, 100.0), (0.1, 400.0), (0.1, 40.0), (0.2, 200.0)])
def test_H_poisson_form(alpha, L):
    """Eq. 4.5 summed directly equals the Poisson form with alpha^2; the form
    as printed (alpha to the first power) does not."""
    Hd = lattice.H_direct(alpha, L, L)
    assert abs(Hd - lattice.H_poisson(alpha, L, L, 2)) < 1e-12 * Hd
    assert abs(Hd - lattice.H_poisson(alpha, L, L, 1)) > 1e-2 * Hd


def test_H_bound():
    """Eq. 4.24: H <= 2 alpha^2 Lx Ly/sqrt(pi)."""
    for alpha, L in [(0.3, 30.0), (0.1, 400.0)]:
        assert lattice.H_direct(alpha, L, L) <= 2 * alpha ** 2 * L * L / math.sqrt(math.pi)


def test_philox_matches_numpy():
    """Philox4x64-10 against numpy's library implementation. numpy advances its
    256-bit counter before each block, so block c of numpy is our counter c+1."""
    key = np.array([0x0123456789ABCDEF, 0xFEDCBA9876543210], np.uint64)
    ctr0 = np.array([0xFFFFFFFFFFFFFFF0, 7, 0, 3], np.uint64)
    g = np.random.Philox(key=key, counter=ctr0)
    raw = g.random_raw(4 * 20).reshape(20, 4)
    ctrs = np.zeros((20, 4), np.uint64)
    for b in range(20):
        c = int(ctr0[0]) + b + 1
        carry = c >> 64
        ctrs[b] = [c & (2**64 - 1), int(ctr0[1]) + carry, 0, 3]
    ours = lattice.philox4x64_10(ctrs, np.tile(key, (20, 1)))
    assert (ours == raw).all()


def test_sampler_distribution():
    """Chi-square goodness of fit of the i.i.d. k-sampler against h(k)."""
    alpha, Lx, Ly = 0.3, 30.0, 30.0
    n = 200_000
    mx, my = lattice.sample_modes(n, seed=12345, call=0, alpha=alpha, Lx=Lx, Ly=Ly)
    assert not ((mx == 0) & (my == 0)).any()
    keys, counts = np.unique(np.stack([mx, my], 1), axis=0, return_counts=True)
    cnt = dict(zip(map(tuple, keys.tolist()), counts.tolist()))
    R = lattice.axis_mmax(alpha, Lx)
    gx, gy = np.meshgrid(np.arange(-R, R + 1), np.arange(-R, R + 1), indexing="ij")
    gx, gy = gx.ravel(), gy.ravel()
    nz = ~((gx == 0) & (gy == 0))
    gx, gy = gx[nz], gy[nz]
    p = lattice.h_pmf(alpha, Lx, Ly, gx, gy)
    exp_ = n * p
    obs = np.array([cnt.get((a, b), 0) for a, b in zip(gx.tolist(), gy.tolist())])
    big = exp_ >= 10
    chi2 = float((((obs - exp_) ** 2 / exp_)[big]).sum())
    dof = int(big.sum()) - 1
    # 5-sigma acceptance on the chi-square
    assert abs(chi2 - dof) < 5 * math.sqrt(2 * dof)
    assert obs[~big].sum() < 5 * max(exp_[~big].sum(), 1.0) + 50


def test_sampler_is_reproducible_and_counter_based():
    a = lattice.sample_modes(50, 7, 3, 0.1, 400.0, 400.0)
    b = lattice.sample_modes(50, 7, 3, 0.1, 400.0, 400.0)
    c = lattice.sample_modes(50, 7, 4, 0.1, 400.0, 400.0)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()
    assert not ((a[0] == c[0]).all() and (a[1] == c[1]).all())
    # the first 20 draws do not depend on how many are requested
    d = lattice.sample_modes(20, 7, 3, 0.1, 400.0, 400.0)
    assert (d[0] == a[0][:20]).all() and (d[1] == a[1][:20]).all()


@pytest.fixture(scope="module")
def rbe_system():
    return workloads.uniform_slab(80, (12.0, 12.0, 6.0), 21, alpha=0.4)


def test_rbe_on_full_lattice_weights_equals_full_sum(rbe_system, soe16):
    """Importance sampling identity: averaging the estimator over the exact
    distribution h (every lattice vector weighted by h(k)) gives the full sum
    (Eq. 4.4 with Eq. 4.7)."""
    s, w = soe16
    sl = rbe_system
    Lx, Ly, _ = sl.box
    kc = lattice.kcut_for_tail(sl.alpha, 1e-16)
    mx, my = lattice.full_modes(Lx, Ly, kc)
    full = soe_ewald2d.soe_full(sl.pos, sl.q, sl.box, sl.alpha, s, w, kc=kc)
    H = lattice.H_direct(sl.alpha, Lx, Ly)
    h = lattice.h_pmf(sl.alpha, Lx, Ly, mx, my)
    # weight each mode by P*h so that (H/P) e^{k^2/4a^2} * P h = 1
    gam = soe_ewald2d.rbe_prefactor(sl.alpha, Lx, Ly, mx, my, H, 1) * h
    pk, Fk = soe_ewald2d.kspace_pairs(sl.pos, sl.q, sl.box, sl.alpha, s, w, mx, my, gam)
    gam1 = soe_ewald2d.mode_prefactor(sl.alpha, Lx, Ly, mx, my, 1.0)
    pk1, Fk1 = soe_ewald2d.kspace_pairs(sl.pos, sl.q, sl.box, sl.alpha, s, w, mx, my, gam1)
    assert np.abs(pk - pk1).max() < 1e-12 * np.abs(pk1).max()
    assert np.abs(Fk - Fk1).max() < 1e-12 * np.abs(Fk1).max()
    # and the whole-lattice diagonal equals the full-k diagonal at a 1e-16 tail
    assert abs(lattice.diag_kspace_all(sl.alpha, Lx, Ly)
               - lattice.diag_kspace(sl.alpha, Lx, Ly, mx, my)) < 1e-14
    assert np.isfinite(full["E"])


@pytest.mark.slow
def test_rbe_unbiased_and_variance(rbe_system, soe16):
    """Prop. 4.1: the random-batch energy is unbiased, and its variance equals
    (1/P)[H sum_k e^{k^2/4a^2} phi~(k)^2 - (sum_k phi~(k))^2]."""
    s, w = soe16
    sl = rbe_system
    Lx, Ly, _ = sl.box
    P, nseed = 10, 400
    kc = lattice.kcut_for_tail(sl.alpha, 1e-16)
    full = soe_ewald2d.soe_full(sl.pos, sl.q, sl.box, sl.alpha, s, w, kc=kc)
    Es = np.array([soe_ewald2d.soe_rbe_seeded(sl.pos, sl.q, sl.box, sl.alpha, s, w, P, 99, c)["E"]
                   for c in range(nseed)])
    mean, sd = Es.mean(), Es.std(ddof=1)
    assert abs(mean - full["E"]) < 4 * sd / math.sqrt(nseed)
    # exact variance from per-mode energies on the half lattice (phi~(k) = phi~(-k))
    mx, my = lattice.full_modes(Lx, Ly, lattice.kcut_for_tail(sl.alpha, 1e-12))
    half = (mx > 0) | ((mx == 0) & (my > 0))
    pm = soe_ewald2d.per_mode_energies(sl.pos, sl.q, sl.box, sl.alpha, s, w, mx[half], my[half])
    _, _, k = lattice.kvec(mx[half], my[half], Lx, Ly)
    H = lattice.H_direct(sl.alpha, Lx, Ly)
    second = 2 * H * float((np.exp(k * k / (4 * sl.alpha ** 2)) * pm ** 2).sum())
    first = 2 * float(pm.sum())
    var_exact = (second - first ** 2) / P
    ratio = sd ** 2 / var_exact
    # sample variance of 400 draws: relative sd ~ sqrt(2/399) ~ 7%
    assert 0.7 < ratio < 1.4


# ------------------------------------------------ Metropolis sampler (App. G)


@pytest.mark.parametrize("aL", [1.5, 7.0, 30.0])
def test_mh_proposal_pmf_is_the_rounded_normal(aL):
    """q(m) of App. G is the mass of N(0, (alpha L)^2/(2 pi^2)) on
    [m - 1/2, m + 1/2]: numerical quadrature of the normal density."""
    from scipy.integrate import quad
    sig = aL / (math.sqrt(2.0) * math.pi)
    dens = lambda t: math.exp(-0.5 * (t / sig) ** 2) / (sig * math.sqrt(2 * math.pi))
    ms = np.arange(0, int(6 * sig) + 3)
    q = lattice.proposal_pmf(ms, aL, 1.0)
    for m, qm in zip(ms, q):
        ref = quad(dens, m - 0.5, m + 0.5, epsabs=0, epsrel=1e-13)[0]
        assert abs(qm - ref) <= 1e-11 * ref + 1e-300
    qall = lattice.proposal_pmf(np.arange(0, int(10 * sig) + 3), aL, 1.0)
    assert abs(qall[0] + 2 * qall[1:].sum() - 1.0) < 1e-12


def test_mh_proposals_follow_q():
    """The Box-Muller proposals, rounded, follow q(mx) q(my): chi-square."""
    alpha, Lx, Ly = 0.3, 10.0, 15.0
    n = 100_000
    w = lattice._mh_words(np.arange(n), 0, 5, 99, 0)
    mx, my = lattice.mh_proposal(w[:, 0], w[:, 1], alpha, Lx, Ly)
    for m, L in ((mx, Lx), (my, Ly)):
        vals, cnt = np.unique(m, return_counts=True)
        exp_ = n * lattice.proposal_pmf(vals, alpha, L)
        big = exp_ >= 10
        chi2 = float((((cnt - exp_) ** 2 / exp_)[big]).sum())
        dof = int(big.sum()) - 1
        assert abs(chi2 - dof) < 5 * math.sqrt(2 * dof)


def test_mh_chain_targets_h():
    """The chain's states follow h(k) (origin excluded): chi-square on a long
    thinned chain of a small box (alpha L = 3, acceptance ~0.67, where a
    wrong acceptance ratio shows), with the variance allowance of a
    correlated chain."""
    alpha, Lx, Ly = 0.25, 12.0, 12.0
    n = 40_000
    mx, my, rate = lattice.metropolis_modes(n, 3, 1, alpha, Lx, Ly, thin=4, return_rate=True)
    assert 0.5 < rate < 0.8
    assert not ((mx == 0) & (my == 0)).any()
    keys, counts = np.unique(np.stack([mx, my], 1), axis=0, return_counts=True)
    cnt = dict(zip(map(tuple, keys.tolist()), counts.tolist()))
    R = lattice.axis_mmax(alpha, Lx)
    gx, gy = np.meshgrid(np.arange(-R, R + 1), np.arange(-R, R + 1), indexing="ij")
    gx, gy = gx.ravel(), gy.ravel()
    nz = ~((gx == 0) & (gy == 0))
    gx, gy = gx[nz], gy[nz]
    exp_ = n * lattice.h_pmf(alpha, Lx, Ly, gx, gy)
    obs = np.array([cnt.get((a, b), 0) for a, b in zip(gx.tolist(), gy.tolist())])
    big = exp_ >= 10
    chi2 = float((((obs - exp_) ** 2 / exp_)[big]).sum())
    dof = int(big.sum()) - 1
    assert chi2 < 1.6 * dof + 5 * math.sqrt(2 * dof)
    # the proposal alone (no acceptance step) is far from h here
    w = lattice._mh_words(np.arange(n), 0, 1, 3, 0)
    px, py = lattice.mh_proposal(w[:, 0], w[:, 1], alpha, Lx, Ly)
    keep = ~((px == 0) & (py == 0))
    kp, cp = np.unique(np.stack([px[keep], py[keep]], 1), axis=0, return_counts=True)
    cntp = dict(zip(map(tuple, kp.tolist()), cp.tolist()))
    obsp = np.array([cntp.get((a, b), 0) for a, b in zip(gx.tolist(), gy.tolist())]) * n / keep.sum()
    chi2p = float((((obsp - exp_) ** 2 / exp_)[big]).sum())
    assert chi2p > 10 * chi2


@pytest.mark.parametrize("alpha,L", [(0.1, 400.0), (0.3, 100.0), (0.25, 40.0)])
def test_mh_acceptance_above_90_percent(alpha, L):
    """App. G reports acceptance rates above 90% on its workloads."""
    _, _, rate = lattice.metropolis_modes(2000, 5, 0, alpha, L, L, return_rate=True)
    assert rate > 0.9


def test_mh_thinning_and_counter():
    a = lattice.metropolis_modes(50, 7, 3, 0.25, 20.0, 20.0, thin=3)
    b = lattice.metropolis_modes(150, 7, 3, 0.25, 20.0, 20.0, thin=1)
    assert (a[0] == b[0][2::3]).all() and (a[1] == b[1][2::3]).all()
    c = lattice.metropolis_modes(50, 7, 4, 0.25, 20.0, 20.0, thin=3)
    d = lattice.metropolis_modes(50, 7, 3, 0.25, 20.0, 20.0, thin=3, stream=1)
    for e in (c, d):
        assert not ((a[0] == e[0]).all() and (a[1] == e[1]).all())


def test_rbe_with_mh_samples_is_unbiased(rbe_system, soe16):
    """The random-batch energy with Metropolis samples averages to the
    full-k energy (over 300 calls of one seed)."""
    s, w = soe16
    sl = rbe_system
    Lx, Ly, _ = sl.box
    kc = lattice.kcut_for_tail(sl.alpha, 1e-14)
    full = soe_ewald2d.soe_full(sl.pos, sl.q, sl.box, sl.alpha, s, w, kc=kc)["E"]
    es = []
    for call in range(300):
        mx, my = lattice.metropolis_modes(20, 13, call, sl.alpha, Lx, Ly, thin=2)
        es.append(soe_ewald2d.soe_rbe(sl.pos, sl.q, sl.box, sl.alpha, s, w, mx, my)["E"])
    es = np.array(es)
    assert abs(es.mean() - full) < 5 * es.std() / math.sqrt(es.size)
