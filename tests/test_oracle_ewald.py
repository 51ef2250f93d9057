"""Pins of the oracle's Ewald2D and SOE-recursion formulas (no GPU).

Each check compares the oracle with something other than itself: a second,
independent formula (brute pair sums, the exact erfc kernel, direct image
sums), an invariance of the physics, or finite differences.
"""
import numpy as np
import pytest

import workloads
from oracle import ewald2d, lattice, soe_ewald2d


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.fixture(scope="module")
def small():
    return workloads.uniform_slab(60, (10.0, 10.0, 5.0), 7, alpha=0.6)


@pytest.fixture(scope="module")
def small_modes(small):
    kc = lattice.kcut_for_tail(small.alpha, 1e-8)
    return kc, lattice.full_modes(small.box[0], small.box[1], kc)


def test_recursion_equals_direct_soe_pairs(small, small_modes, soe16):
    """Eqs. 3.28-3.30 (sorted recursion, both directions) are exact algebra for
    the SOE pair kernels of Eqs. 3.21 and 3.26: they must agree with the
    O(N^2) pair sum to rounding."""
    s, w = soe16
    _, (mx, my) = small_modes
    Lx, Ly, _ = small.box
    gam = soe_ewald2d.mode_prefactor(small.alpha, Lx, Ly, mx, my, 1.0)
    d = ewald2d.soe_pair_direct(small.pos, small.q, small.box, small.alpha, s, w, mx, my, gam)
    pk, Fk = soe_ewald2d.kspace_pairs(small.pos, small.q, small.box, small.alpha, s, w, mx, my, gam)
    p0, f0 = soe_ewald2d.kzero_pairs(small.pos, small.q, small.box, small.alpha, s, w)
    assert _rel(pk, d["phi_k"]) < 1e-12
    assert _rel(Fk, d["F_k"]) < 1e-12
    assert _rel(p0, d["phi_0"]) < 1e-12
    assert _rel(f0, d["fz_0"]) < 1e-11


def test_recursion_with_ties_and_tiny_n(soe16):
    """N = 2, 3 and exactly coincident z values (the recursion's edge cases)."""
    s, w = soe16
    box = (8.0, 9.0, 4.0)
    for pos, q in [
        (np.array([[1.0, 2.0, 1.5], [3.0, 7.0, 2.5]]), np.array([1.0, -1.0])),
        (np.array([[1.0, 2.0, 1.5], [3.0, 7.0, 1.5], [5.0, 1.0, 3.0]]), np.array([1.0, -2.0, 1.0])),
        (np.array([[1.0, 2.0, 0.0], [3.0, 7.0, 4.0], [6.0, 5.0, 0.0], [2.0, 2.0, 4.0]]),
         np.array([1.0, -1.0, 1.0, -1.0])),
    ]:
        mx, my = lattice.full_modes(box[0], box[1], lattice.kcut_for_tail(0.5, 1e-8))
        gam = soe_ewald2d.mode_prefactor(0.5, box[0], box[1], mx, my, 1.0)
        d = ewald2d.soe_pair_direct(pos, q, box, 0.5, s, w, mx, my, gam)
        pk, Fk = soe_ewald2d.kspace_pairs(pos, q, box, 0.5, s, w, mx, my, gam)
        p0, f0 = soe_ewald2d.kzero_pairs(pos, q, box, 0.5, s, w)
        assert _rel(pk, d["phi_k"]) < 1e-12
        assert _rel(Fk[:, :2], d["F_k"][:, :2]) < 1e-12
        # ties: the k!=0 SOE kernel has zero slope at z=0; the k=0 one has
        # slope -sum(w s)/sqrt(pi) ~ eps, so the tie order moves F_z by ~eps
        assert np.abs(Fk[:, 2] - d["F_k"][:, 2]).max() < 1e-12
        assert _rel(p0, d["phi_0"]) < 1e-12
        assert np.abs(f0 - d["fz_0"]).max() < 1e-9


def test_soe_equals_exact_ewald(small, small_modes, soe16):
    """SOEwald2D vs Ewald2D (Thm 3.3): with eps ~ 4e-13 they agree to ~1e-12."""
    s, w = soe16
    kc, (mx, my) = small_modes
    ex = ewald2d.ewald2d_longrange(small.pos, small.q, small.box, small.alpha, mx, my)
    so = soe_ewald2d.soe_full(small.pos, small.q, small.box, small.alpha, s, w, kc=kc)
    assert abs(so["E"] - ex["E"]) < 1e-12 * abs(ex["E"])
    assert _rel(so["phi"], ex["phi"]) < 1e-11
    assert _rel(so["F"], ex["F"]) < 1e-10


def test_soe_error_grows_with_eps(small, small_modes, soe8):
    """With M = 8 (eps ~ 5e-8) the SOE energy error is visible but bounded by
    the Thm 3.3 scale eps * Q * O(1)."""
    s, w = soe8
    kc, (mx, my) = small_modes
    ex = ewald2d.ewald2d_longrange(small.pos, small.q, small.box, small.alpha, mx, my)
    so = soe_ewald2d.soe_full(small.pos, small.q, small.box, small.alpha, s, w, kc=kc)
    Q = float((small.q ** 2).sum())
    err = abs(so["E"] - ex["E"])
    assert 1e-14 * Q < err < 50 * 5e-8 * Q


def test_alpha_independence(small):
    """Ewald splitting: Eq. 2.9's total (long-range + real-space) does not
    depend on alpha when both truncations are negligible."""
    totals, forces = [], []
    for alpha in (0.5, 0.6, 0.7, 0.8):
        mx, my = lattice.full_modes(small.box[0], small.box[1], lattice.kcut_for_tail(alpha, 1e-15))
        ex = ewald2d.ewald2d_longrange(small.pos, small.q, small.box, alpha, mx, my)
        rs = ewald2d.realspace(small.pos, small.q, small.box, alpha, 6.2 / alpha)
        totals.append(ex["E"] + rs["E"])
        forces.append(ex["F"] + rs["F"])
    totals = np.array(totals)
    assert np.ptp(totals) < 1e-12 * abs(totals[0])
    for f in forces[1:]:
        assert _rel(f, forces[0]) < 1e-11


def test_image_sum_pins_the_constant():
    """Eq. 2.8 summed over images in growing discs (the symmetric shape of
    Thm 2.1), extrapolated in 1/R, equals the Ewald2D total, including the
    k = 0 constant (the diagonal of Eq. 3.25 read as -sqrt(pi) Q/(alpha A))."""
    sl = workloads.uniform_slab(4, (10.0, 10.0, 5.0), 11, alpha=0.6)
    mx, my = lattice.full_modes(10.0, 10.0, lattice.kcut_for_tail(0.6, 1e-16))
    ex = ewald2d.ewald2d_longrange(sl.pos, sl.q, sl.box, 0.6, mx, my)
    rs = ewald2d.realspace(sl.pos, sl.q, sl.box, 0.6, 7.0 / 0.6)
    total = ex["E"] + rs["E"]
    Einf, _ = ewald2d.image_sum_extrapolated(sl.pos, sl.q, sl.box, [1000, 2000, 4000, 8000])
    assert abs(Einf - total) < 3e-7 * abs(total)
    # the constant as printed would be off by (pi - sqrt(pi)) Q/(alpha A)
    Q = float((sl.q ** 2).sum())
    assert (np.pi - np.sqrt(np.pi)) * Q / (0.6 * 100.0) > 1e3 * abs(Einf - total)


def _energy(pos, q, box, alpha, s, w, kc):
    return soe_ewald2d.soe_full(pos, q, box, alpha, s, w, kc=kc)


def test_forces_are_minus_gradient(small, small_modes, soe16):
    """F = -dE/dr by central differences (h = 1e-5 L), SOE recursion path."""
    s, w = soe16
    kc, _ = small_modes
    base = _energy(small.pos, small.q, small.box, small.alpha, s, w, kc)
    h = 1e-5 * 5.0
    for i in (0, 17, 42):
        for c in range(3):
            p1 = small.pos.copy()
            p2 = small.pos.copy()
            p1[i, c] += h
            p2[i, c] -= h
            e1 = _energy(p1, small.q, small.box, small.alpha, s, w, kc)["E"]
            e2 = _energy(p2, small.q, small.box, small.alpha, s, w, kc)["E"]
            fd = -(e1 - e2) / (2 * h)
            assert abs(fd - base["F"][i, c]) < 1e-7 * max(1.0, abs(base["F"][i, c]))


def test_exact_forces_are_minus_gradient(small, small_modes):
    """Same check for the exact Ewald2D oracle (Lemma 2.1)."""
    _, (mx, my) = small_modes
    base = ewald2d.ewald2d_longrange(small.pos, small.q, small.box, small.alpha, mx, my)
    h = 1e-5 * 5.0
    for i in (3, 33):
        for c in range(3):
            p1 = small.pos.copy()
            p2 = small.pos.copy()
            p1[i, c] += h
            p2[i, c] -= h
            e1 = ewald2d.ewald2d_longrange(p1, small.q, small.box, small.alpha, mx, my)["E"]
            e2 = ewald2d.ewald2d_longrange(p2, small.q, small.box, small.alpha, mx, my)["E"]
            assert abs(-(e1 - e2) / (2 * h) - base["F"][i, c]) < 1e-7 * max(1.0, abs(base["F"][i, c]))


def test_potential_is_dE_dq(small, small_modes, soe16):
    """phi_i = dE/dq_i (E is a quadratic form in q), by central differences."""
    s, w = soe16
    kc, _ = small_modes
    base = _energy(small.pos, small.q, small.box, small.alpha, s, w, kc)
    h = 1e-4
    for i in (1, 30):
        q1 = small.q.copy()
        q2 = small.q.copy()
        q1[i] += h
        q2[i] -= h
        e1 = _energy(small.pos, q1, small.box, small.alpha, s, w, kc)["E"]
        e2 = _energy(small.pos, q2, small.box, small.alpha, s, w, kc)["E"]
        assert abs((e1 - e2) / (2 * h) - base["phi"][i]) < 1e-8


def test_invariances(small, small_modes, soe16):
    s, w = soe16
    kc, _ = small_modes
    box = small.box
    base = _energy(small.pos, small.q, box, small.alpha, s, w, kc)
    E0 = base["E"]
    F0 = base["F"]
    # zero net force (Newton's third law)
    assert np.abs(F0.sum(0)).max() < 1e-12 * np.abs(F0).sum()
    # common shift in x,y (periodic) and in z (inside the slab)
    p = small.pos.copy()
    p[:, 0] = (p[:, 0] + 3.3) % box[0]
    p[:, 1] = (p[:, 1] + 7.1) % box[1]
    zs = 0.5 * (box[2] - p[:, 2].max())
    p[:, 2] += zs
    e = _energy(p, small.q, box, small.alpha, s, w, kc)
    assert abs(e["E"] - E0) < 1e-12 * abs(E0)
    assert _rel(e["F"], F0) < 1e-10
    # reflection z -> Lz - z flips F_z
    p = small.pos.copy()
    p[:, 2] = box[2] - p[:, 2]
    e = _energy(p, small.q, box, small.alpha, s, w, kc)
    assert abs(e["E"] - E0) < 1e-12 * abs(E0)
    assert _rel(e["F"][:, 2], -F0[:, 2]) < 1e-10
    # particle permutation
    perm = np.random.default_rng(0).permutation(small.N)
    e = _energy(small.pos[perm], small.q[perm], box, small.alpha, s, w, kc)
    assert abs(e["E"] - E0) < 1e-12 * abs(E0)
    assert _rel(e["F"], F0[perm]) < 1e-12
    # E(lambda q) = lambda^2 E
    e = _energy(small.pos, 1.7 * small.q, box, small.alpha, s, w, kc)
    assert abs(e["E"] - 1.7 ** 2 * E0) < 1e-12 * abs(E0)


def test_large_alpha_kzero_limit():
    """g0(z) -> |z| as alpha -> infinity: the k = 0 mode becomes the field of
    charged sheets (Eq. 2.7 / Prop. 2.2)."""
    z = np.linspace(0.5, 5.0, 10)
    assert np.abs(ewald2d.g0_exact(z, 50.0) - z).max() < 1e-2
    assert np.abs(ewald2d.g0_exact(z, 500.0) - z).max() < 2e-3


@pytest.mark.slow
def test_small_full_workload_soe_vs_exact(soe16):
    """The N = 1000 parity workload: SOE recursion vs exact Ewald2D."""
    sl = workloads.small_full()
    kc = lattice.kcut_for_tail(sl.alpha, sl.tail)
    mx, my = lattice.full_modes(sl.box[0], sl.box[1], kc)
    assert len(mx) == 480
    s, w = soe16
    ex = ewald2d.ewald2d_longrange(sl.pos, sl.q, sl.box, sl.alpha, mx, my)
    so = soe_ewald2d.soe_full(sl.pos, sl.q, sl.box, sl.alpha, s, w, kc=kc)
    assert abs(so["E"] - ex["E"]) < 1e-11 * abs(ex["E"])
    assert _rel(so["phi"], ex["phi"]) < 1e-10
    assert _rel(so["F"], ex["F"]) < 1e-9


def test_realspace_at_equals_all_pairs():
    """The sampled real-space sum is the all-pairs one restricted to targets."""
    sl = workloads.uniform_slab(300, (15.0, 12.0, 6.0), 77, alpha=0.5)
    full = ewald2d.realspace(sl.pos, sl.q, sl.box, 0.5, 5.5)
    idx = np.array([0, 17, 150, 299])
    some = ewald2d.realspace_at(sl.pos, sl.q, sl.box, 0.5, 5.5, idx)
    assert np.allclose(some["phi"], full["phi"][idx], rtol=1e-13, atol=1e-15)
    assert np.allclose(some["F"], full["F"][idx], rtol=1e-12, atol=1e-14)
