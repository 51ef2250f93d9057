"""Pins of the oracle's virial tensor (no GPU).

The virial W_ab = -dE/d eps_ab is checked against central finite differences
of the oracle's energies under the strain itself (the box, the particles and
the walls deformed together), against an independent evaluation of the
oblique-lattice energy for the shear component, against brute-force SOE pair
sums, and against the virial theorem of the Coulomb energy: E is homogeneous
of degree -1 in all lengths, so W_xx + W_yy + W_zz = E for the whole
(alpha-independent) Ewald2D energy.
"""
import numpy as np
import pytest

import workloads
from oracle import ewald2d, lattice, soe_ewald2d, virial, walls

H = 1e-5


def _slab(n=24, box=(10.0, 12.0, 5.0), seed=11, alpha=0.6):
    return workloads.uniform_slab(n, box, seed, alpha=alpha)


def _modes(box, alpha, tail=1e-10):
    return lattice.full_modes(box[0], box[1], lattice.kcut_for_tail(alpha, tail))


def _strain(pos, box, key, e):
    """Positions and box under the strain eps_key = e (lattice stays rectangular)."""
    p = pos.copy()
    Lx, Ly, Lz = box
    if key == "xx":
        p[:, 0] *= 1 + e
        Lx *= 1 + e
    elif key == "yy":
        p[:, 1] *= 1 + e
        Ly *= 1 + e
    elif key == "zz":
        p[:, 2] *= 1 + e
        Lz *= 1 + e
    elif key == "xz":
        p[:, 0] += e * pos[:, 2]
    elif key == "yz":
        p[:, 1] += e * pos[:, 2]
    return p, (Lx, Ly, Lz)


def _fd(energy, pos, box, key):
    pp, bp = _strain(pos, box, key, H)
    pm, bm = _strain(pos, box, key, -H)
    return -(energy(pp, bp) - energy(pm, bm)) / (2 * H)


def _scale(W):
    return max(abs(W["xx"]), abs(W["yy"]), abs(W["zz"]))


@pytest.mark.parametrize("key", ["xx", "yy", "zz", "xz", "yz"])
def test_exact_virial_is_minus_strain_derivative(key):
    """Lemma 2.1 energy over a fixed mode list, differentiated numerically."""
    s = _slab()
    mx, my = _modes(s.box, s.alpha)
    W = virial.longrange_virial_exact(s.pos, s.q, s.box, s.alpha, mx, my)["W"]

    def energy(p, b):
        return ewald2d.ewald2d_longrange(p, s.q, b, s.alpha, mx, my)["E"]
    fd = _fd(energy, s.pos, s.box, key)
    assert abs(W[key] - fd) < 2e-8 * _scale(W)


def test_oblique_lattice_energy():
    """The oblique-lattice energy equals the rectangular one for h = diag(L),
    and does not depend on the basis chosen for the same lattice."""
    s = _slab()
    Lx, Ly, _ = s.box
    mx, my = _modes(s.box, s.alpha)
    m = np.stack([mx, my], 1)
    frac = s.pos[:, :2] / np.array([Lx, Ly])
    h = np.diag([Lx, Ly])
    E0 = ewald2d.ewald2d_longrange(s.pos, s.q, s.box, s.alpha, mx, my)["E"]
    E1 = virial.longrange_energy_lattice(frac, s.pos[:, 2], s.q, h, s.alpha, m)
    assert abs(E1 - E0) < 1e-12 * abs(E0)
    # new basis h U, U unimodular: frac' = U^-1 frac, modes m' = U^T m
    U = np.array([[1, 1], [0, 1]])
    h2 = h @ U
    frac2 = frac @ np.linalg.inv(U).T
    m2 = m @ U
    E2 = virial.longrange_energy_lattice(frac2, s.pos[:, 2], s.q, h2, s.alpha, m2)
    assert abs(E2 - E0) < 1e-12 * abs(E0)
    # an oblique lattice that is not rectangular gives another energy
    E3 = virial.longrange_energy_lattice(frac, s.pos[:, 2], s.q, np.array([[Lx, 1.0], [0, Ly]]),
                                         s.alpha, m)
    assert abs(E3 - E0) > 1e-6 * abs(E0)


def test_exact_virial_shear():
    """W_xy from a symmetric shear eps_xy = eps_yx = e of the lattice:
    -dE/de = W_xy + W_yx = 2 W_xy."""
    s = _slab()
    Lx, Ly, _ = s.box
    mx, my = _modes(s.box, s.alpha)
    m = np.stack([mx, my], 1)
    frac = s.pos[:, :2] / np.array([Lx, Ly])
    W = virial.longrange_virial_exact(s.pos, s.q, s.box, s.alpha, mx, my)["W"]

    def energy(e):
        h = np.array([[1.0, e], [e, 1.0]]) @ np.diag([Lx, Ly])
        return virial.longrange_energy_lattice(frac, s.pos[:, 2], s.q, h, s.alpha, m)
    fd = -(energy(H) - energy(-H)) / (2 * H)
    assert abs(2 * W["xy"] - fd) < 2e-8 * _scale(W)
    assert abs(W["xy"]) > 1e-4 * _scale(W)      # not trivially zero


def test_soe_dk_recursion_equals_direct(soe16):
    """The k-derivatives of the SOE pair sums by the sorted recursion equal
    the direct pair sums, and finite differences in |k| of the SOE kernel."""
    s, w = soe16
    sl = _slab(n=40, seed=12)
    Lx, Ly, _ = sl.box
    mx, my = _modes(sl.box, sl.alpha, 1e-8)
    R = virial.soe_dk(sl.pos, sl.q, sl.box, sl.alpha, s, w, mx, my)
    Rd = virial.soe_dk_direct(sl.pos, sl.q, sl.box, sl.alpha, s, w, mx, my)
    assert np.abs(R - Rd).max() < 1e-11 * np.abs(Rd).max()
    kx, ky, kk = lattice.kvec(mx, my, Lx, Ly)
    x, y, z = sl.pos.T
    adz = np.abs(z[:, None] - z[None, :])
    off = ~np.eye(sl.N, dtype=bool)
    for j in range(0, len(kk), 7):
        th = kx[j] * x + ky[j] * y
        c, sn = sl.q * np.cos(th), sl.q * np.sin(th)

        def pairsum(k):
            G = ewald2d.soe_kernel_k(k, adz, sl.alpha, s, w) * off
            return c @ G @ c + sn @ G @ sn
        h = 1e-5 * kk[j]
        fd = (pairsum(kk[j] + h) - pairsum(kk[j] - h)) / (2 * h)
        assert abs(R[j] - fd) < 1e-7 * np.abs(R).max()


@pytest.mark.parametrize("key", ["xx", "yy", "zz", "xz", "yz"])
def test_soe_virial_is_minus_strain_derivative(key, soe16):
    """The SOE recursion's virial against finite differences of the SOE
    energy itself (same modes, same table)."""
    s, w = soe16
    sl = _slab(n=40, seed=13)
    modes = _modes(sl.box, sl.alpha, 1e-8)
    W = virial.soe_full_virial(sl.pos, sl.q, sl.box, sl.alpha, s, w, modes=modes)["W"]

    def energy(p, b):
        return soe_ewald2d.soe_full(p, sl.q, b, sl.alpha, s, w, modes=modes)["E"]
    fd = _fd(energy, sl.pos, sl.box, key)
    assert abs(W[key] - fd) < 2e-8 * _scale(W)


def test_soe_virial_close_to_exact(soe16):
    """SOE kernel (fit error 3e-10) against the exact erfc kernel."""
    s, w = soe16
    sl = _slab(n=40, seed=14)
    modes = _modes(sl.box, sl.alpha, 1e-8)
    W = virial.soe_full_virial(sl.pos, sl.q, sl.box, sl.alpha, s, w, modes=modes)["W"]
    We = virial.longrange_virial_exact(sl.pos, sl.q, sl.box, sl.alpha, *modes)["W"]
    for k in virial.KEYS:
        assert abs(W[k] - We[k]) < 1e-8 * _scale(We), k


def _total_virial(sl, alpha, rc, tail=1e-13):
    mx, my = _modes(sl.box, alpha, tail)
    lr = virial.longrange_virial_exact(sl.pos, sl.q, sl.box, alpha, mx, my)
    rs = virial.realspace_virial(sl.pos, sl.q, sl.box, alpha, rc)
    W = {k: lr["W"][k] + rs["W"][k] for k in virial.KEYS}
    return W, lr["E"] + rs["E"]


def test_virial_theorem_total():
    """W_xx + W_yy + W_zz = E for the whole Ewald2D energy (long range plus
    real space), at two splitting parameters, which must also agree."""
    sl = _slab(n=30, box=(9.0, 9.0, 4.0), seed=15)
    out = []
    for alpha, rc in [(1.0, 4.4), (1.3, 3.4)]:
        W, E = _total_virial(sl, alpha, rc)
        assert abs(W["xx"] + W["yy"] + W["zz"] - E) < 1e-8 * _scale(W)
        out.append(W)
    for k in virial.KEYS:
        assert abs(out[0][k] - out[1][k]) < 1e-8 * _scale(out[0]), k


@pytest.mark.parametrize("key", ["xx", "zz", "xz"])
def test_realspace_virial_fd(key):
    sl = _slab(n=30, box=(9.0, 9.0, 4.0), seed=16)
    alpha, rc = 0.8, 3.5
    W = virial.realspace_virial(sl.pos, sl.q, sl.box, alpha, rc)["W"]

    def energy(p, b):
        return ewald2d.realspace(p, sl.q, b, alpha, rc)["E"]
    fd = _fd(energy, sl.pos, sl.box, key)
    assert abs(W[key] - fd) < 1e-7 * _scale(W)


def _wall_case():
    sl = _slab(n=20, box=(10.0, 12.0, 5.0), seed=17)
    q = sl.q.copy()
    q[:3] = [1.0, 1.0, 1.0]          # net charge 2 + ... balanced by the walls
    A = sl.box[0] * sl.box[1]
    Q = q.sum()
    sb0, st0 = -0.3 * Q / A, -0.7 * Q / A
    modes = [(1, 0), (1, 2)]
    sb = [0.01 + 0.02j, -0.015j]
    st = [0.02 - 0.01j, 0.012 + 0.004j]
    return sl, q, sb0, st0, modes, sb, st


def _wall_strained(sl, q, sb0, st0, modes, sb, st, key, e):
    p, b = _strain(sl.pos, sl.box, key, e)
    f = 1.0
    if key in ("xx", "yy"):
        f = 1.0 / (1 + e)                    # charge per cell kept: sigma ~ 1/A
    sbn = [c * f for c in sb]
    stn = [c * f for c in st]
    if key in ("xz", "yz"):
        # the top wall shifts by e Lz; its pattern sigma(rho - d) gains e^{-i k.d}
        Lx, Ly, Lz = sl.box
        d = np.array([e * Lz, 0.0]) if key == "xz" else np.array([0.0, e * Lz])
        stn = [c * np.exp(-1j * (2 * np.pi * m[0] / Lx * d[0] + 2 * np.pi * m[1] / Ly * d[1]))
               for c, m in zip(st, modes)]
    return walls.wall_potential(p, q, b, sb0 * f, st0 * f, modes, sbn, stn)["E"]


@pytest.mark.parametrize("key", ["xx", "yy", "zz", "xz", "yz"])
def test_wall_virial_fd(key):
    """Particle-slab energy of Thm 2.4 with the walls strained with the box."""
    sl, q, sb0, st0, modes, sb, st = _wall_case()
    W = virial.wall_virial(sl.pos, q, sl.box, sb0, st0, modes, sb, st)["W"]
    fd = -(_wall_strained(sl, q, sb0, st0, modes, sb, st, key, H)
           - _wall_strained(sl, q, sb0, st0, modes, sb, st, key, -H)) / (2 * H)
    assert abs(W[key] - fd) < 1e-7 * _scale(W), (W[key], fd)


def test_virial_theorem_with_walls():
    """Particles plus uniform walls with a net charge each: the particle
    energy and the particle-wall energy together are homogeneous of degree -1
    as well (the walls keep their charge per cell and move with the box)."""
    sl, q, sb0, st0, modes, sb, st = _wall_case()
    alpha, rc = 1.0, 4.4
    mx, my = _modes(sl.box, alpha, 1e-13)
    lr = virial.longrange_virial_exact(sl.pos, q, sl.box, alpha, mx, my)
    rs = virial.realspace_virial(sl.pos, q, sl.box, alpha, rc)
    wv = virial.wall_virial(sl.pos, q, sl.box, sb0, st0, modes, sb, st)
    W = {k: lr["W"][k] + rs["W"][k] + wv["W"][k] for k in virial.KEYS}
    E = lr["E"] + rs["E"] + wv["E"]
    assert abs(W["xx"] + W["yy"] + W["zz"] - E) < 1e-8 * _scale(W)
    # the explicit L_z term of the top wall is needed for it
    Wno = W["zz"] + sl.box[2] * float(q.sum()) * (-2 * np.pi * st0)
    assert abs(W["xx"] + W["yy"] + Wno - E) > 1e-3 * _scale(W)


def test_rbe_virial_unbiased(soe16):
    """The random-batch virial (Eq. 4.7 weights) averages to the full k-sum's."""
    s, w = soe16
    sl = _slab(n=60, box=(8.0, 8.0, 6.0), seed=18, alpha=0.5)
    full = virial.soe_full_virial(sl.pos, sl.q, sl.box, sl.alpha, s, w, tail=1e-12)["W"]
    P, nseed = 20, 300
    vals = {k: [] for k in virial.KEYS}
    for seed in range(nseed):
        mx, my = lattice.sample_modes(P, 7, seed, sl.alpha, sl.box[0], sl.box[1])
        Wr = virial.soe_rbe_virial(sl.pos, sl.q, sl.box, sl.alpha, s, w, mx, my, P)["W"]
        for k in virial.KEYS:
            vals[k].append(Wr[k])
    for k in virial.KEYS:
        v = np.asarray(vals[k])
        se = v.std(ddof=1) / np.sqrt(nseed)
        assert abs(v.mean() - full[k]) < 4.5 * se + 1e-9 * _scale(full), k
