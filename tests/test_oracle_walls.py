"""Pins of the oracle's charged-wall terms (Section 2.4, Thm 2.4) and of the
particle-particle part for particles that are not neutral on their own.

The walls are checked against things other than their own formula: the
uniform-density special case the paper states, the exact Ewald2D sum of
point charges that sample the walls on a fine grid, the far-field limit of
the paper's well-definedness proposition, and finite differences.
"""
import numpy as np
import pytest

from oracle import ewald2d, lattice, soe_ewald2d, walls


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def _ions(n, box, seed, zlo, zhi, net):
    rng = np.random.default_rng(seed)
    pos = np.column_stack([rng.uniform(0, box[0], n), rng.uniform(0, box[1], n),
                           rng.uniform(zlo, zhi, n)])
    q = np.where(np.arange(n) < (n + net) // 2, 1.0, -1.0)
    rng.shuffle(q)
    assert q.sum() == net
    return pos, q


def _ewald_total(pos, q, box, alpha):
    """Exact Ewald2D potential, forces and energy (Lemma 2.1 + Eq. 2.10 +
    self term) of point charges, converged to ~1e-14."""
    kc = lattice.kcut_for_tail(alpha, 1e-15)
    mx, my = lattice.full_modes(box[0], box[1], kc)
    lr = ewald2d.ewald2d_longrange(pos, q, box, alpha, mx, my)
    rs = ewald2d.realspace(pos, q, box, alpha, 6.5 / alpha)
    phi = lr["phi"] + rs["phi"]
    return {"phi": phi, "F": lr["F"] + rs["F"], "E": 0.5 * float(q @ phi)}


def test_uniform_walls_closed_form():
    """Uniform densities: only the zero mode remains, the potential
    -2 pi [sigma_top (Lz - z) + sigma_bot z] stated after Thm 2.4, and
    the field 2 pi (sigma_bot - sigma_top) along z."""
    box = (7.0, 9.0, 5.0)
    pos, q = _ions(40, box, 3, 0.0, 5.0, 4)
    pos[0, 2], pos[1, 2] = 0.0, 5.0                       # on both walls
    sb, st = -0.013, 0.031
    w = walls.wall_potential(pos, q, box, sb, st)
    z = pos[:, 2]
    phi = -2 * np.pi * (st * (box[2] - z) + sb * z)
    assert np.abs(w["phi"] - phi).max() < 1e-15
    assert np.abs(w["F"][:, :2]).max() == 0.0
    assert np.abs(w["F"][:, 2] - q * 2 * np.pi * (sb - st)).max() < 1e-15
    assert abs(w["E"] - float(q @ phi)) < 1e-14


@pytest.fixture(scope="module")
def sheets_case():
    """20 ions (net charge +2) in the middle of a 6 x 6 x 6 cell, walls with
    a uniform part that makes the whole neutral and two Fourier modes each,
    and the walls sampled by 16 x 16 point charges."""
    box = (6.0, 6.0, 6.0)
    pos, q = _ions(20, box, 11, 1.5, 4.5, 2)
    A = box[0] * box[1]
    sb0, st0 = -1.5 / A, -0.5 / A
    modes = np.array([[1, 0], [1, 2]])
    sb = np.array([0.004 + 0.002j, -0.003j])
    st = np.array([-0.002 + 0.001j, 0.0025])
    pb, qb = walls.discretise_wall(box, 0.0, sb0, modes, sb, n=16)
    pt, qt = walls.discretise_wall(box, box[2], st0, modes, st, n=16)
    assert abs(qb.sum() - A * sb0) < 1e-14 and abs(qt.sum() - A * st0) < 1e-14
    alpha = 1.5
    ions = _ewald_total(pos, q, box, alpha)
    sheets_pos = np.vstack([pb, pt])
    sheets_q = np.concatenate([qb, qt])
    sheets = _ewald_total(sheets_pos, sheets_q, box, alpha)
    allp = _ewald_total(np.vstack([pos, sheets_pos]), np.concatenate([q, sheets_q]), box, alpha)
    wall = walls.wall_potential(pos, q, box, sb0, st0, modes, sb, st)
    return dict(pos=pos, q=q, ions=ions, sheets=sheets, all=allp, wall=wall, n=q.size)


def test_walls_equal_sampled_sheets_potential(sheets_case):
    """phi at an ion of the neutral whole (ions + sampled walls, exact Ewald2D)
    = phi_p-p (ions alone, not neutral) + phi_p-s (Thm 2.4). The grid's
    aliases have wave numbers >= 2 pi (16 - 2)/6 and the ions are 1.5 or
    more from a wall, so the sampling error is below e^{-22} (measured: 1e-13)."""
    c = sheets_case
    n = c["n"]
    got = c["ions"]["phi"] + c["wall"]["phi"]
    assert _rel(got, c["all"]["phi"][:n]) < 1e-11
    # the wall part alone is O(1) here: the comparison is not dominated by phi_p-p
    assert np.abs(c["wall"]["phi"]).max() > 0.3 * np.abs(c["all"]["phi"][:n]).max()


def test_walls_equal_sampled_sheets_forces(sheets_case):
    c = sheets_case
    n = c["n"]
    got = c["ions"]["F"] + c["wall"]["F"]
    assert _rel(got, c["all"]["F"][:n]) < 1e-11
    # the modes matter: without them the forces differ visibly
    w0 = walls.wall_potential(c["pos"], c["q"], (6.0, 6.0, 6.0), -1.5 / 36, -0.5 / 36)
    assert _rel(c["ions"]["F"] + w0["F"], c["all"]["F"][:n]) > 1e-4


def test_walls_energy_counts_each_ion_wall_pair_once(sheets_case):
    """U(ions + walls) - U(walls alone) = U_p-p + U_p-s with
    U_p-s = sum_i q_i phi_p-s (no factor 1/2)."""
    c = sheets_case
    lhs = c["all"]["E"] - c["sheets"]["E"]
    rhs = c["ions"]["E"] + c["wall"]["E"]
    assert abs(lhs - rhs) < 1e-11 * abs(rhs)
    assert abs(lhs - (c["ions"]["E"] + 0.5 * c["wall"]["E"])) > 1e-3 * abs(rhs)


def test_far_field_limit_of_the_whole():
    """Well-definedness proposition of Section 2.4: with particles and walls
    neutral together, phi -> +-(2 pi / A) [sum_j q_j z_j + Lz sig^_top(0)]
    as z -> +-inf. Probes of zero charge 200 above and below the slab."""
    box = (8.0, 7.0, 5.0)
    pos, q = _ions(30, box, 5, 0.0, 5.0, 6)
    A = box[0] * box[1]
    sb0, st0 = -4.0 / A, -2.0 / A
    modes, sb, st = np.array([[0, 1]]), np.array([0.01j]), np.array([0.02])
    probes = np.array([[1.0, 2.0, box[2] + 200.0], [3.0, 4.0, -200.0]])
    P = np.vstack([pos, probes])
    Q = np.concatenate([q, [0.0, 0.0]])
    alpha = 0.8
    mx, my = lattice.full_modes(box[0], box[1], lattice.kcut_for_tail(alpha, 1e-15))
    pp = ewald2d.ewald2d_longrange(P, Q, box, alpha, mx, my)   # real space: 0 at the probes
    ps = walls.wall_potential(P, Q, box, sb0, st0, modes, sb, st)
    lim = 2 * np.pi / A * (float(q @ pos[:, 2]) + box[2] * A * st0)
    top, bot = pp["phi"][-2] + ps["phi"][-2], pp["phi"][-1] + ps["phi"][-1]
    assert abs(top - lim) < 1e-12 * abs(lim)
    assert abs(bot + lim) < 1e-12 * abs(lim)


def test_wall_forces_are_minus_gradient():
    box = (6.0, 5.0, 4.0)
    pos, q = _ions(8, box, 9, 0.3, 3.7, 0)
    args = (box, 0.02, -0.01, np.array([[1, 1], [0, 2], [2, -1]]),
            np.array([0.01 + 0.02j, -0.005, 0.003j]), np.array([0.004j, 0.01 - 0.01j, 0.002]))
    w = walls.wall_potential(pos, q, *args)
    h = 1e-6
    for i in range(len(q)):
        for d in range(3):
            p1, p2 = pos.copy(), pos.copy()
            p1[i, d] += h
            p2[i, d] -= h
            fd = -(walls.wall_potential(p1, q, *args)["E"] - walls.wall_potential(p2, q, *args)["E"]) / (2 * h)
            assert abs(fd - w["F"][i, d]) < 1e-7 * max(1.0, abs(w["F"][i, d]))
    # phi_p-s = dU_p-s/dq_i (U_p-s is linear in q)
    q2 = q.copy()
    q2[3] += 0.5
    assert abs(walls.wall_potential(pos, q2, *args)["E"] - w["E"] - 0.5 * w["phi"][3]) < 1e-12


def test_recursion_for_particles_not_neutral(soe16):
    """The sorted recursion (k != 0 and k = 0 terms) of particles with net
    charge equals the exact Ewald2D long-range part: neither side relies on
    neutrality."""
    s, w = soe16
    box = (10.0, 10.0, 5.0)
    pos, q = _ions(60, box, 21, 0.0, 5.0, 10)
    alpha = 0.6
    kc = lattice.kcut_for_tail(alpha, 1e-8)
    mx, my = lattice.full_modes(box[0], box[1], kc)
    ex = ewald2d.ewald2d_longrange(pos, q, box, alpha, mx, my)
    so = soe_ewald2d.soe_full(pos, q, box, alpha, s, w, kc=kc)
    assert abs(so["E"] - ex["E"]) < 1e-11 * abs(ex["E"])
    assert _rel(so["phi"], ex["phi"]) < 1e-11
    assert _rel(so["F"], ex["F"]) < 1e-10
