"""Pins of the oracle's molecular-dynamics pieces (Section 4.3's Langevin
dynamics, Section 5.2's short-range model): finite differences, invariances,
the generator's moments and the known sampling properties of the BAOAB
splitting."""
import math

import numpy as np

from oracle import md


def _pos(n, box, seed, zlo=None, zhi=None):
    rng = np.random.default_rng(seed)
    zlo = 0.0 if zlo is None else zlo
    zhi = box[2] if zhi is None else zhi
    return np.column_stack([rng.uniform(0, box[0], n), rng.uniform(0, box[1], n), rng.uniform(zlo, zhi, n)])


def test_lj_pairs_forces_are_minus_gradient():
    box = (3.0, 3.0, 3.0)
    g = np.arange(3) + 0.5               # a jittered lattice of spacing 1: most
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)   # neighbours within the cut-off
    pos = pos + np.random.default_rng(1).uniform(-0.12, 0.12, pos.shape)
    lj = md.lj_pairs(pos, box, 1.3, 0.9)
    assert (lj["F"] != 0).all(axis=1).sum() > 20
    assert lj["E"] > 0
    assert np.abs(lj["F"].sum(0)).max() < 1e-10 * np.abs(lj["F"]).max()   # Newton's third law
    h = 1e-6
    for i in range(0, 27, 5):
        for d in range(3):
            p1, p2 = pos.copy(), pos.copy()
            p1[i, d] += h
            p2[i, d] -= h
            fd = -(md.lj_pairs(p1, box, 1.3, 0.9)["E"] - md.lj_pairs(p2, box, 1.3, 0.9)["E"]) / (2 * h)
            assert abs(fd - lj["F"][i, d]) < 1e-5 * max(1.0, abs(lj["F"][i, d]))


def test_lj_pairs_cutoff_and_images():
    box = (10.0, 10.0, 10.0)
    rc = md.TWO16 * 1.0
    # a pair just inside and one just outside the cut-off, across the x boundary
    pos = np.array([[0.1, 5.0, 5.0], [10.0 - (rc - 1e-7 - 0.1), 5.0, 5.0],
                    [5.0, 0.05, 1.0], [5.0, 10.0 - (rc + 1e-6 - 0.05), 1.0]])
    lj = md.lj_pairs(pos, box, 1.0, 1.0)
    assert lj["F"][0, 0] > 0 and abs(lj["F"][0, 0]) < 1e-4   # repulsive, vanishing at r_c
    assert np.abs(lj["F"][2:]).max() == 0.0
    assert 0 < lj["E"] < 1e-12


def test_lj_walls():
    box = (5.0, 5.0, 6.0)
    pos = np.array([[1.0, 1.0, 0.3], [2.0, 2.0, 3.0], [3.0, 3.0, 5.8]])
    w = md.lj_walls(pos, box, 1.0, 0.5)
    assert w["F"][0, 2] > 0 and w["F"][2, 2] < 0 and w["F"][1, 2] == 0.0
    h = 1e-7
    for i in (0, 2):
        p1, p2 = pos.copy(), pos.copy()
        p1[i, 2] += h
        p2[i, 2] -= h
        fd = -(md.lj_walls(p1, box, 1.0, 0.5)["E"] - md.lj_walls(p2, box, 1.0, 0.5)["E"]) / (2 * h)
        assert abs(fd - w["F"][i, 2]) < 1e-5 * abs(w["F"][i, 2])


def test_noise_moments():
    n = 200_000
    xi = md.noise(n, 7, 123)
    assert np.abs(xi.mean(0)).max() < 5 / math.sqrt(n)
    assert np.abs(xi.var(0) - 1).max() < 5 * math.sqrt(2 / n)
    c = np.corrcoef(xi.T)
    assert np.abs(c - np.eye(3)).max() < 5 / math.sqrt(n)
    assert not np.array_equal(md.noise(10, 7, 123), md.noise(10, 8, 123))


def test_baoab_free_flight_and_wrap():
    box = (3.0, 4.0, 10.0)
    pos = _pos(5, box, 2, 2.0, 8.0)
    vel = np.random.default_rng(3).normal(size=(5, 3))
    p = md.MDParams(dt=0.01, gamma=0.0, seed=1)
    zero = lambda x: np.zeros_like(x)
    x, v = pos, vel
    F = zero(x)
    for n in range(300):
        x, v, F = md.baoab_step(x, v, F, box, p, n, zero)
    want = pos + 300 * 0.01 * vel
    want[:, 0] = np.mod(want[:, 0], box[0])
    want[:, 1] = np.mod(want[:, 1], box[1])
    assert np.abs(x - want).max() < 1e-12
    assert np.array_equal(v, vel)


def test_baoab_samples_harmonic_configurations_exactly():
    """For a harmonic well, BAOAB's stationary position variance is kT/k at
    any stable step size (Leimkuhler and Matthews 2013); with dt = 0.5 the
    other orderings are off by several per cent."""
    n, k, kT = 20_000, 1.0, 1.0
    box = (50.0, 50.0, 100.0)
    p = md.MDParams(dt=0.5, gamma=1.0, kT=kT, seed=9)
    force = lambda x: np.column_stack([np.zeros(len(x)), np.zeros(len(x)), -k * (x[:, 2] - 50.0)])
    rng = np.random.default_rng(4)
    x = np.column_stack([rng.uniform(0, 50, n), rng.uniform(0, 50, n), 50.0 + rng.normal(size=n)])
    v = rng.normal(size=(n, 3))
    F = force(x)
    acc = []
    for step in range(240):
        x, v, F = md.baoab_step(x, v, F, box, p, step, force)
        if step >= 40:
            acc.append(((x[:, 2] - 50.0) ** 2).mean())
    var = float(np.mean(acc))
    assert abs(var - kT / k) < 0.01
    # velocities: the free directions are exactly Maxwellian after the O step
    assert abs(v[:, 0].var() - kT) < 0.05
