"""GPU: the differentiable strongly confined slab at its full size.

Workload: N = 2e5 in 200 x 200 x 2, z exponential from a randomly chosen
wall (decay length 0.2), charges N(0, 1) minus their mean, alpha = 0.2,
M = 24 (conditioned SOE), full k-sum at Gaussian tail 1e-8 (9392 lattice
vectors, 4696 half-plane modes).

Expected values come from tests/golden/confined_fullk.json, written by
tests/golden/make_golden.py from the FP64 oracle alone: the energy, its three
parts, and the potential and force of 512 seeded particles, on the FP64
inputs and on the inputs rounded to FP32.

Checks (App. E's forces; the differentiation pattern of an autograd energy
whose backward is the library's adjoint):
  - FP64 path: energy, and phi, F at the sampled particles, to 1e-10;
  - FP32C path: phi, F RMS over the sample to 1e-5; energy to 1e-6 of the
    magnitude of its parts, |E_k| + |E_0| + |E_c| (this energy, 233.8, is
    what is left of parts of +2140, +45 and -1951);
  - the autograd backward of the energy-only forward (adjoint = True):
    -dE/dr and dE/dq against the oracle's forces and potentials at the
    sample, both precisions;
  - the same backward (FP64) against central differences of the GPU FP64
    energy, h = 1e-4, at 20 seeded particles (x, y, z), and dE/dq against
    differences along q_i - q_j (which keep the slab neutral) for 10 pairs.
"""
import json
import os

import numpy as np
import pytest

import workloads
from oracle import lattice

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def qslab():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01521_gb300 as q
    q.load()
    return q


@pytest.fixture(scope="module")
def gold():
    with open(os.path.join(HERE, "golden", "confined_fullk.json")) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def slab5():
    return workloads.confined()


@pytest.fixture(scope="module")
def soe24():
    from paper_2403_01521_gb300.soe import load_soe
    return load_soe(24)


def _inputs(sl, prec, gold):
    from golden_check import fingerprint_matches
    dt = torch.float64 if prec == "fp64" else torch.float32
    pos = torch.tensor(sl.pos, device="cuda", dtype=dt)
    q = torch.tensor(sl.q, device="cuda", dtype=dt)
    g = gold["fp64" if prec == "fp64" else "fp32"]
    assert fingerprint_matches(g, pos.double().cpu().numpy(), q.double().cpu().numpy())
    return pos, q, g


def _maxrel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _rmsrel(a, b):
    return float(np.sqrt(((a - b) ** 2).mean()) / np.sqrt((b ** 2).mean()))


def _slab(qslab, sl, prec, soe):
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    return qslab.QSlab(0, prec).configure(sl.box, sl.alpha, soe, kcut=kc)


def _check(prec, g, E, phi, F):
    idx = np.array(g["sample_idx"])
    phi_ref = np.array(g["phi"])
    F_ref = np.array(g["F"])
    if prec == "fp64":
        assert abs(E - g["E"]) <= 1e-10 * abs(g["E"]), (E, g["E"])
        assert _maxrel(phi[idx], phi_ref) <= 1e-10
        assert _maxrel(F[idx], F_ref) <= 1e-10
    else:
        scale = sum(abs(v) for v in g["E_parts"])
        assert abs(E - g["E"]) <= 1e-6 * scale, (E, g["E"], scale)
        assert _rmsrel(phi[idx], phi_ref) <= 1e-5
        assert _rmsrel(F[idx], F_ref) <= 1e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_confined_full_size(qslab, slab5, soe24, gold, prec):
    pos, q, g = _inputs(slab5, prec, gold)
    s = _slab(qslab, slab5, prec, soe24)
    assert s.num_modes() == g["modes_full_lattice"] // 2
    e, phi, F = s.compute(pos, q)
    assert s.status() == 0
    s.close()
    _check(prec, g, float(e.item()), phi.double().cpu().numpy(), F.double().cpu().numpy())


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_confined_autograd_adjoint(qslab, slab5, soe24, gold, prec):
    """Energy-only forward, adjoint backward (nothing N x K stored)."""
    pos, q, g = _inputs(slab5, prec, gold)
    s = _slab(qslab, slab5, prec, soe24)
    p_ = pos.clone().requires_grad_(True)
    q_ = q.clone().requires_grad_(True)
    E = qslab.slab_energy(p_, q_, s, adjoint=True)
    E.backward()
    assert s.status() == 0
    s.close()
    _check(prec, g, float(E.item()), q_.grad.double().cpu().numpy(),
           -p_.grad.double().cpu().numpy())


def test_confined_finite_differences(qslab, slab5, soe24):
    """Central differences (h = 1e-4) of the GPU FP64 energy against the
    autograd backward, at 20 particles and 10 neutral charge pairs."""
    sl = slab5
    h = 1e-4
    s = _slab(qslab, sl, "fp64", soe24)
    pos = torch.tensor(sl.pos, device="cuda", dtype=torch.float64)
    q = torch.tensor(sl.q, device="cuda", dtype=torch.float64)
    p_ = pos.clone().requires_grad_(True)
    q_ = q.clone().requires_grad_(True)
    qslab.slab_energy(p_, q_, s, adjoint=True).backward()
    gpos = p_.grad.cpu().numpy()
    gq = q_.grad.cpu().numpy()
    rng = np.random.default_rng(77)
    z = sl.pos[:, 2]
    inside = np.flatnonzero((z > 2 * h) & (z < sl.box[2] - 2 * h))
    pick = rng.choice(inside, size=20, replace=False)

    def energy(p, qq):
        e = s.compute_energy(p, qq)
        assert s.status() == 0
        return float(e.item())

    fd = np.zeros((20, 3))
    for a, i in enumerate(pick):
        for d in range(3):
            pp = pos.clone()
            pp[i, d] += h
            ep = energy(pp, q)
            pp[i, d] -= 2 * h
            em = energy(pp, q)
            fd[a, d] = (ep - em) / (2 * h)
    an = gpos[pick]
    assert np.abs(fd - an).max() <= 1e-6 * np.abs(an).max() + 1e-9, (fd, an)
    # dE/dq along e_i - e_j: E is quadratic in q, so the central difference
    # is exact up to rounding
    pairs = rng.choice(sl.N, size=(10, 2), replace=False)
    for i, j in pairs:
        qp = q.clone()
        qp[i] += h
        qp[j] -= h
        ep = energy(pos, qp)
        qp[i] -= 2 * h
        qp[j] += 2 * h
        em = energy(pos, qp)
        fdq = (ep - em) / (2 * h)
        assert abs(fdq - (gq[i] - gq[j])) <= 1e-7 * (abs(gq[i]) + abs(gq[j])) + 1e-9
    s.close()
