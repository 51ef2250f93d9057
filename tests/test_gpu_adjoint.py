"""GPU: the energy-only call (forward sums, each pair once) and its adjoint
(the bidirectional scans over the stored sorted order), through the C ABI.

The energy-only call must give the full call's energy (FP64: to rounding,
1e-12 relative, and the oracle's to 1e-10), and the adjoint must reproduce
the full call's potentials and forces bit for bit: it runs the same
recurrence and combine kernels on the same sorted data, carries and sample.

FP32: the energy-only call within the FP32 energy budget, 1e-6 of the
energy scale. It sums each pair once; the pairs within a chunk come from
recurrences started from zero (small states, small rounding) and the pairs
with earlier chunks from the carries and pass A's aggregates, one product
per chunk and state.
"""
import numpy as np
import pytest

import workloads
from oracle import lattice, soe_ewald2d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qslab():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01521_gb300 as q
    q.load()
    return q


def _t(a, dt):
    return torch.tensor(a, device="cuda", dtype=dt)


def test_fp64_full_k_energy_and_adjoint(qslab, soe16):
    sl = workloads.small_full()
    kc = lattice.kcut_for_tail(sl.alpha, sl.tail)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, kcut=kc)
    pos, q = _t(sl.pos, torch.float64), _t(sl.q, torch.float64)
    e_full, phi_full, F_full = slab.compute(pos, q)
    e = slab.compute_energy(pos, q)
    phi, F = slab.adjoint()
    assert slab.status() == 0
    ref = soe_ewald2d.soe_full(sl.pos, sl.q, sl.box, sl.alpha, *soe16, kc=kc)
    assert abs(e.item() - e_full.item()) <= 1e-12 * abs(e_full.item())
    assert abs(e.item() - ref["E"]) <= 1e-10 * abs(ref["E"])
    assert torch.equal(phi, phi_full) and torch.equal(F, F_full)
    # the adjoint may be repeated
    phi2, F2 = slab.adjoint()
    assert torch.equal(phi2, phi_full) and torch.equal(F2, F_full)
    slab.close()


@pytest.mark.parametrize("tuning", [(32, 32), (96, 64)])
def test_fp64_ragged_chunks(qslab, soe16, tuning):
    sl = workloads.small_full()
    kc = lattice.kcut_for_tail(sl.alpha, sl.tail)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, kcut=kc).tuning(*tuning)
    pos, q = _t(sl.pos, torch.float64), _t(sl.q, torch.float64)
    e_full, phi_full, F_full = slab.compute(pos, q)
    e = slab.compute_energy(pos, q)
    phi, F = slab.adjoint()
    assert slab.status() == 0
    assert abs(e.item() - e_full.item()) <= 1e-12 * abs(e_full.item())
    assert torch.equal(phi, phi_full) and torch.equal(F, F_full)
    slab.close()


def test_fp64_random_batch_same_sample(qslab, soe16):
    """Energy-only then adjoint reuse one random-batch sample: the same as a
    full call drawing the same sample (counter rewound)."""
    sl = workloads.uniform_slab(3000, (50.0, 44.0, 15.0), 51, alpha=0.15)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, rbe=(64, 9))
    pos, q = _t(sl.pos, torch.float64), _t(sl.q, torch.float64)
    e = slab.compute_energy(pos, q)
    modes = slab.sampled_modes()
    phi, F = slab.adjoint()
    slab.set_rng_state(9, 0)
    e_full, phi_full, F_full = slab.compute(pos, q)
    assert slab.status() == 0
    assert np.array_equal(slab.sampled_modes()[0], modes[0])
    assert abs(e.item() - e_full.item()) <= 1e-12 * abs(e_full.item())
    assert torch.equal(phi, phi_full) and torch.equal(F, F_full)
    ref = soe_ewald2d.soe_rbe(sl.pos, sl.q, sl.box, sl.alpha, *soe16, modes[0], modes[1], 64)
    assert abs(e.item() - ref["E"]) <= 1e-10 * abs(ref["E"])
    slab.close()


def test_fp64_walls_net_charge(qslab, soe16):
    sl = workloads.cations_walls(n=200, L=50.0)
    A = sl.box[0] * sl.box[1]
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, kcut=kc)
    slab.set_walls(-0.4 * sl.N / A, -0.6 * sl.N / A, [(1, 1)], [0.01 + 0.002j], [-0.004j])
    pos, q = _t(sl.pos, torch.float64), _t(sl.q, torch.float64)
    e_full, phi_full, F_full = slab.compute(pos, q)
    e = slab.compute_energy(pos, q)
    phi, F = slab.adjoint()
    assert slab.status() == 0
    assert abs(e.item() - e_full.item()) <= 1e-12 * abs(e_full.item())
    assert torch.equal(phi, phi_full) and torch.equal(F, F_full)
    slab.close()


def test_fp64_batched(qslab, soe16):
    sls = [workloads.uniform_slab(500, (20.0, 24.0, 6.0), 52, alpha=0.3),
           workloads.uniform_slab(900, (28.0, 26.0, 9.0), 53, alpha=0.3)]
    kc = lattice.kcut_for_tail(0.3, 1e-8)
    slab = qslab.QSlab(0, "fp64").configure((1.0, 1.0, 1.0), 0.3, soe16, kcut=kc)
    pos = _t(np.concatenate([s.pos for s in sls]), torch.float64)
    q = _t(np.concatenate([s.q for s in sls]), torch.float64)
    off = [0, 500, 1400]
    boxes = [s.box for s in sls]
    e_full, phi_full, F_full = slab.compute_batched(pos, q, off, boxes)
    e = slab.compute_batched_energy(pos, q, off, boxes)
    phi, F = slab.adjoint()
    assert slab.status() == 0
    assert torch.allclose(e, e_full, rtol=1e-12, atol=0)
    assert torch.equal(phi, phi_full) and torch.equal(F, F_full)
    slab.close()


def test_fp32_large_random_batch(qslab, soe16):
    """The N = 1e6 workload in FP32: the energy-only call against the oracle
    on the same sample (FP32-rounded inputs), within 1e-6 of the energy scale
    |E_full-k| (the estimator's expectation, golden file); the adjoint's
    outputs equal the full call's."""
    import json
    import os
    sl = workloads.rbe_large()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rbe_large_fullk.json")
    with open(path) as fh:
        escale = abs(json.load(fh)["E_fullk"])
    slab = qslab.QSlab(0, "fp32c").configure(sl.box, sl.alpha, soe16, rbe=(200, 4))
    pos, q = _t(sl.pos, torch.float32), _t(sl.q, torch.float32)
    e = slab.compute_energy(pos, q)
    mx, my, _ = slab.sampled_modes()
    phi, F = slab.adjoint()
    slab.set_rng_state(4, 0)
    e_full, phi_full, F_full = slab.compute(pos, q)
    assert slab.status() == 0
    assert torch.equal(phi, phi_full) and torch.equal(F, F_full)
    ref = soe_ewald2d.soe_rbe(pos.double().cpu().numpy(), q.double().cpu().numpy(), sl.box,
                              sl.alpha, *soe16, mx, my)
    err_e, err_full = abs(e.item() - ref["E"]) / escale, abs(e_full.item() - ref["E"]) / escale
    assert err_e <= 1e-6, (err_e, err_full)
    slab.close()


def test_adjoint_needs_a_fresh_energy_call(qslab, soe16):
    sl = workloads.uniform_slab(400, (20.0, 20.0, 6.0), 54, alpha=0.3)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, kcut=kc)
    pos, q = _t(sl.pos, torch.float64), _t(sl.q, torch.float64)
    N = sl.N
    phi = torch.empty(N, dtype=torch.float64, device="cuda")
    F = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    lib = qslab.load()
    st = torch.cuda.current_stream().cuda_stream
    assert lib.qslab_compute_adjoint(slab.h, phi.data_ptr(), F.data_ptr(), st) == -2
    slab.compute_energy(pos, q)
    assert lib.qslab_compute_adjoint(slab.h, phi.data_ptr(), F.data_ptr(), st) == 0
    slab.compute(pos, q)           # a full call reuses the workspace
    assert lib.qslab_compute_adjoint(slab.h, phi.data_ptr(), F.data_ptr(), st) == -2
    slab.compute_energy(pos, q)
    slab.set_walls(0.0, 0.0)       # a configuration change
    assert lib.qslab_compute_adjoint(slab.h, phi.data_ptr(), F.data_ptr(), st) == -2
    assert lib.qslab_compute_adjoint(slab.h, None, None, st) == -1
    assert slab.status() == 0
    slab.close()


def test_autograd_adjoint_mode(qslab, soe16):
    """slab_energy(adjoint=True): energy-only forward, adjoint backward; the
    gradients equal those of the default mode."""
    sl = workloads.uniform_slab(600, (22.0, 20.0, 7.0), 55, alpha=0.35)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, kcut=kc)
    grads = []
    for adj in (False, True):
        pos = _t(sl.pos, torch.float64).requires_grad_(True)
        q = _t(sl.q, torch.float64).requires_grad_(True)
        E = qslab.slab_energy(pos, q, slab, adjoint=adj)
        E.backward()
        grads.append((float(E.item()), pos.grad.clone(), q.grad.clone()))
    assert abs(grads[0][0] - grads[1][0]) <= 1e-12 * abs(grads[0][0])
    assert torch.equal(grads[0][1], grads[1][1]) and torch.equal(grads[0][2], grads[1][2])
    slab.close()


@pytest.mark.parametrize("n", [1, 2])
def test_fp64_tiny(qslab, soe16, n):
    """N = 1 (neutralised by a uniform wall) and N = 2 with equal z."""
    box = (9.0, 8.0, 4.0)
    pos = np.array([[1.0, 2.0, 1.5], [6.0, 7.0, 1.5]])[:n]
    q = np.array([1.0, -1.0])[:n]
    kc = lattice.kcut_for_tail(0.5, 1e-8)
    slab = qslab.QSlab(0, "fp64").configure(box, 0.5, soe16, kcut=kc)
    if n == 1:
        slab.set_walls(-1.0 / (box[0] * box[1]), 0.0)
    p, qq = _t(pos, torch.float64), _t(q, torch.float64)
    e_full, phi_full, F_full = slab.compute(p, qq)
    e = slab.compute_energy(p, qq)
    phi, F = slab.adjoint()
    assert slab.status() == 0
    assert abs(e.item() - e_full.item()) <= 1e-12 * max(abs(e_full.item()), 1e-300)
    assert torch.equal(phi, phi_full) and torch.equal(F, F_full)
    slab.close()
