"""GPU parity of the real-space part (Eq. 2.10, cut-off rc, images in x and
y) against the FP64 oracle, and the alpha-independence of the GPU total
(real space + long range), which ties the two parts of the splitting
together (Eq. 2.9)."""
import numpy as np
import pytest

import workloads
from oracle import ewald2d, lattice

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qslab():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01521_gb300 as q
    q.load()
    return q


def _maxrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _rmsrel(a, b):
    return float(np.sqrt(((a - b) ** 2).mean()) / max(np.sqrt((b ** 2).mean()), 1e-300))


def _rs(qslab, sl, prec, alpha, rc, soe):
    slab = qslab.QSlab(0, prec).configure(sl.box, alpha, soe, kcut=1.0, rcut=rc)
    dt = torch.float64 if prec == "fp64" else torch.float32
    pos = torch.tensor(sl.pos, device="cuda", dtype=dt)
    q = torch.tensor(sl.q, device="cuda", dtype=dt)
    e, phi, F = slab.compute_realspace(pos, q)
    out = {"E": float(e.item()), "phi": phi.double().cpu().numpy(), "F": F.double().cpu().numpy(),
           "status": slab.status(), "pos": pos.double().cpu().numpy()}
    slab.close()
    return out


def test_realspace_fp64_small(qslab, soe16):
    sl = workloads.small_full()                      # 1000 ions in 30 x 30 x 10
    got = _rs(qslab, sl, "fp64", 0.3, 10.0, soe16)
    ref = ewald2d.realspace(sl.pos, sl.q, sl.box, 0.3, 10.0)
    assert got["status"] == 0
    assert abs(got["E"] - ref["E"]) <= 1e-10 * abs(ref["E"])
    assert _maxrel(got["phi"], ref["phi"]) <= 1e-10
    assert _maxrel(got["F"], ref["F"]) <= 1e-10


def test_realspace_fp32_small(qslab, soe16):
    sl = workloads.small_full()
    got = _rs(qslab, sl, "fp32c", 0.3, 10.0, soe16)
    ref = ewald2d.realspace(got["pos"], sl.q, sl.box, 0.3, 10.0)
    assert got["status"] == 0
    assert abs(got["E"] - ref["E"]) <= 1e-6 * abs(ref["E"])
    assert _rmsrel(got["phi"], ref["phi"]) <= 1e-5
    assert _rmsrel(got["F"], ref["F"]) <= 1e-5


def test_realspace_edges(qslab, soe16):
    """Particles on cell faces, on both walls and outside the box in x, y;
    a tiny system with rc = L/3 exactly."""
    box = (9.0, 12.0, 4.0)
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 4.0], [8.999, 11.999, 2.0], [-1.5, 13.0, 1.0],
                    [6.0, 8.0, 3.0], [4.5, 6.0, 0.5]])
    q = np.array([1.0, -1.0, 1.0, -1.0, 0.5, -0.5])
    sl = workloads.Slab("edge", pos, q, box, 0.8, 16)
    got = _rs(qslab, sl, "fp64", 0.8, 3.0, soe16)
    ref = ewald2d.realspace(pos, q, box, 0.8, 3.0)
    assert got["status"] == 0
    assert abs(got["E"] - ref["E"]) <= 1e-12 * max(abs(ref["E"]), 1.0)
    assert np.abs(got["phi"] - ref["phi"]).max() <= 1e-12 * max(np.abs(ref["phi"]).max(), 1.0)
    assert np.abs(got["F"] - ref["F"]).max() <= 1e-12 * max(np.abs(ref["F"]).max(), 1.0)


def test_total_alpha_independent(qslab):
    """Real space + long range on the GPU (FP64, SOE M = 16, kc at a 1e-14
    Gaussian tail, rc = 6.5/alpha) gives the same total energy, potentials
    and forces for two splitting parameters, and equals the oracle's exact
    Ewald2D total."""
    from paper_2403_01521_gb300.soe import load_soe
    soe = load_soe(16, "accurate")
    sl = workloads.uniform_slab(300, (30.0, 30.0, 10.0), 55, alpha=0.7)
    tot = []
    for alpha in (0.7, 0.9):
        rc = 6.5 / alpha
        kc = lattice.kcut_for_tail(alpha, 1e-14)
        slab = qslab.QSlab(0, "fp64").configure(sl.box, alpha, soe, kcut=kc, rcut=rc)
        pos = torch.tensor(sl.pos, device="cuda")
        q = torch.tensor(sl.q, device="cuda")
        e1, p1, f1 = slab.compute(pos, q)
        e2, p2, f2 = slab.compute_realspace(pos, q)
        assert slab.status() == 0
        tot.append((float(e1.item() + e2.item()), (p1 + p2).cpu().numpy(), (f1 + f2).cpu().numpy()))
        slab.close()
    (Ea, pa, fa), (Eb, pb, fb) = tot
    assert abs(Ea - Eb) <= 1e-9 * abs(Ea)
    assert _maxrel(pa, pb) <= 1e-8
    assert _maxrel(fa, fb) <= 1e-8
    mx, my = lattice.full_modes(sl.box[0], sl.box[1], lattice.kcut_for_tail(0.7, 1e-14))
    lr = ewald2d.ewald2d_longrange(sl.pos, sl.q, sl.box, 0.7, mx, my)
    rs = ewald2d.realspace(sl.pos, sl.q, sl.box, 0.7, 6.5 / 0.7)
    assert abs(Ea - (lr["E"] + rs["E"])) <= 1e-9 * abs(Ea)


def test_realspace_fp32_at_scale(qslab, soe16):
    """N = 1e5 ions in 100 x 100 x 20, alpha = 0.25, rc = 10 (the FP32
    full-k workload with its real-space cut-off): 64 particles against the
    oracle on the FP32-rounded inputs; bitwise-repeatable sums."""
    sl = workloads.fp32_full()
    slab = qslab.QSlab(0, "fp32c").configure(sl.box, 0.25, soe16, kcut=1.0, rcut=10.0)
    pos = torch.tensor(sl.pos, device="cuda", dtype=torch.float32)
    q = torch.tensor(sl.q, device="cuda", dtype=torch.float32)
    e, phi, F = slab.compute_realspace(pos, q)
    e2, phi2, F2 = slab.compute_realspace(pos, q)
    assert slab.status() == 0
    assert torch.equal(e, e2) and torch.equal(phi, phi2) and torch.equal(F, F2)
    idx = np.random.default_rng(0).choice(sl.N, 64, replace=False)
    pos64 = pos.double().cpu().numpy()
    ref = ewald2d.realspace_at(pos64, sl.q, sl.box, 0.25, 10.0, idx)
    assert _rmsrel(phi.double().cpu().numpy()[idx], ref["phi"]) <= 1e-5
    assert _rmsrel(F.double().cpu().numpy()[idx], ref["F"]) <= 1e-5
    slab.close()


def test_realspace_errors(qslab, soe16):
    sl = workloads.small_full()
    pos = torch.tensor(sl.pos, device="cuda")
    q = torch.tensor(sl.q, device="cuda")
    slab = qslab.QSlab(0, "fp64").configure(sl.box, 0.3, soe16, kcut=1.0)
    with pytest.raises(qslab.QslabError) as e:              # rc not set
        slab.compute_realspace(pos, q)
    assert e.value.code == -2
    qslab.qslab_set_rcut(slab.h, 10.5)                       # 30/10.5 < 3 cells
    with pytest.raises(qslab.QslabError) as e:
        slab.compute_realspace(pos, q)
    assert e.value.code == -1
    qslab.qslab_set_rcut(slab.h, 10.0)
    p2 = sl.pos.copy()
    p2[5, 2] = 11.0                                          # z > Lz
    slab.compute_realspace(torch.tensor(p2, device="cuda"), q)
    assert slab.status() == -4
    slab.close()
