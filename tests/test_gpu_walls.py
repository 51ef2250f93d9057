"""GPU parity with charged walls (Section 2.4, Thm 2.4): the long-range path
of particles that are not neutral on their own, plus the particle-slab
potential of uniform and Fourier-mode wall densities, against the FP64
oracle (sorted recursion for the particles, Thm 2.4 for the walls)."""
import numpy as np
import pytest

import workloads
from oracle import lattice, soe_ewald2d, walls

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


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


MODES = np.array([[1, 0], [0, 2], [3, -1]])
BOT = np.array([0.002 + 0.001j, -0.0015j, 0.0008])
TOP = np.array([-0.001 + 0.0005j, 0.002, 0.0004 - 0.0009j])


def _oracle(pos, q, box, alpha, soe, kc, sw, modes=(), bot=(), top=()):
    s, w = soe
    pp = soe_ewald2d.soe_full(pos, q, box, alpha, s, w, kc=kc)
    ps = walls.wall_potential(pos, q, box, sw[0], sw[1], modes, bot, top)
    return {"E": pp["E"] + ps["E"], "phi": pp["phi"] + ps["phi"], "F": pp["F"] + ps["F"]}


def _gpu(qslab, sl, prec, soe, kc, sw, modes=None, bot=None, top=None, chunk=0):
    slab = qslab.QSlab(0, prec).configure(sl.box, sl.alpha, soe, kcut=kc).tuning(chunk, 0)
    slab.set_walls(sw[0], sw[1], modes, bot, top)
    dt = torch.float64 if prec == "fp64" else torch.float32
    pos = torch.tensor(sl.pos, device="cuda", dtype=dt)
    q = torch.tensor(sl.q, device="cuda", dtype=dt)
    e, phi, F = slab.compute(pos, q)
    out = {"E": float(e.item()), "phi": phi.double().cpu().numpy(), "F": F.double().cpu().numpy(),
           "status": slab.status(), "pos": pos.double().cpu().numpy(), "q": q.double().cpu().numpy()}
    slab.close()
    return out


@pytest.mark.parametrize("chunk", [0, 64])
def test_cations_uniform_walls_fp64(qslab, soe16, chunk):
    """436 cations neutralised by the top wall (sigma_top = -0.0436): the
    cation-only system of Section 5.2."""
    sl = workloads.cations_walls()
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    got = _gpu(qslab, sl, "fp64", soe16, kc, sl.walls, chunk=chunk)
    ref = _oracle(sl.pos, sl.q, sl.box, sl.alpha, soe16, kc, sl.walls)
    assert got["status"] == 0
    assert abs(got["E"] - ref["E"]) <= FP64_TOL * abs(ref["E"])
    assert _maxrel(got["phi"], ref["phi"]) <= FP64_TOL
    assert _maxrel(got["F"], ref["F"]) <= FP64_TOL


def test_electrolyte_mode_walls_fp64(qslab, soe16):
    """1:1 electrolyte between walls of density +-0.0218 plus three Fourier
    modes on each wall."""
    sl = workloads.electrolyte_walls()
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    got = _gpu(qslab, sl, "fp64", soe16, kc, sl.walls, MODES, BOT, TOP)
    ref = _oracle(sl.pos, sl.q, sl.box, sl.alpha, soe16, kc, sl.walls, MODES, BOT, TOP)
    assert got["status"] == 0
    assert abs(got["E"] - ref["E"]) <= FP64_TOL * abs(ref["E"])
    assert _maxrel(got["phi"], ref["phi"]) <= FP64_TOL
    assert _maxrel(got["F"], ref["F"]) <= FP64_TOL


def test_mode_walls_fp32(qslab, soe16):
    """FP32C: 8720 cations in 200 x 200 x 30 with the top wall neutralising
    them plus Fourier modes, against the oracle on the FP32-rounded inputs."""
    sl = workloads.cations_walls(n=8720, L=200.0)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    got = _gpu(qslab, sl, "fp32c", soe16, kc, sl.walls, MODES, BOT, TOP)
    ref = _oracle(got["pos"], got["q"], sl.box, sl.alpha, soe16, kc, sl.walls, MODES, BOT, TOP)
    assert got["status"] == 0
    assert abs(got["E"] - ref["E"]) <= 1e-6 * abs(ref["E"])
    assert _rmsrel(got["phi"], ref["phi"]) <= 1e-5
    assert _rmsrel(got["F"], ref["F"]) <= 1e-5


def test_walls_batched_fp64(qslab, soe16):
    """Three slabs of different boxes with net charges +1, +2, +3 and walls
    of total density -1/100 per unit area: every slab is neutral with its
    walls, and each equals the oracle on that slab alone."""
    rng = np.random.default_rng(17)
    boxes = [(10.0, 10.0, 6.0), (20.0, 10.0, 4.0), (10.0, 30.0, 8.0)]
    sw = (-0.004, -0.006)
    alpha = 0.5
    kc = lattice.kcut_for_tail(alpha, 1e-8)
    slabs = []
    for b, net in zip(boxes, (1, 2, 3)):
        n = 40 + net
        pos = np.column_stack([rng.uniform(0, b[0], n), rng.uniform(0, b[1], n), rng.uniform(0, b[2], n)])
        q = np.where(np.arange(n) < (n + net) // 2, 1.0, -1.0)
        slabs.append((pos, q, b))
    off = np.concatenate([[0], np.cumsum([len(s[1]) for s in slabs])]).astype(np.int64)
    slab = qslab.QSlab(0, "fp64").configure(boxes[0], alpha, soe16, kcut=kc)
    slab.set_walls(*sw, MODES[:2], BOT[:2], TOP[:2])
    pos = torch.tensor(np.concatenate([s[0] for s in slabs]), device="cuda")
    q = torch.tensor(np.concatenate([s[1] for s in slabs]), device="cuda")
    e, phi, F = slab.compute_batched(pos, q, off, np.array(boxes))
    assert slab.status() == 0
    e, phi, F = e.cpu().numpy(), phi.cpu().numpy(), F.cpu().numpy()
    for r, (p, qq, b) in enumerate(slabs):
        ref = _oracle(p, qq, b, alpha, soe16, kc, sw, MODES[:2], BOT[:2], TOP[:2])
        sl = slice(off[r], off[r + 1])
        assert abs(e[r] - ref["E"]) <= FP64_TOL * abs(ref["E"])
        assert _maxrel(phi[sl], ref["phi"]) <= FP64_TOL
        assert _maxrel(F[sl], ref["F"]) <= FP64_TOL
    slab.close()


def test_walls_energy_gradient_fp64(qslab, soe16):
    """F = -dE/dr and phi = dE/dq with walls (central differences of the GPU
    energy, FP64)."""
    sl = workloads.cations_walls(n=60, L=20.0)
    sl.alpha = 0.4
    kc = lattice.kcut_for_tail(sl.alpha, 1e-10)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, kcut=kc)
    slab.set_walls(*sl.walls, MODES, BOT, TOP)
    slab.set_neutrality_tol(-1.0)     # q is perturbed below
    pos = torch.tensor(sl.pos, device="cuda")
    q = torch.tensor(sl.q, device="cuda")
    e, phi, F = slab.compute(pos, q)
    F = F.cpu().numpy()
    phi = phi.cpu().numpy()
    h = 1e-5
    for i, d in [(0, 0), (7, 1), (13, 2), (42, 2)]:
        p1, p2 = pos.clone(), pos.clone()
        p1[i, d] += h
        p2[i, d] -= h
        fd = -(slab.compute(p1, q)[0].item() - slab.compute(p2, q)[0].item()) / (2 * h)
        assert abs(fd - F[i, d]) <= 1e-6 * max(1.0, abs(F[i, d]))
    q1, q2 = q.clone(), q.clone()
    q1[5] += h
    q2[5] -= h
    fd = (slab.compute(pos, q1)[0].item() - slab.compute(pos, q2)[0].item()) / (2 * h)
    assert abs(fd - phi[5]) <= 1e-6 * max(1.0, abs(phi[5]))
    slab.close()


def test_walls_neutrality_and_input_errors(qslab, soe16):
    sl = workloads.cations_walls()
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, kcut=kc)
    pos = torch.tensor(sl.pos, device="cuda")
    q = torch.tensor(sl.q, device="cuda")
    slab.compute(pos, q)                                  # cations alone
    assert slab.status() == qslab.QSLAB_ERR_NONNEUTRAL
    slab.set_walls(0.0, -0.04)                            # walls short of neutral
    slab.compute(pos, q)
    assert slab.status() == qslab.QSLAB_ERR_NONNEUTRAL
    slab.set_walls(*sl.walls)                             # neutral together
    slab.compute(pos, q)
    assert slab.status() == 0
    slab.set_walls(None, None)                            # cleared
    slab.compute(pos, q)
    assert slab.status() == qslab.QSLAB_ERR_NONNEUTRAL
    for modes, bot, top in [([[0, 0]], [0.1], [0.1]),             # the zero mode
                            ([[1, 2], [-1, -2]], [0.1, 0.1], [0, 0]),   # m and -m
                            ([[1, 2], [1, 2]], [0.1, 0.1], [0, 0]),     # twice
                            (np.ones((65, 2)) * np.arange(65)[:, None] + 1, np.zeros(65), np.zeros(65))]:
        with pytest.raises(qslab.QslabError) as e:
            slab.set_walls(0.0, 0.0, np.asarray(modes), bot, top)
        assert e.value.code == qslab.QSLAB_ERR_INVALID_ARG
    with pytest.raises(qslab.QslabError):
        slab.set_walls(float("nan"), 0.0)
    slab.close()
