"""GPU parity of the virial tensor W = (xx, yy, zz, xy, xz, yz) against the
FP64 oracle (oracle/virial.py) on the same seeded inputs, through the C ABI.

Tolerances, relative to the scale max(|W_xx|, |W_yy|, |W_zz|) of the oracle's
tensor: 1e-10 on the FP64 path. On the compensated-FP32 path the lateral
components are sums over modes of k-derivatives of the FP32 recurrences'
pair sums, rounded like the energy: 2e-5 of the tensor's scale. The
components zz, xz, yz are sums of z_i F_i,a over the FP32 forces, whose
budget is 1e-5 relative RMS: independent force errors of that size move such
a sum by about 1e-5 (sum_i z_i^2 F_i,a^2)^{1/2}, which is added to their
tolerance (twice that, for margin).
"""
import numpy as np
import pytest

import workloads
from oracle import lattice, virial

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORDER = ("xx", "yy", "zz", "xy", "xz", "yz")
FP64_TOL = 1e-10
FP32_TOL = 2e-5


@pytest.fixture(scope="module")
def qslab():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01521_gb300 as q
    q.load()
    return q


def _vec(W):
    return np.array([W[k] for k in ORDER])


def _scale(W):
    return max(abs(W["xx"]), abs(W["yy"]), abs(W["zz"]))


def _err(got, W):
    return float(np.abs(np.asarray(got) - _vec(W)).max() / _scale(W))


def _check_fp32(got, ref):
    """FP32 bound: FP32_TOL of the scale, plus for zz, xz, yz the propagated
    force budget 2e-5 (sum_i z_i^2 F_i,a^2)^{1/2} (oracle forces)."""
    W = ref["W"]
    z = np.asarray(ref["pos"])[:, 2]
    F = np.asarray(ref["F"])
    prop = {"zz": F[:, 2], "xz": F[:, 0], "yz": F[:, 1]}
    for j, k in enumerate(ORDER):
        tol = FP32_TOL * _scale(W)
        if k in prop:
            tol += 2e-5 * float(np.sqrt(((z * prop[k]) ** 2).sum()))
        assert abs(got[j] - W[k]) <= tol, (k, got[j], W[k], tol)


def _tensors(sl, dt):
    pos = torch.tensor(sl.pos, device="cuda", dtype=dt)
    q = torch.tensor(sl.q, device="cuda", dtype=dt)
    return pos, q


def _gpu_virial(qslab, sl, prec, soe, kc=None, rbe=None, tuning=(0, 0), walls=None):
    slab = qslab.QSlab(0, prec).configure(sl.box, sl.alpha, soe, kcut=kc, rbe=rbe)
    slab.tuning(*tuning)
    if walls is not None:
        slab.set_walls(*walls)
    dt = torch.float64 if prec == "fp64" else torch.float32
    pos, q = _tensors(sl, dt)
    e, phi, F, W = slab.compute_virial(pos, q)
    out = {"E": float(e.item()), "F": F.double().cpu().numpy(), "W": W.cpu().numpy(),
           "status": slab.status(), "pos": pos.double().cpu().numpy(),
           "q": q.double().cpu().numpy()}
    if rbe is not None:
        out["modes"] = slab.sampled_modes()
    slab.close()
    return out


@pytest.mark.parametrize("tuning", [(0, 0), (32, 32), (96, 64)])
def test_fp64_full_k(qslab, soe16, tuning):
    sl = workloads.small_full()
    kc = lattice.kcut_for_tail(sl.alpha, sl.tail)
    got = _gpu_virial(qslab, sl, "fp64", soe16, kc=kc, tuning=tuning)
    assert got["status"] == 0
    ref = virial.soe_full_virial(sl.pos, sl.q, sl.box, sl.alpha, *soe16, kc=kc)
    assert abs(got["E"] - ref["E"]) <= FP64_TOL * abs(ref["E"])
    assert _err(got["W"], ref["W"]) <= FP64_TOL
    assert abs(ref["W"]["xy"]) > 1e-6 * _scale(ref["W"])


def test_fp64_virial_call_keeps_outputs(qslab, soe16):
    """The virial call returns the same energy, potentials and forces as the
    plain call, bit for bit (the virial kernels only read them)."""
    sl = workloads.uniform_slab(900, (24.0, 20.0, 8.0), 41, alpha=0.35)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, kcut=kc)
    pos, q = _tensors(sl, torch.float64)
    e0, p0, f0 = slab.compute(pos, q)
    e1, p1, f1, _ = slab.compute_virial(pos, q)
    assert slab.status() == 0
    assert torch.equal(e0, e1) and torch.equal(p0, p1) and torch.equal(f0, f1)
    slab.close()


def test_fp64_random_batch_same_sample(qslab, soe16):
    sl = workloads.uniform_slab(2000, (40.0, 36.0, 12.0), 42, alpha=0.2)
    got = _gpu_virial(qslab, sl, "fp64", soe16, rbe=(40, 7))
    assert got["status"] == 0
    mx, my, _ = got["modes"]
    ref = virial.soe_rbe_virial(sl.pos, sl.q, sl.box, sl.alpha, *soe16, mx, my, 40)
    assert _err(got["W"], ref["W"]) <= FP64_TOL


def test_fp64_walls_net_charge(qslab, soe16):
    """Cations only between charged walls (Section 5.2's system), plus two
    wall modes: particle-particle and particle-slab virials together, with the
    top wall's L_z term (Thm 2.4)."""
    sl = workloads.cations_walls(n=300, L=60.0)
    A = sl.box[0] * sl.box[1]
    sb0, st0 = -0.25 * sl.N / A, -0.75 * sl.N / A
    modes = [(1, 0), (2, -1)]
    sb = [0.01 + 0.004j, -0.006j]
    st = [0.008 - 0.003j, 0.005 + 0.002j]
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    got = _gpu_virial(qslab, sl, "fp64", soe16, kc=kc,
                      walls=(sb0, st0, modes, [complex(c) for c in sb], [complex(c) for c in st]))
    assert got["status"] == 0
    pp = virial.soe_full_virial(sl.pos, sl.q, sl.box, sl.alpha, *soe16, kc=kc)
    ps = virial.wall_virial(sl.pos, sl.q, sl.box, sb0, st0, modes, sb, st)
    W = {k: pp["W"][k] + ps["W"][k] for k in ORDER}
    assert abs(got["E"] - (pp["E"] + ps["E"])) <= FP64_TOL * abs(pp["E"] + ps["E"])
    assert _err(got["W"], W) <= FP64_TOL


def test_fp64_batched(qslab, soe16):
    """Three slabs of different size and box, one of them empty, in one call:
    each slab's virial equals the oracle's on that slab alone."""
    sls = [workloads.uniform_slab(600, (20.0, 22.0, 6.0), 43, alpha=0.3),
           None,
           workloads.uniform_slab(1100, (30.0, 26.0, 10.0), 44, alpha=0.3)]
    kc = lattice.kcut_for_tail(0.3, 1e-8)
    slab = qslab.QSlab(0, "fp64").configure((1.0, 1.0, 1.0), 0.3, soe16, kcut=kc)
    pos = np.concatenate([s.pos for s in sls if s is not None])
    q = np.concatenate([s.q for s in sls if s is not None])
    off = [0, 600, 600, 1700]
    boxes = [sls[0].box, (15.0, 15.0, 5.0), sls[2].box]
    e, _, _, W = slab.compute_batched_virial(torch.tensor(pos, device="cuda"),
                                             torch.tensor(q, device="cuda"), off, boxes)
    assert slab.status() == 0
    W = W.cpu().numpy()
    assert np.all(W[1] == 0.0)
    for r in (0, 2):
        s = sls[r]
        ref = virial.soe_full_virial(s.pos, s.q, s.box, s.alpha, *soe16, kc=kc)
        assert _err(W[r], ref["W"]) <= FP64_TOL
    slab.close()


def test_fp64_virial_theorem(qslab, soe16):
    """Long range plus real space on the GPU: trace W = E, the Coulomb virial
    theorem (alpha-independent setting: rc = 4.6/alpha, k tail 1e-12)."""
    from paper_2403_01521_gb300.soe import load_soe
    sl = workloads.uniform_slab(800, (30.0, 30.0, 10.0), 45, alpha=0.5)
    soe = load_soe(16, "accurate")
    kc = lattice.kcut_for_tail(sl.alpha, 1e-12)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe, kcut=kc, rcut=9.2)
    pos, q = _tensors(sl, torch.float64)
    e, _, _, W = slab.compute_virial(pos, q)
    es, _, _, Ws = slab.compute_realspace_virial(pos, q)
    assert slab.status() == 0
    Wt = W.cpu().numpy() + Ws.cpu().numpy()
    E = float(e.item() + es.item())
    assert abs(Wt[0] + Wt[1] + Wt[2] - E) <= 1e-8 * np.abs(Wt[:3]).max()
    slab.close()


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32c", FP32_TOL)])
def test_realspace_virial(qslab, soe16, prec, tol):
    sl = workloads.small_full()
    slab = qslab.QSlab(0, prec).configure(sl.box, sl.alpha, soe16,
                                          kcut=lattice.kcut_for_tail(sl.alpha, 1e-8), rcut=10.0)
    dt = torch.float64 if prec == "fp64" else torch.float32
    pos, q = _tensors(sl, dt)
    e, _, _, W = slab.compute_realspace_virial(pos, q)
    assert slab.status() == 0
    ref = virial.realspace_virial(pos.double().cpu().numpy(), q.double().cpu().numpy(), sl.box,
                                  sl.alpha, 10.0)
    assert _err(W.cpu().numpy(), ref["W"]) <= tol
    slab.close()


def test_fp32_full_k(qslab, soe16):
    sl = workloads.uniform_slab(10000, (100.0, 100.0, 20.0), 46, alpha=0.25)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    got = _gpu_virial(qslab, sl, "fp32c", soe16, kc=kc)
    assert got["status"] == 0
    ref = virial.soe_full_virial(got["pos"], got["q"], sl.box, sl.alpha, *soe16, kc=kc)
    ref["pos"] = got["pos"]
    _check_fp32(got["W"], ref)


def test_fp32_random_batch_1e6(qslab, soe16):
    """The N = 1e6 random-batch workload (400 x 400 x 50, alpha = 0.1) with a
    batch of 12 modes, so that the oracle's recursion stays in seconds."""
    sl = workloads.rbe_large()
    got = _gpu_virial(qslab, sl, "fp32c", soe16, rbe=(12, 3))
    assert got["status"] == 0
    mx, my, _ = got["modes"]
    ref = virial.soe_rbe_virial(got["pos"], got["q"], sl.box, sl.alpha, *soe16, mx, my, 12)
    ref["pos"] = got["pos"]
    _check_fp32(got["W"], ref)


def test_fp32_confined_m24(qslab):
    """The strongly confined slab (Lz = 2, wall layers, Gaussian charges) with
    M = 24, reduced to N = 1e4 in a 42 x 42 box (the same density) for the
    oracle."""
    from paper_2403_01521_gb300.soe import load_soe
    soe = load_soe(24)
    full = workloads.confined()
    L = 200.0 * np.sqrt(1e4 / full.N)
    sel = np.flatnonzero((full.pos[:, 0] < L) & (full.pos[:, 1] < L))
    pos = full.pos[sel].copy()
    q = full.q[sel] - full.q[sel].mean()
    sl = workloads.Slab("confined_small", pos, q, (L, L, 2.0), 0.2, 24)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    got = _gpu_virial(qslab, sl, "fp32c", soe, kc=kc)
    assert got["status"] == 0
    ref = virial.soe_full_virial(got["pos"], got["q"], sl.box, sl.alpha, *soe, kc=kc)
    ref["pos"] = got["pos"]
    _check_fp32(got["W"], ref)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_fp64_tiny_slabs(qslab, soe16, n):
    """N = 1, 2, 3 (a lone particle is neutral only with walls; N = 2, 3 with
    equal z for two of them): the virial against the oracle."""
    box = (9.0, 8.0, 4.0)
    pos = np.array([[1.0, 2.0, 1.5], [6.0, 7.0, 1.5], [3.0, 1.0, 3.0]])[:n]
    q = np.array([1.0, -1.0, 0.0])[:n] if n > 1 else np.array([1.0])
    if n == 3:
        q = np.array([1.0, -2.0, 1.0])
    sl = workloads.Slab("tiny", pos, q, box, 0.5, 16)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    walls = None
    if n == 1:
        A = box[0] * box[1]
        walls = (-0.5 / A, -0.5 / A, [], [], [])
    got = _gpu_virial(qslab, sl, "fp64", soe16, kc=kc, walls=walls)
    assert got["status"] == 0
    ref = virial.soe_full_virial(pos, q, box, sl.alpha, *soe16, kc=kc)
    W = ref["W"]
    if walls is not None:
        ps = virial.wall_virial(pos, q, box, walls[0], walls[1])
        W = {k: W[k] + ps["W"][k] for k in ORDER}
    assert _err(got["W"], W) <= FP64_TOL


def test_fp64_metropolis_sample(qslab, soe16):
    """The virial on the paper's Metropolis k-sampler (App. G): the oracle on
    the modes the chain drew."""
    sl = workloads.uniform_slab(1500, (36.0, 36.0, 12.0), 47, alpha=0.2)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, rbe=(50, 3))
    slab.sampler("metropolis", thin=2)
    pos, q = _tensors(sl, torch.float64)
    e, _, _, W = slab.compute_virial(pos, q)
    assert slab.status() == 0
    mx, my, _ = slab.sampled_modes()
    ref = virial.soe_rbe_virial(sl.pos, sl.q, sl.box, sl.alpha, *soe16, mx, my, 50)
    assert _err(W.cpu().numpy(), ref["W"]) <= FP64_TOL
    slab.close()


def test_fp64_virial_theorem_with_walls(qslab):
    """Particles with net charge between charged walls (uniform parts and two
    Fourier modes), long range plus real space on the GPU: trace W = E, which
    needs the walls to move with the box, the top wall's L_z term included."""
    from paper_2403_01521_gb300.soe import load_soe
    soe = load_soe(16, "accurate")
    rng = np.random.default_rng(48)
    n = 600
    box = (30.0, 30.0, 10.0)
    pos = np.column_stack([rng.random(n) * box[0], rng.random(n) * box[1], rng.random(n) * box[2]])
    q = np.where(rng.random(n) < 0.6, 1.0, -1.0)
    A = box[0] * box[1]
    Q = q.sum()
    sb0, st0 = -0.3 * Q / A, -0.7 * Q / A
    modes = [(1, 0), (1, 2)]
    sb = [0.004 + 0.002j, -0.003j]
    st = [0.002 - 0.001j, 0.003 + 0.001j]
    alpha = 0.5
    kc = lattice.kcut_for_tail(alpha, 1e-12)
    slab = qslab.QSlab(0, "fp64").configure(box, alpha, soe, kcut=kc, rcut=9.2)
    slab.set_walls(sb0, st0, modes, sb, st)
    pt = torch.tensor(pos, device="cuda")
    qt = torch.tensor(q, device="cuda")
    e, _, _, W = slab.compute_virial(pt, qt)
    es, _, _, Ws = slab.compute_realspace_virial(pt, qt)
    assert slab.status() == 0
    Wt = W.cpu().numpy() + Ws.cpu().numpy()
    E = float(e.item() + es.item())
    assert abs(Wt[0] + Wt[1] + Wt[2] - E) <= 1e-8 * np.abs(Wt[:3]).max()
    slab.close()
