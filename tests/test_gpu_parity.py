"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element.

Tolerances (relative): FP64 path 1e-10 for the energy and for the max-norm
of phi and F; compensated-FP32 path 1e-6 for the energy and 1e-5 for the RMS
of phi and F at the N = 1e6 workload. The FP32 path is compared with the
oracle run on the same FP32-rounded inputs.

Energy scale of a random-batch sample: the estimator's energy fluctuates by
thousands between samples around its expectation (the full-k energy), and a
single sample can land near zero, so its errors are measured relative to
the expectation |E_full-k| of the configuration (tests/golden/).
"""
import math

import numpy as np
import pytest

import workloads
from oracle import lattice, soe_ewald2d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_E_TOL = 1e-6
FP32_RMS_TOL = 1e-5


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


def _run(qslab, sl, prec, soe, kc=None, rbe=None, tuning=(0, 0)):
    slab = qslab.QSlab(0, prec).configure(sl.box, sl.alpha, soe, kcut=kc, rbe=rbe)
    slab.tuning(*tuning)
    dt = torch.float64 if prec == "fp64" else torch.float32
    pos = torch.tensor(sl.pos, device="cuda", dtype=dt)
    q = torch.tensor(sl.q, device="cuda", dtype=dt)
    e, phi, F = slab.compute(pos, q)
    status = slab.status()
    out = {"E": float(e.item()), "phi": phi.double().cpu().numpy(), "F": F.double().cpu().numpy(),
           "status": status, "pos": pos.double().cpu().numpy(), "q": q.double().cpu().numpy()}
    if rbe is not None:
        out["modes"] = slab.sampled_modes()
    slab.close()
    return out


def _check_fp64(got, ref, escale=None):
    assert got["status"] == 0
    assert abs(got["E"] - ref["E"]) <= FP64_TOL * (escale or abs(ref["E"]))
    assert _maxrel(got["phi"], ref["phi"]) <= FP64_TOL
    assert _maxrel(got["F"], ref["F"]) <= FP64_TOL


def _check_fp32(got, ref, escale=None, etol=FP32_E_TOL):
    assert got["status"] == 0
    assert abs(got["E"] - ref["E"]) <= etol * (escale or abs(ref["E"]))
    assert _rmsrel(got["phi"], ref["phi"]) <= FP32_RMS_TOL
    assert _rmsrel(got["F"], ref["F"]) <= FP32_RMS_TOL


def _golden(name):
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def small_full():
    return workloads.small_full()


@pytest.fixture(scope="module")
def small_ref(small_full, soe16):
    sl = small_full
    kc = lattice.kcut_for_tail(sl.alpha, sl.tail)
    return soe_ewald2d.soe_full(sl.pos, sl.q, sl.box, sl.alpha, *soe16, kc=kc)


# launch shapes: automatic, one warp of modes with 32-particle chunks,
# ragged chunks (1000 = 10*96 + 40), full-size chunks
@pytest.mark.parametrize("tuning", [(0, 0), (32, 32), (96, 64), (256, 256)])
def test_fp64_full_k_small(qslab, small_full, small_ref, soe16, tuning):
    sl = small_full
    kc = lattice.kcut_for_tail(sl.alpha, sl.tail)
    got = _run(qslab, sl, "fp64", soe16, kc=kc, tuning=tuning)
    _check_fp64(got, small_ref)


def test_fp64_modes_count(qslab, small_full, soe16):
    sl = small_full
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16,
                                              kcut=lattice.kcut_for_tail(sl.alpha, sl.tail))
    assert slab.num_modes() == 240          # half of the 480 lattice vectors
    slab.close()


@pytest.mark.parametrize("M,kind", [(8, "conditioned"), (24, "conditioned"), (16, "accurate")])
def test_fp64_other_soe_tables(qslab, M, kind):
    from paper_2403_01521_gb300.soe import load_soe
    soe = load_soe(M, kind)
    sl = workloads.uniform_slab(700, (25.0, 20.0, 9.0), 31, alpha=0.4)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    ref = soe_ewald2d.soe_full(sl.pos, sl.q, sl.box, sl.alpha, *soe, kc=kc)
    _check_fp64(_run(qslab, sl, "fp64", soe, kc=kc, tuning=(64, 0)), ref)


def test_fp64_edge_cases(qslab, soe16):
    """Tiny N, coincident z, particles on both walls, x,y outside the box."""
    box = (8.0, 9.0, 4.0)
    cases = [
        (np.array([[1.0, 2.0, 1.5], [3.0, 7.0, 2.5]]), np.array([1.0, -1.0])),
        (np.array([[1.0, 2.0, 1.5], [3.0, 7.0, 1.5], [5.0, 1.0, 3.0]]), np.array([1.0, -2.0, 1.0])),
        (np.array([[1.0, 2.0, 0.0], [3.0, 7.0, 4.0], [6.0, 5.0, 0.0], [2.0, 2.0, 4.0]]),
         np.array([1.0, -1.0, 1.0, -1.0])),
        (np.array([[-3.0, 20.0, 1.0], [11.0, -4.5, 3.0]]), np.array([0.5, -0.5])),
    ]
    for pos, q in cases:
        sl = workloads.Slab("edge", pos, q, box, 0.5, 16)
        kc = lattice.kcut_for_tail(0.5, 1e-8)
        ref = soe_ewald2d.soe_full(pos, q, box, 0.5, *soe16, kc=kc)
        got = _run(qslab, sl, "fp64", soe16, kc=kc)
        assert got["status"] == 0
        assert abs(got["E"] - ref["E"]) <= FP64_TOL * max(abs(ref["E"]), 1.0)
        assert np.abs(got["phi"] - ref["phi"]).max() <= FP64_TOL * max(np.abs(ref["phi"]).max(), 1.0)
        # with exactly equal z the k = 0 force depends on the tie order at the
        # eps level (the SOE slope at z = 0 is -sum(w s)/sqrt(pi) ~ eps)
        assert np.abs(got["F"] - ref["F"]).max() <= 1e-8 * max(np.abs(ref["F"]).max(), 1.0)


def test_single_particle(qslab, soe16):
    """N = 1 (not neutral: the check is switched off): only the j = i constants."""
    box = (10.0, 10.0, 5.0)
    pos = np.array([[2.0, 3.0, 1.0]])
    q = np.array([1.0])
    kc = lattice.kcut_for_tail(0.5, 1e-8)
    ref = soe_ewald2d.soe_full(pos, q, box, 0.5, *soe16, kc=kc)
    slab = qslab.QSlab(0, "fp64").configure(box, 0.5, soe16, kcut=kc)
    qslab.qslab_set_neutrality_tol(slab.h, -1.0)
    e, phi, F = slab.compute(torch.tensor(pos, device="cuda"), torch.tensor(q, device="cuda"))
    assert slab.status() == 0
    assert abs(float(e.item()) - ref["E"]) <= 1e-12 * abs(ref["E"])
    assert np.abs(F.cpu().numpy()).max() <= 1e-12
    slab.close()


def test_fp64_rbe_same_sample(qslab, soe16):
    """RBE: the device sampler draws exactly the oracle's modes, and the
    estimator on that sample matches the oracle (Eqs. 4.7-4.9)."""
    sl = workloads.uniform_slab(2000, (40.0, 40.0, 20.0), 77, alpha=0.2)
    got = _run(qslab, sl, "fp64", soe16, rbe=(200, 4242))
    mx, my, weight = got["modes"]
    omx, omy = lattice.sample_modes(200, 4242, 0, sl.alpha, 40.0, 40.0)
    assert (mx == omx).all() and (my == omy).all()
    assert abs(weight - lattice.H_direct(sl.alpha, 40.0, 40.0) / 200) <= 1e-12 * weight
    ref = soe_ewald2d.soe_rbe(sl.pos, sl.q, sl.box, sl.alpha, *soe16, omx, omy)
    _check_fp64(got, ref)


def test_rbe_counter_and_resume(qslab, soe16):
    """Each call advances the counter; restoring (seed, counter) replays a sample."""
    sl = workloads.uniform_slab(500, (30.0, 30.0, 10.0), 3, alpha=0.3)
    slab = qslab.QSlab(0, "fp32c").configure(sl.box, sl.alpha, soe16, rbe=(50, 9))
    pos = torch.tensor(sl.pos, device="cuda", dtype=torch.float32)
    q = torch.tensor(sl.q, device="cuda", dtype=torch.float32)
    draws = []
    for call in range(3):
        slab.compute(pos, q)
        mx, my, _ = slab.sampled_modes()
        omx, omy = lattice.sample_modes(50, 9, call, sl.alpha, 30.0, 30.0)
        assert (mx == omx).all() and (my == omy).all()
        draws.append((mx.copy(), my.copy()))
    assert slab.rng_state() == (9, 3)
    slab.set_rng_state(9, 1)
    slab.compute(pos, q)
    mx, my, _ = slab.sampled_modes()
    assert (mx == draws[1][0]).all() and (my == draws[1][1]).all()
    slab.close()


def test_fp32c_full_k(qslab, soe16):
    sl = workloads.uniform_slab(20_000, (60.0, 60.0, 12.0), 5, alpha=0.25)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    got = _run(qslab, sl, "fp32c", soe16, kc=kc)
    ref = soe_ewald2d.soe_full(got["pos"], got["q"], sl.box, sl.alpha, *soe16, kc=kc)
    _check_fp32(got, ref)


def test_fp32c_full_k_workload(qslab, soe16):
    """The N = 1e5 compensated-FP32 workload (full k-sum, 1836 half-plane
    modes) at its full size: energy to 1e-6 of |E|, phi and F RMS to 1e-5."""
    sl = workloads.fp32_full()
    kc = lattice.kcut_for_tail(sl.alpha, sl.tail)
    got = _run(qslab, sl, "fp32c", soe16, kc=kc)
    ref = soe_ewald2d.soe_full(got["pos"], got["q"], sl.box, sl.alpha, *soe16, kc=kc)
    _check_fp32(got, ref)


def test_rbe_large_fp32c_and_fp64(qslab, soe16):
    """The N = 1e6 random-batch workload at full size, both precisions, on the
    same seeded sample as the oracle, in the launch configuration the
    benchmark times. Energy errors relative to |E_full-k| (golden file)."""
    from golden_check import fingerprint_matches
    sl = workloads.rbe_large()
    gold = _golden("rbe_large_fullk.json")
    got32 = _run(qslab, sl, "fp32c", soe16, rbe=(200, 11))
    assert fingerprint_matches(gold, got32["pos"], got32["q"])
    escale = abs(gold["E_fullk"])
    mx, my, _ = got32["modes"]
    ref32 = soe_ewald2d.soe_rbe(got32["pos"], got32["q"], sl.box, sl.alpha, *soe16, mx, my)
    _check_fp32(got32, ref32, escale=escale)
    got64 = _run(qslab, sl, "fp64", soe16, rbe=(200, 11))
    assert (got64["modes"][0] == mx).all() and (got64["modes"][1] == my).all()
    ref64 = soe_ewald2d.soe_rbe(sl.pos, sl.q, sl.box, sl.alpha, *soe16, mx, my)
    _check_fp64(got64, ref64, escale=escale)


def test_confined_slab_m24(qslab):
    """Strongly confined slab: wall-layered z, Gaussian charges, M = 24,
    full k-sum (reduced N so the oracle stays fast)."""
    from paper_2403_01521_gb300.soe import load_soe
    soe = load_soe(24)
    sl = workloads.confined(n=20_000)
    sl.box = (63.2455532, 63.2455532, 2.0)    # same density as 2e5 in 200 x 200
    sl.pos[:, :2] *= 63.2455532 / 200.0
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    ref = soe_ewald2d.soe_full(sl.pos, sl.q, sl.box, sl.alpha, *soe, kc=kc)
    _check_fp64(_run(qslab, sl, "fp64", soe, kc=kc), ref)
    got = _run(qslab, sl, "fp32c", soe, kc=kc)
    ref32 = soe_ewald2d.soe_full(got["pos"], got["q"], sl.box, sl.alpha, *soe, kc=kc)
    # this energy (~292) is a small remainder of its three parts (k != 0
    # pairs, k = 0 pairs, j = i constants, each of order 1e3): the FP32 path's
    # energy is held to 1e-6 of the magnitude of the parts it is summed from
    _check_fp32(got, ref32, escale=sum(abs(v) for v in ref32["E_parts"]))


def test_deterministic(qslab, soe16):
    """Two runs give bitwise-identical outputs (fixed reduction order)."""
    sl = workloads.uniform_slab(5000, (40.0, 40.0, 10.0), 8, alpha=0.3)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    a = _run(qslab, sl, "fp32c", soe16, kc=kc)
    b = _run(qslab, sl, "fp32c", soe16, kc=kc)
    assert a["E"] == b["E"]
    assert (a["phi"] == b["phi"]).all() and (a["F"] == b["F"]).all()


def test_host_buffers_match_device(qslab, soe16):
    sl = workloads.uniform_slab(3000, (30.0, 30.0, 10.0), 12, alpha=0.3)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, kcut=kc)
    e, phi, F = slab.compute(torch.tensor(sl.pos, device="cuda"), torch.tensor(sl.q, device="cuda"))
    e2, phi2, F2 = slab.compute_host(sl.pos, sl.q)
    assert float(e.item()) == e2
    assert (phi.cpu().numpy() == phi2).all() and (F.cpu().numpy() == F2).all()
    slab.close()


def test_input_errors(qslab, soe16):
    box = (10.0, 10.0, 5.0)
    kc = lattice.kcut_for_tail(0.5, 1e-8)
    slab = qslab.QSlab(0, "fp64").configure(box, 0.5, soe16, kcut=kc)
    good = np.array([[1.0, 1.0, 1.0], [2.0, 2.0, 2.0]])
    qn = np.array([1.0, -1.0])

    def status(pos, q):
        slab.compute(torch.tensor(pos, device="cuda"), torch.tensor(q, device="cuda"))
        return slab.status()

    assert status(good, qn) == 0
    bad = good.copy(); bad[1, 2] = 5.5
    assert status(bad, qn) == -4
    bad = good.copy(); bad[0, 2] = -0.1
    assert status(bad, qn) == -4
    bad = good.copy(); bad[0, 0] = np.nan
    assert status(bad, qn) == -3
    assert status(good, np.array([1.0, -0.5])) == -5
    assert status(good, qn) == 0             # the status word is cleared by reading it
    with pytest.raises(qslab.QslabError):
        qslab.qslab_set_alpha(slab.h, -1.0)
    with pytest.raises(qslab.QslabError):     # not conjugate-closed
        qslab.qslab_set_soe(slab.h, np.array([1 + 1j]), np.array([1 + 0j]))
    slab.close()
    unconf = qslab.QSlab(0, "fp64")
    with pytest.raises(qslab.QslabError):
        unconf.compute(torch.tensor(good, device="cuda"), torch.tensor(qn, device="cuda"))
    unconf.close()


def test_autograd_adjoint(qslab, soe16):
    """SlabEnergy backward: dE/dpos = -F and dE/dq = phi, checked by FP64
    central differences (h = 1e-4) at a few particles."""
    sl = workloads.uniform_slab(400, (20.0, 20.0, 2.0), 15, alpha=0.35)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, kcut=kc)
    pos = torch.tensor(sl.pos, device="cuda", requires_grad=True)
    q = torch.tensor(sl.q, device="cuda", requires_grad=True)
    E = qslab.slab_energy(pos, q, slab)
    E.backward()
    gpos = pos.grad.cpu().numpy()
    gq = q.grad.cpu().numpy()
    h = 1e-4
    for i in (0, 57, 311):
        for c in range(3):
            p1 = sl.pos.copy(); p1[i, c] += h
            p2 = sl.pos.copy(); p2[i, c] -= h
            e1 = slab.compute(torch.tensor(p1, device="cuda"), q.detach())[0].item()
            e2 = slab.compute(torch.tensor(p2, device="cuda"), q.detach())[0].item()
            assert abs((e1 - e2) / (2 * h) - gpos[i, c]) <= 1e-6 * max(1.0, abs(gpos[i, c]))
        q1 = sl.q.copy(); q1[i] += h
        q2 = sl.q.copy(); q2[i] -= h
        qslab.qslab_set_neutrality_tol(slab.h, -1.0)
        e1 = slab.compute(pos.detach(), torch.tensor(q1, device="cuda"))[0].item()
        e2 = slab.compute(pos.detach(), torch.tensor(q2, device="cuda"))[0].item()
        assert abs((e1 - e2) / (2 * h) - gq[i]) <= 1e-6 * max(1.0, abs(gq[i]))
    slab.close()


def test_net_force_and_fp32_invariance(qslab, soe16):
    """Sum of forces vanishes (Newton) and a common x,y shift leaves E unchanged."""
    sl = workloads.uniform_slab(10_000, (50.0, 50.0, 10.0), 21, alpha=0.3)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    a = _run(qslab, sl, "fp64", soe16, kc=kc)
    assert np.abs(a["F"].sum(0)).max() <= 1e-10 * np.abs(a["F"]).sum()
    sh = workloads.Slab("s", sl.pos.copy(), sl.q, sl.box, sl.alpha, 16)
    sh.pos[:, 0] = (sh.pos[:, 0] + 17.0) % 50.0
    sh.pos[:, 1] = (sh.pos[:, 1] + 3.5) % 50.0
    b = _run(qslab, sh, "fp64", soe16, kc=kc)
    assert abs(a["E"] - b["E"]) <= 1e-11 * abs(a["E"])


# FP32C launch shapes: automatic; chunk lengths that are not whole k-steps
# of the tensor-core aggregates (37, 100: ragged tails of 5 and 0 or 4
# particles); one warp of modes; a random batch of 200 modes (a warp with
# 8 real modes runs as a remainder warp) in several chunk lengths
@pytest.mark.parametrize("tuning", [(0, 0), (37, 0), (100, 64), (16, 32)])
def test_fp32c_full_k_launch_shapes(qslab, small_full, soe16, tuning):
    sl = small_full
    kc = lattice.kcut_for_tail(sl.alpha, sl.tail)
    got = _run(qslab, sl, "fp32c", soe16, kc=kc, tuning=tuning)
    ref = soe_ewald2d.soe_full(got["pos"], got["q"], sl.box, sl.alpha, *soe16, kc=kc)
    _check_fp32(got, ref)


@pytest.mark.parametrize("chunk", [0, 37, 64, 200])
def test_fp32c_rbe_launch_shapes(qslab, soe16, chunk):
    sl = workloads.uniform_slab(3000, (40.0, 40.0, 15.0), 41, alpha=0.2)
    got = _run(qslab, sl, "fp32c", soe16, rbe=(200, 9), tuning=(chunk, 0))
    mx, my, _ = got["modes"]
    ref = soe_ewald2d.soe_rbe(got["pos"], got["q"], sl.box, sl.alpha, *soe16, mx, my)
    _check_fp32(got, ref, escale=0.5 * float(np.abs(got["q"] * ref["phi"]).sum()))


@pytest.mark.parametrize("M,kind", [(8, "conditioned"), (24, "conditioned"), (16, "accurate")])
def test_fp32c_other_soe_tables(qslab, M, kind):
    """FP32C with the other SOE tables: 4 pair representatives (tensor-core
    aggregates with two n-tiles), 12 (the scalar aggregate kernel) and the
    accurate M = 16 table."""
    from paper_2403_01521_gb300.soe import load_soe
    soe = load_soe(M, kind)
    sl = workloads.uniform_slab(3000, (25.0, 20.0, 9.0), 33, alpha=0.4)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    got = _run(qslab, sl, "fp32c", soe, kc=kc, tuning=(64, 0))
    ref = soe_ewald2d.soe_full(got["pos"], got["q"], sl.box, sl.alpha, *soe, kc=kc)
    _check_fp32(got, ref, escale=sum(abs(x) for x in ref["E_parts"]))


@pytest.mark.parametrize("tuning", [(0, 0), (64, 64), (48, 32)])
def test_fp32c_remainder_warp_mode_ranges(qslab, soe16, tuning):
    """A full k-sum of 295 half-plane modes (295 = 9 * 32 + 7): the warp
    holding the last 7 modes runs as a remainder warp in the last of several
    mode ranges; the warps past K hold padding only."""
    sl = workloads.uniform_slab(2500, (26.0, 24.0, 9.0), 47, alpha=0.4)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    got = _run(qslab, sl, "fp32c", soe16, kc=kc, tuning=tuning)
    ref = soe_ewald2d.soe_full(got["pos"], got["q"], sl.box, sl.alpha, *soe16, kc=kc)
    _check_fp32(got, ref, escale=sum(abs(x) for x in ref["E_parts"]))
