"""GPU parity of the batched entry point, qslab_compute_batched: many
independent slabs of uneven size and box in one call.

Each replica is compared with the FP64 oracle run on that replica alone
(full k-sum, and the random batch on the replica's own sample, drawn with
the replica index as the generator's stream), with single-slab calls of the
same library (bit-identical for a fixed launch shape: the chunking restarts
at every replica), across a CUDA-graph capture and its replays, and on the
512-replica workload (sampled replicas against the oracle; net force and
energy properties for all of them). Tolerances as in test_gpu_parity.py.
"""
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


def _empty(box):
    return workloads.Slab("empty", np.zeros((0, 3)), np.zeros(0), box, 0.3, 16)


def _stack(slabs):
    """Concatenated inputs: offsets (R+1), boxes (R x 3), pos, q."""
    sizes = [s.pos.shape[0] for s in slabs]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    boxes = np.array([s.box for s in slabs], float)
    pos = np.concatenate([s.pos for s in slabs])
    q = np.concatenate([s.q for s in slabs])
    return off, boxes, pos, q


@pytest.fixture(scope="module")
def mixed():
    """Five replicas: uneven N (one empty, one of 64, ragged tails against
    every chunk length used below), different boxes and densities."""
    alpha = 0.3
    return [
        workloads.uniform_slab(300, (20.0, 24.0, 8.0), 101, alpha=alpha),
        _empty((10.0, 10.0, 5.0)),
        workloads.uniform_slab(1000, (30.0, 30.0, 10.0), 102, alpha=alpha),
        workloads.uniform_slab(64, (12.0, 15.0, 3.0), 103, alpha=alpha),
        workloads.uniform_slab(2050, (36.0, 30.0, 14.0), 104, alpha=alpha),
    ]


def _run_batched(qslab, slabs, prec, soe, kc=None, rbe=None, tuning=(0, 0)):
    off, boxes, pos, q = _stack(slabs)
    slab = qslab.QSlab(0, prec).configure(slabs[0].box, slabs[0].alpha, soe, kcut=kc, rbe=rbe)
    slab.tuning(*tuning)
    dt = torch.float64 if prec == "fp64" else torch.float32
    tpos = torch.tensor(pos, device="cuda", dtype=dt)
    tq = torch.tensor(q, device="cuda", dtype=dt)
    e, phi, F = slab.compute_batched(tpos, tq, off, boxes)
    out = {"E": e.cpu().numpy(), "phi": phi.double().cpu().numpy(),
           "F": F.double().cpu().numpy(), "status": slab.status(), "off": off,
           "pos": tpos.double().cpu().numpy(), "q": tq.double().cpu().numpy()}
    if rbe is not None:
        out["modes"] = slab.sampled_modes()
    slab.close()
    return out


@pytest.mark.parametrize("tuning", [(0, 0), (64, 64), (96, 32)])
def test_batched_fp64_full_k(qslab, mixed, soe16, tuning):
    kc = lattice.kcut_for_tail(0.3, 1e-8)
    got = _run_batched(qslab, mixed, "fp64", soe16, kc=kc, tuning=tuning)
    assert got["status"] == 0
    off = got["off"]
    for r, sl in enumerate(mixed):
        a, b = off[r], off[r + 1]
        if a == b:
            assert got["E"][r] == 0.0
            continue
        ref = soe_ewald2d.soe_full(sl.pos, sl.q, sl.box, sl.alpha, *soe16, kc=kc)
        assert abs(got["E"][r] - ref["E"]) <= FP64_TOL * abs(ref["E"]), r
        assert _maxrel(got["phi"][a:b], ref["phi"]) <= FP64_TOL, r
        assert _maxrel(got["F"][a:b], ref["F"]) <= FP64_TOL, r


def test_batched_fp64_rbe(qslab, mixed, soe16):
    """Every replica draws its own P modes from its own h(k) (stream r of the
    counter-based generator) and matches the oracle on that sample."""
    P, seed = 120, 77
    got = _run_batched(qslab, mixed, "fp64", soe16, rbe=(P, seed), tuning=(64, 0))
    assert got["status"] == 0
    mx, my, wts = got["modes"]
    off = got["off"]
    for r, sl in enumerate(mixed):
        Lx, Ly, _ = sl.box
        omx, omy = lattice.sample_modes(P, seed, 0, 0.3, Lx, Ly, stream=r)
        assert (mx[r] == omx).all() and (my[r] == omy).all(), r
        assert abs(wts[r] - lattice.H_direct(0.3, Lx, Ly) / P) <= 1e-12 * wts[r]
        a, b = off[r], off[r + 1]
        if a == b:
            continue
        ref = soe_ewald2d.soe_rbe(sl.pos, sl.q, sl.box, 0.3, *soe16, omx, omy)
        assert abs(got["E"][r] - ref["E"]) <= FP64_TOL * 0.5 * float(np.abs(sl.q * ref["phi"]).sum())
        assert _maxrel(got["phi"][a:b], ref["phi"]) <= FP64_TOL, r
        assert _maxrel(got["F"][a:b], ref["F"]) <= FP64_TOL, r


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_batched_equals_single(qslab, mixed, soe16, prec):
    """With a fixed launch shape the batched call gives each replica exactly
    (bit for bit) what a single-slab call on that replica gives."""
    kc = lattice.kcut_for_tail(0.3, 1e-8)
    tuning = (64, 64)
    got = _run_batched(qslab, mixed, prec, soe16, kc=kc, tuning=tuning)
    dt = torch.float64 if prec == "fp64" else torch.float32
    off = got["off"]
    for r, sl in enumerate(mixed):
        a, b = off[r], off[r + 1]
        if a == b:
            continue
        one = qslab.QSlab(0, prec).configure(sl.box, sl.alpha, soe16, kcut=kc).tuning(*tuning)
        e, phi, F = one.compute(torch.tensor(sl.pos, device="cuda", dtype=dt),
                                torch.tensor(sl.q, device="cuda", dtype=dt))
        assert one.status() == 0
        assert float(e.item()) == got["E"][r], r
        assert np.array_equal(phi.double().cpu().numpy(), got["phi"][a:b]), r
        assert np.array_equal(F.double().cpu().numpy(), got["F"][a:b]), r
        one.close()


def test_batched_all_short_chains(qslab, soe16):
    """Every slab's carry chains shorter than 32 chunks: each is one group,
    replayed from zero, and the group and chain phases are not launched at
    all. Each replica against the oracle, and bit for bit against its own
    single-slab call with the same launch shape."""
    slabs = [workloads.uniform_slab(100, (14.0, 16.0, 5.0), 111, alpha=0.3),
             _empty((10.0, 10.0, 5.0)),
             workloads.uniform_slab(250, (20.0, 18.0, 6.0), 112, alpha=0.3),
             workloads.uniform_slab(400, (22.0, 22.0, 8.0), 113, alpha=0.3)]
    kc = lattice.kcut_for_tail(0.3, 1e-8)
    tuning = (16, 64)            # 7, 16 and 25 chunks of 16 particles
    got = _run_batched(qslab, slabs, "fp64", soe16, kc=kc, tuning=tuning)
    assert got["status"] == 0
    off = got["off"]
    for r, sl in enumerate(slabs):
        a, b = off[r], off[r + 1]
        if a == b:
            assert got["E"][r] == 0.0
            continue
        ref = soe_ewald2d.soe_full(sl.pos, sl.q, sl.box, sl.alpha, *soe16, kc=kc)
        # energy scale: one slab's E is a small remainder (0.47 against
        # sum |q phi| / 2 = 213)
        escale = max(abs(ref["E"]), 0.5 * float(np.abs(sl.q * ref["phi"]).sum()))
        assert abs(got["E"][r] - ref["E"]) <= FP64_TOL * escale, r
        assert _maxrel(got["phi"][a:b], ref["phi"]) <= FP64_TOL, r
        assert _maxrel(got["F"][a:b], ref["F"]) <= FP64_TOL, r
        one = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, kcut=kc).tuning(*tuning)
        e, phi, F = one.compute(torch.tensor(sl.pos, device="cuda", dtype=torch.float64),
                                torch.tensor(sl.q, device="cuda", dtype=torch.float64))
        assert one.status() == 0
        assert float(e.item()) == got["E"][r], r
        assert np.array_equal(phi.cpu().numpy(), got["phi"][a:b]), r
        assert np.array_equal(F.cpu().numpy(), got["F"][a:b]), r
        one.close()


def test_batched_graph_replay(qslab, mixed, soe16):
    """A CUDA graph of the batched call: every replay draws a fresh sample
    (device-side counter) and equals a plain call made with that counter."""
    P, seed = 64, 5
    off, boxes, pos, q = _stack(mixed)
    slab = qslab.QSlab(0, "fp32c").configure(mixed[0].box, 0.3, soe16, rbe=(P, seed))
    tpos = torch.tensor(pos, device="cuda", dtype=torch.float32)
    tq = torch.tensor(q, device="cuda", dtype=torch.float32)
    g = qslab.GraphedBatch(slab, tpos, tq, off, boxes)          # one warm-up call: counter 1
    assert slab.status() == 0
    assert slab.rng_state() == (seed, 1)
    outs = []
    for _ in range(3):
        e, phi, F = g.replay()                                  # counters 1, 2, 3
        torch.cuda.synchronize()
        outs.append((e.cpu().numpy().copy(), phi.cpu().numpy().copy(), F.cpu().numpy().copy()))
    assert slab.status() == 0
    assert slab.rng_state() == (seed, 4)
    assert not np.array_equal(outs[0][0], outs[1][0])          # fresh samples
    slab.set_rng_state(seed, 3)
    e, phi, F = slab.compute_batched(tpos, tq, off, boxes)
    assert np.array_equal(e.cpu().numpy(), outs[2][0])
    assert np.array_equal(phi.cpu().numpy(), outs[2][1])
    assert np.array_equal(F.cpu().numpy(), outs[2][2])
    mx, my, _ = slab.sampled_modes()
    for r, sl in enumerate(mixed):
        omx, omy = lattice.sample_modes(P, seed, 3, 0.3, sl.box[0], sl.box[1], stream=r)
        assert (mx[r] == omx).all() and (my[r] == omy).all()
    slab.close()


def test_batched_input_errors(qslab, mixed, soe16):
    off, boxes, pos, q = _stack(mixed)
    slab = qslab.QSlab(0, "fp64").configure(mixed[0].box, 0.3, soe16,
                                              kcut=lattice.kcut_for_tail(0.3, 1e-8))
    tpos = torch.tensor(pos, device="cuda")
    tq = torch.tensor(q, device="cuda")
    nonmono = off.copy()
    nonmono[2] = nonmono[3] + 1
    for bad in (off + 1, nonmono, np.array([0], np.int64)):
        R = len(bad) - 1
        bx = np.ones((max(R, 1), 3)) if R != len(boxes) else boxes
        with pytest.raises(qslab.QslabError) as ei:
            qslab.qslab_compute_batched(slab.h, bad, bx[:max(R, 0)] if R > 0 else bx[:0],
                                        tpos.data_ptr(), tq.data_ptr(), None, None, None, None)
        assert ei.value.code == -1
    bad_box = boxes.copy()
    bad_box[2, 0] = -1.0
    with pytest.raises(qslab.QslabError):
        slab.compute_batched(tpos, tq, off, bad_box)
    # each replica must be neutral on its own (the total here is neutral)
    q2 = q.copy()
    q2[off[0]] += 1.0
    q2[off[2]] -= 1.0
    slab.compute_batched(tpos, torch.tensor(q2, device="cuda"), off, boxes)
    rc = slab.status()
    assert rc == -5, rc
    # z outside the replica's own [0, Lz] (inside another replica's)
    p2 = pos.copy()
    p2[off[3], 2] = mixed[3].box[2] + 1.0
    slab.compute_batched(torch.tensor(p2, device="cuda"), tq, off, boxes)
    assert slab.status() == -4
    slab.close()


@pytest.fixture(scope="module")
def replicas512():
    return workloads.replicas()


def test_replicas_workload_fp32c(qslab, replicas512, soe16):
    """The 512-replica random-batch workload (N uniform in [500, 50000],
    number density 0.05, Lz uniform in [5, 40], P = 200, M = 16, alpha =
    0.25) in one FP32C call: three replicas (smallest, median, largest)
    against the FP64 oracle on the same sample and FP32-rounded inputs; the
    net force and the energy identity for all 512."""
    slabs = replicas512
    P, seed = 200, 2024
    got = _run_batched(qslab, slabs, "fp32c", soe16, rbe=(P, seed))
    assert got["status"] == 0
    off = got["off"]
    mx, my, _ = got["modes"]
    sizes = np.diff(off)
    order = np.argsort(sizes)
    for r in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        a, b = off[r], off[r + 1]
        sl = slabs[r]
        omx, omy = lattice.sample_modes(P, seed, 0, 0.25, sl.box[0], sl.box[1], stream=r)
        assert (mx[r] == omx).all() and (my[r] == omy).all()
        ref = soe_ewald2d.soe_rbe(got["pos"][a:b], got["q"][a:b], sl.box, 0.25, *soe16, omx, omy)
        scale = 0.5 * float(np.abs(got["q"][a:b] * ref["phi"]).sum())
        assert abs(got["E"][r] - ref["E"]) <= FP32_E_TOL * scale, r
        assert _rmsrel(got["phi"][a:b], ref["phi"]) <= FP32_RMS_TOL, r
        assert _rmsrel(got["F"][a:b], ref["F"]) <= FP32_RMS_TOL, r
    for r in range(len(slabs)):
        a, b = off[r], off[r + 1]
        F = got["F"][a:b]
        assert np.abs(F.sum(axis=0)).max() <= 1e-5 * np.abs(F).sum(), r
        e_phi = 0.5 * float(got["q"][a:b] @ got["phi"][a:b])
        scale = 0.5 * float(np.abs(got["q"][a:b] * got["phi"][a:b]).sum())
        assert abs(got["E"][r] - e_phi) <= 1e-6 * scale, r


def test_autotune(qslab, mixed, soe16):
    """The autotuner picks a valid launch shape, keeps the random-batch
    counter, and the tuned call equals a call with that shape set by hand."""
    off, boxes, pos, q = _stack(mixed)
    slab = qslab.QSlab(0, "fp32c").configure(mixed[0].box, 0.3, soe16, rbe=(64, 11))
    tpos = torch.tensor(pos, device="cuda", dtype=torch.float32)
    tq = torch.tensor(q, device="cuda", dtype=torch.float32)
    L, kr = slab.autotune(tpos, tq, off, boxes, reps=2)
    assert L in (64, 128, 256, 512) and kr in (0, 64, 128, 192, 256)
    assert slab.rng_state() == (11, 0)
    e1, phi1, F1 = slab.compute_batched(tpos, tq, off, boxes)
    other = qslab.QSlab(0, "fp32c").configure(mixed[0].box, 0.3, soe16, rbe=(64, 11)).tuning(L, kr)
    e2, phi2, F2 = other.compute_batched(tpos, tq, off, boxes)
    assert slab.status() == 0 and other.status() == 0
    assert torch.equal(e1, e2) and torch.equal(phi1, phi2) and torch.equal(F1, F2)
    other.close()
    slab.close()
