"""GPU parity of the Metropolis k-sampler (App. G): the device chain keeps
exactly the oracle's states (integer, bit-exact), for single slabs, every
slab of a batch, several calls and downsampling rates, and the random-batch
estimator on those samples matches the oracle."""
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


def _maxrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("thin", [1, 3])
def test_metropolis_samples_equal_oracle(qslab, soe16, thin):
    sl = workloads.uniform_slab(2000, (40.0, 30.0, 20.0), 77, alpha=0.2)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, rbe=(200, 4242))
    slab.sampler("metropolis", thin)
    pos = torch.tensor(sl.pos, device="cuda")
    q = torch.tensor(sl.q, device="cuda")
    for call in range(3):
        e, phi, F = slab.compute(pos, q)
        assert slab.status() == 0
        mx, my, weight = slab.sampled_modes()
        omx, omy = lattice.metropolis_modes(200, 4242, call, sl.alpha, 40.0, 30.0, thin=thin)
        assert (mx == omx).all() and (my == omy).all()
        assert abs(weight - lattice.H_direct(sl.alpha, 40.0, 30.0) / 200) <= 1e-12 * weight
    ref = soe_ewald2d.soe_rbe(sl.pos, sl.q, sl.box, sl.alpha, *soe16, omx, omy)
    escale = abs(soe_ewald2d.soe_full(sl.pos, sl.q, sl.box, sl.alpha, *soe16)["E"])
    assert abs(float(e.item()) - ref["E"]) <= 1e-10 * escale
    assert _maxrel(phi.cpu().numpy(), ref["phi"]) <= 1e-10
    assert _maxrel(F.cpu().numpy(), ref["F"]) <= 1e-10
    slab.close()


def test_metropolis_small_box_rejects(qslab, soe16):
    """alpha L = 3: a third of the proposals are rejected and some are the
    origin, so the chain repeats states; still the oracle's chain exactly."""
    sl = workloads.uniform_slab(200, (12.0, 12.0, 6.0), 5, alpha=0.25)
    slab = qslab.QSlab(0, "fp32c").configure(sl.box, sl.alpha, soe16, rbe=(500, 31)).sampler("metropolis", 2)
    pos = torch.tensor(sl.pos, device="cuda", dtype=torch.float32)
    q = torch.tensor(sl.q, device="cuda", dtype=torch.float32)
    slab.compute(pos, q)
    assert slab.status() == 0
    mx, my, _ = slab.sampled_modes()
    omx, omy, rate = lattice.metropolis_modes(500, 31, 0, sl.alpha, 12.0, 12.0, thin=2,
                                              return_rate=True)
    assert rate < 0.8
    assert (mx == omx).all() and (my == omy).all()
    assert (np.diff(mx) == 0).any()
    slab.close()


def test_metropolis_long_chain_many_rejections(qslab, soe16):
    """alpha L = 1.5: most proposals are the origin or rejected, so runs of
    more than 8 rejections occur (the device then decides from the current
    state instead of its precomputed 8-step window), and P thin = 2400
    steps span three rounds of 1024 proposals; still the oracle's chain."""
    sl = workloads.uniform_slab(100, (6.0, 6.0, 4.0), 6, alpha=0.25)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, rbe=(400, 17)).sampler("metropolis", 6)
    pos = torch.tensor(sl.pos, device="cuda")
    q = torch.tensor(sl.q, device="cuda")
    for call in range(2):
        slab.compute(pos, q)
        assert slab.status() == 0
        mx, my, _ = slab.sampled_modes()
        omx, omy, rate = lattice.metropolis_modes(400, 17, call, sl.alpha, 6.0, 6.0, thin=6,
                                                  return_rate=True)
        assert rate < 0.5
        assert (mx == omx).all() and (my == omy).all()
    slab.close()


def test_metropolis_batched_streams(qslab, soe16):
    """Every slab of a batch runs its own chain (stream r); a CUDA-graph
    replay draws the next call's chains."""
    boxes = [(30.0, 30.0, 10.0), (50.0, 20.0, 8.0), (12.0, 40.0, 6.0)]
    slabs = [workloads.uniform_slab(300 + 100 * r, b, 40 + r, alpha=0.3) for r, b in enumerate(boxes)]
    off = np.concatenate([[0], np.cumsum([s.N for s in slabs])]).astype(np.int64)
    P, seed = 80, 17
    slab = qslab.QSlab(0, "fp32c").configure(boxes[0], 0.3, soe16, rbe=(P, seed)).sampler("metropolis", 4)
    pos = torch.tensor(np.concatenate([s.pos for s in slabs]), device="cuda", dtype=torch.float32)
    q = torch.tensor(np.concatenate([s.q for s in slabs]), device="cuda", dtype=torch.float32)
    g = qslab.GraphedBatch(slab, pos, q, off, np.array(boxes))     # warm-up call: counter 0
    mx, my, _ = slab.sampled_modes()
    for r, b in enumerate(boxes):
        omx, omy = lattice.metropolis_modes(P, seed, 0, 0.3, b[0], b[1], stream=r, thin=4)
        assert (mx[r] == omx).all() and (my[r] == omy).all()
    g.replay()
    g.replay()                                                     # counters 1, 2
    torch.cuda.synchronize()
    assert slab.status() == 0
    mx, my, _ = slab.sampled_modes()
    for r, b in enumerate(boxes):
        omx, omy = lattice.metropolis_modes(P, seed, 2, 0.3, b[0], b[1], stream=r, thin=4)
        assert (mx[r] == omx).all() and (my[r] == omy).all()
    slab.close()


def test_sampler_switch_and_errors(qslab, soe16):
    sl = workloads.uniform_slab(400, (20.0, 20.0, 8.0), 9, alpha=0.3)
    slab = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, rbe=(40, 3))
    pos = torch.tensor(sl.pos, device="cuda")
    q = torch.tensor(sl.q, device="cuda")
    slab.sampler("metropolis", 1)
    slab.compute(pos, q)
    a = slab.sampled_modes()
    slab.sampler("iid")
    slab.set_rng_state(3, 0)
    slab.compute(pos, q)
    b = slab.sampled_modes()
    omx, omy = lattice.sample_modes(40, 3, 0, sl.alpha, 20.0, 20.0)
    assert (b[0] == omx).all() and (b[1] == omy).all()
    assert not (a[0] == b[0]).all()
    for kind, thin in [(2, 1), (1, 0), (1, 5000), (-1, 1)]:
        with pytest.raises(qslab.QslabError) as e:
            qslab.qslab_set_rbe_sampler(slab.h, kind, thin)
        assert e.value.code == qslab.QSLAB_ERR_INVALID_ARG
    slab.close()
