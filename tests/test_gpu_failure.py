"""Failure handling of the library's device allocations, injected on the
host (qslab_debug_fail_alloc: the next n allocations fail as an
out-of-memory cudaMalloc would, without calling the runtime; no GPU fault).

A call whose allocation fails returns QSLAB_ERR_ALLOC and changes no
configuration, random-batch counter or output; the context stays usable and
later calls give the same results as before the failure. One failed attempt
is absorbed (the old buffer is released and the allocation retried), two
fail the call.
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qslab():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01521_gb300 as q
    q.load()
    yield q
    q.qslab_debug_fail_alloc(0)


def _dev(sl):
    return (torch.tensor(sl.pos, device="cuda"), torch.tensor(sl.q, device="cuda"))


def test_failed_allocation_changes_nothing(qslab, soe16):
    box = (40.0, 40.0, 20.0)
    small = workloads.uniform_slab(2000, box, 41, alpha=0.2)
    big = workloads.uniform_slab(40000, box, 42, alpha=0.2)
    slab = qslab.QSlab(0, "fp64").configure(box, 0.2, soe16, rbe=(64, 9))
    p1, q1 = _dev(small)
    e, phi, F = slab.compute(p1, q1)
    assert slab.status() == 0
    E1, phi1, F1 = float(e.item()), phi.cpu().numpy(), F.cpu().numpy()
    assert slab.rng_state() == (9, 1)
    p2, q2 = _dev(big)
    out = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    n0 = qslab.qslab_debug_alloc_count()
    qslab.qslab_debug_fail_alloc(2)           # both attempts of the table buffer fail
    with pytest.raises(qslab.QslabError) as err:
        slab.compute(p2, q2, energy=out)
    assert err.value.code == -6
    qslab.qslab_debug_fail_alloc(0)
    assert qslab.qslab_debug_alloc_count() == n0
    assert float(out.item()) == 7.0           # no output written
    assert slab.rng_state() == (9, 1)         # no sample drawn
    # the same call as before the failure gives the same results, bit for bit
    slab.set_rng_state(9, 0)
    e, phi, F = slab.compute(p1, q1)
    assert slab.status() == 0
    assert float(e.item()) == E1
    assert (phi.cpu().numpy() == phi1).all() and (F.cpu().numpy() == F1).all()
    # and the larger call now runs
    e2, _, _ = slab.compute(p2, q2)
    assert slab.status() == 0 and np.isfinite(e2.item())
    slab.close()


def test_one_failed_attempt_is_absorbed(qslab, soe16):
    box = (30.0, 30.0, 10.0)
    a = workloads.uniform_slab(1000, box, 43, alpha=0.3)
    b = workloads.uniform_slab(20000, box, 44, alpha=0.3)
    kc = qslab.kcut_for_tail(0.3, 1e-8)
    ref = qslab.QSlab(0, "fp64").configure(box, 0.3, soe16, kcut=kc)
    pb, qb = _dev(b)
    Eref = float(ref.compute(pb, qb)[0].item())
    ref.close()
    slab = qslab.QSlab(0, "fp64").configure(box, 0.3, soe16, kcut=kc)
    pa, qa = _dev(a)
    slab.compute(pa, qa)
    n0 = qslab.qslab_debug_alloc_count()
    qslab.qslab_debug_fail_alloc(1)
    E = float(slab.compute(pb, qb)[0].item())   # first attempt fails, the retry succeeds
    assert slab.status() == 0
    assert E == Eref
    assert qslab.qslab_debug_alloc_count() > n0
    slab.close()


def test_failed_workspace_growth(qslab, soe16):
    """Tables fit, the larger workspace of the virial call does not: the call
    fails, and the plain call and then the virial call still work."""
    box = (30.0, 30.0, 10.0)
    sl = workloads.uniform_slab(3000, box, 45, alpha=0.3)
    kc = qslab.kcut_for_tail(0.3, 1e-8)
    slab = qslab.QSlab(0, "fp64").configure(box, 0.3, soe16, kcut=kc)
    p, q = _dev(sl)
    E0 = float(slab.compute(p, q)[0].item())
    qslab.qslab_debug_fail_alloc(2)
    with pytest.raises(qslab.QslabError) as err:
        slab.compute_virial(p, q)
    qslab.qslab_debug_fail_alloc(0)
    assert err.value.code == -6
    assert float(slab.compute(p, q)[0].item()) == E0
    e, _, _, W = slab.compute_virial(p, q)
    assert slab.status() == 0 and float(e.item()) == E0
    slab.close()


def test_failed_create(qslab):
    qslab.qslab_debug_fail_alloc(1)
    with pytest.raises(qslab.QslabError) as err:
        qslab.qslab_create(0, qslab.QSLAB_FP64)
    qslab.qslab_debug_fail_alloc(0)
    assert err.value.code == -6
    h = qslab.qslab_create(0, qslab.QSLAB_FP64)
    qslab.qslab_destroy(h)


def test_bounded_wait_times_out(qslab, soe16):
    """The z-sort's look-back between CTAs waits a bounded time: with one
    tile made to publish nothing (a host-side test hook), the next tile's
    wait runs out, the call reports QSLAB_ERR_TIMEOUT (no GPU fault, no
    hang), and the context stays usable: the same call again gives the
    first result bit for bit."""
    box = (40.0, 40.0, 20.0)
    sl = workloads.uniform_slab(20000, box, 46, alpha=0.25)     # 5 sort tiles of 4096
    slab = qslab.QSlab(0, "fp32c").configure(box, 0.25, soe16, rbe=(64, 3))
    p = torch.tensor(sl.pos, device="cuda", dtype=torch.float32)
    q = torch.tensor(sl.q, device="cuda", dtype=torch.float32)
    e, phi, F = slab.compute(p, q)
    assert slab.status() == 0
    E0, phi0 = float(e.item()), phi.cpu().numpy()
    slab.set_rng_state(3, 0)
    qslab.qslab_debug_stall_sort(2)
    slab.compute(p, q)
    assert slab.status() == -8
    slab.set_rng_state(3, 0)
    e, phi, F = slab.compute(p, q)
    assert slab.status() == 0
    assert float(e.item()) == E0 and (phi.cpu().numpy() == phi0).all()
    slab.close()
