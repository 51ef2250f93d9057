"""qslab_compute_static: the entry point for callers that cannot allocate
device memory when they need the forces (for example inside another
framework's memory pool or under a fixed memory budget). It takes all its
scratch from the library's fixed device array instead of allocating, and must
give the same results as qslab_compute() on the same inputs, call after call,
and the oracle's, while the library's count of device allocations stays
unchanged across the call.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import workloads
from oracle import lattice, soe_ewald2d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10          # the parity tolerances of the other GPU tests
FP32_RMS_TOL = 1e-5


@pytest.fixture(scope="module")
def qslab():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01521_gb300 as q
    q.load()
    return q


def _both(qslab, slab, pos, q):
    """Results of qslab_compute and of qslab_compute_static on the same inputs."""
    N = q.shape[0]
    e1, phi1, F1 = slab.compute(pos, q)
    assert slab.status() == 0
    e2 = torch.empty(1, dtype=torch.float64, device="cuda")
    phi2 = torch.empty_like(phi1)
    F2 = torch.empty_like(F1)
    stream = torch.cuda.current_stream().cuda_stream
    n0 = qslab.qslab_debug_alloc_count()
    qslab.qslab_compute_static(slab.h, N, pos.data_ptr(), q.data_ptr(), e2.data_ptr(),
                               phi2.data_ptr(), F2.data_ptr(), stream)
    assert qslab.qslab_debug_alloc_count() == n0     # no device allocation
    return ([float(e1.item()), phi1.double().cpu().numpy(), F1.double().cpu().numpy()],
            [float(e2.item()), phi2.double().cpu().numpy(), F2.double().cpu().numpy()])


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_static_matches_compute_twice(qslab, soe16, prec):
    sl = workloads.uniform_slab(5000, (40.0, 40.0, 12.0), 17, alpha=0.3)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    slab = qslab.QSlab(0, prec).configure(sl.box, sl.alpha, soe16, kcut=kc)
    dt = torch.float64 if prec == "fp64" else torch.float32
    pos = torch.tensor(sl.pos, device="cuda", dtype=dt)
    q = torch.tensor(sl.q, device="cuda", dtype=dt)
    orc = soe_ewald2d.soe_full(pos.double().cpu().numpy(), q.double().cpu().numpy(), sl.box,
                               sl.alpha, *soe16, kc=kc)
    oracle = [orc["E"], orc["phi"], orc["F"]]
    for _ in range(2):                       # two calls in a row
        ref, got = _both(qslab, slab, pos, q)
        if prec == "fp64":
            assert abs(got[0] - oracle[0]) <= FP64_TOL * abs(oracle[0])
            for a, b in zip(got[1:], oracle[1:]):
                assert np.abs(a - b).max() <= FP64_TOL * np.abs(b).max()
        else:
            assert abs(got[0] - oracle[0]) <= 1e-6 * abs(oracle[0])
            for a, b in zip(got[1:], oracle[1:]):
                assert np.sqrt(((a - b) ** 2).mean()) <= FP32_RMS_TOL * np.sqrt((b ** 2).mean())
        if prec == "fp64":
            assert abs(got[0] - ref[0]) <= FP64_TOL * abs(ref[0])
            for a, b in zip(got[1:], ref[1:]):
                assert np.abs(a - b).max() <= FP64_TOL * np.abs(b).max()
        else:
            assert abs(got[0] - ref[0]) <= 1e-6 * abs(ref[0])
            for a, b in zip(got[1:], ref[1:]):
                assert np.sqrt(((a - b) ** 2).mean()) <= FP32_RMS_TOL * np.sqrt((b ** 2).mean())
    slab.close()


def test_static_random_batch_twice(qslab, soe16):
    """Random batch: the same seed and counter give the same sample on both
    entry points, and each call advances the counter."""
    sl = workloads.uniform_slab(4000, (40.0, 40.0, 20.0), 23, alpha=0.2)
    a = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, rbe=(64, 5))
    b = qslab.QSlab(0, "fp64").configure(sl.box, sl.alpha, soe16, rbe=(64, 5))
    pos = torch.tensor(sl.pos, device="cuda")
    q = torch.tensor(sl.q, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        e1, phi1, F1 = a.compute(pos, q)
        e2 = torch.empty(1, dtype=torch.float64, device="cuda")
        phi2 = torch.empty_like(phi1)
        F2 = torch.empty_like(F1)
        qslab.qslab_compute_static(b.h, sl.N, pos.data_ptr(), q.data_ptr(), e2.data_ptr(),
                                   phi2.data_ptr(), F2.data_ptr(), stream)
        assert b.rng_state() == (5, call + 1)
        assert abs(e2.item() - e1.item()) <= FP64_TOL * abs(e1.item())
        assert (torch.abs(F2 - F1).max() <= FP64_TOL * torch.abs(F1).max()).item()
    a.close()
    b.close()


def test_static_rejects_too_large(qslab, soe16):
    sl = workloads.uniform_slab(400_000, (200.0, 200.0, 50.0), 29, alpha=0.1)
    slab = qslab.QSlab(0, "fp32c").configure(sl.box, sl.alpha, soe16, rbe=(200, 1))
    pos = torch.tensor(sl.pos, device="cuda", dtype=torch.float32)
    q = torch.tensor(sl.q, device="cuda", dtype=torch.float32)
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(qslab.QslabError) as err:
        qslab.qslab_compute_static(slab.h, sl.N, pos.data_ptr(), q.data_ptr(), e.data_ptr(),
                                   None, None, torch.cuda.current_stream().cuda_stream)
    assert err.value.code == -9
    slab.close()


def test_static_two_contexts_on_a_side_stream(qslab, soe16):
    """Two contexts of different size and configuration take turns on the
    static entry from a non-default stream; every call matches qslab_compute
    on the same inputs (the array keeps the previous call's contents, and each
    call's tables are uploaded in its stream's order)."""
    s1 = workloads.uniform_slab(3000, (30.0, 30.0, 10.0), 31, alpha=0.3)
    s2 = workloads.uniform_slab(7000, (50.0, 40.0, 15.0), 32, alpha=0.25)
    k1 = lattice.kcut_for_tail(s1.alpha, 1e-8)
    a1 = qslab.QSlab(0, "fp64").configure(s1.box, s1.alpha, soe16, kcut=k1)
    # random batch: twin contexts (same seed) so that both entries draw the same sample
    a2 = qslab.QSlab(0, "fp32c").configure(s2.box, s2.alpha, soe16, rbe=(96, 3))
    b2 = qslab.QSlab(0, "fp32c").configure(s2.box, s2.alpha, soe16, rbe=(96, 3))
    p1 = torch.tensor(s1.pos, device="cuda")
    q1 = torch.tensor(s1.q, device="cuda")
    p2 = torch.tensor(s2.pos, device="cuda", dtype=torch.float32)
    q2 = torch.tensor(s2.q, device="cuda", dtype=torch.float32)
    side = torch.cuda.Stream()
    for _ in range(2):
        for slab, twin, p, q, tol in [(a1, a1, p1, q1, FP64_TOL), (b2, a2, p2, q2, 1e-6)]:
            e_ref, phi_ref, F_ref = twin.compute(p, q)
            assert twin.status() == 0
            torch.cuda.synchronize()
            e = torch.empty(1, dtype=torch.float64, device="cuda")
            phi = torch.empty_like(phi_ref)
            F = torch.empty_like(F_ref)
            with torch.cuda.stream(side):
                n0 = qslab.qslab_debug_alloc_count()
                qslab.qslab_compute_static(slab.h, q.shape[0], p.data_ptr(), q.data_ptr(),
                                           e.data_ptr(), phi.data_ptr(), F.data_ptr(),
                                           side.cuda_stream)
                assert qslab.qslab_debug_alloc_count() == n0
            side.synchronize()
            assert abs(e.item() - e_ref.item()) <= tol * abs(e_ref.item())
            assert (torch.abs(F - F_ref).max() <= 1e-5 * torch.abs(F_ref).max()).item()
            assert (torch.abs(phi - phi_ref).max() <= 1e-5 * torch.abs(phi_ref).max()).item()
    for s_ in (a1, a2, b2):
        s_.close()
