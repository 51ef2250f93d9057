"""GPU: the full k-sum at N = 1e6 (400 x 400 x 50, alpha = 0.1, kc at
Gaussian tail 1e-8: 9392 lattice vectors, 4696 half-plane modes, M = 16).

The oracle's energy of this configuration (positions rounded to FP32) and
its potentials and forces at 512 seeded particles are stored in
tests/golden/rbe_large_fullk.json, written by tests/golden/make_golden.py
from the oracle alone (about 10 minutes on 8 cores). Against them: the FP64
path to 1e-10 (energy; max-norm of phi and F over the sample), the FP32 path
to 1e-6 (energy) and 1e-5 (RMS of phi and F over the sample). Every
particle's FP32 phi and F are also checked against the FP64 path's (RMS
relative 1e-5), and both against the zero net force of a neutral slab
without walls.
"""
import json
import os

import numpy as np
import pytest

import workloads
from oracle import lattice

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qslab():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01521_gb300 as q
    q.load()
    return q


def _rmsrel(a, b):
    return float(np.sqrt(((a - b) ** 2).mean()) / np.sqrt((b ** 2).mean()))


def _maxrel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_full_k_1e6(qslab, soe16):
    from golden_check import fingerprint_matches
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "rbe_large_fullk.json")) as fh:
        gold = json.load(fh)
    sl = workloads.rbe_large()
    kc = lattice.kcut_for_tail(sl.alpha, gold["kc_tail"])
    pos32 = torch.tensor(sl.pos, device="cuda", dtype=torch.float32)
    q32 = torch.tensor(sl.q, device="cuda", dtype=torch.float32)
    assert fingerprint_matches(gold, pos32.double().cpu().numpy(), q32.double().cpu().numpy())
    out = {}
    for prec, pos, q in [("fp32c", pos32, q32), ("fp64", pos32.double(), q32.double())]:
        slab = qslab.QSlab(0, prec).configure(sl.box, sl.alpha, soe16, kcut=kc)
        assert slab.num_modes() == gold["modes_full_lattice"] // 2
        e, phi, F = slab.compute(pos, q)
        assert slab.status() == 0
        out[prec] = (float(e.item()), phi.double().cpu().numpy(), F.double().cpu().numpy())
        slab.close()
    E_ref = gold["E_fullk"]
    idx = np.array(gold["sample_idx"])
    phi_ref = np.array(gold["phi"])
    F_ref = np.array(gold["F"])
    assert abs(out["fp64"][0] - E_ref) <= 1e-10 * abs(E_ref)
    assert _maxrel(out["fp64"][1][idx], phi_ref) <= 1e-10
    assert _maxrel(out["fp64"][2][idx], F_ref) <= 1e-10
    assert abs(out["fp32c"][0] - E_ref) <= 1e-6 * abs(E_ref)
    assert _rmsrel(out["fp32c"][1][idx], phi_ref) <= 1e-5
    assert _rmsrel(out["fp32c"][2][idx], F_ref) <= 1e-5
    assert _rmsrel(out["fp32c"][1], out["fp64"][1]) <= 1e-5
    assert _rmsrel(out["fp32c"][2], out["fp64"][2]) <= 1e-5
    for prec in out:
        F = out[prec][2]
        assert np.abs(F.sum(0)).max() <= 1e-8 * np.abs(F).sum()
