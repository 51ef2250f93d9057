"""Write the stored expected values used by the GPU tests.

Every value here is computed by the FP64 oracle (oracle/) from the seeded
workloads (workloads.py); nothing comes from the CUDA library.

  rbe_large_fullk.json   the full-k long-range energy (kc at Gaussian tail
                         1e-8, M = 16 conditioned SOE) of the N = 1e6
                         random-batch workload, i.e. the expectation of its
                         random-batch estimator, its three parts (as for
                         confined_fullk.json), and the potential and force
                         of a seeded sample of 512 particles. The positions
                         are rounded to FP32 first, as the FP32 path sees
                         them. A fingerprint of the inputs is stored beside it.
  confined_fullk.json    the strongly confined N = 2e5 slab (200 x 200 x 2,
                         wall-exponential z, Gaussian charges, alpha = 0.2,
                         M = 24 conditioned SOE, full k-sum at tail 1e-8):
                         energy (and its three parts: k != 0 pairs, k = 0
                         pairs, j = i constants with the self term), and
                         potential and force of a seeded sample of
                         512 particles, once on the FP64 inputs and once on
                         the inputs rounded to FP32 (positions and charges).

Run: python tests/golden/make_golden.py [rbe_large|confined ...]
(about 8 minutes for rbe_large and 5 for confined on 8 cores)
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

SAMPLE = 512          # particles whose potential and force are stored
SAMPLE_SEED = 20240302


def fingerprint(pos, q):
    return [float(np.sum(pos[:, 0])), float(np.sum(pos[:, 2] * q)), int(pos.shape[0])]


def sample_index(n):
    rng = np.random.default_rng(SAMPLE_SEED)
    return np.sort(rng.choice(n, size=SAMPLE, replace=False))


def _values(out, idx):
    return {"sample_idx": [int(i) for i in idx],
            "phi": [float(v) for v in out["phi"][idx]],
            "F": [[float(v) for v in row] for row in out["F"][idx]]}


def rbe_large_fullk():
    import workloads
    from oracle import lattice, soe_ewald2d
    from paper_2403_01521_gb300.soe import load_soe   # SOE table: a method input
    sl = workloads.rbe_large()
    pos = sl.pos.astype(np.float32).astype(np.float64)
    s, w = load_soe(16)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    t = time.time()
    out = soe_ewald2d.soe_full(pos, sl.q, sl.box, sl.alpha, s, w, kc=kc)
    d = {"workload": "rbe_large (seed 3), positions rounded to float32",
         "kc_tail": 1e-8, "M": 16, "soe": "conditioned",
         "E_fullk": out["E"], "E_parts": list(out["E_parts"]),
         "modes_full_lattice": int(len(out["modes"][0])),
         "fingerprint": fingerprint(pos, sl.q), "oracle_seconds": time.time() - t}
    d.update(_values(out, sample_index(sl.N)))
    return d


def confined_fullk():
    import workloads
    from oracle import lattice, soe_ewald2d
    from paper_2403_01521_gb300.soe import load_soe
    sl = workloads.confined()
    s, w = load_soe(24)
    kc = lattice.kcut_for_tail(sl.alpha, 1e-8)
    idx = sample_index(sl.N)
    d = {"workload": "confined (seed 5): N = 2e5 in 200 x 200 x 2, alpha = 0.2",
         "kc_tail": 1e-8, "M": 24, "soe": "conditioned"}
    for name, pos, q in [("fp64", sl.pos, sl.q),
                         ("fp32", sl.pos.astype(np.float32).astype(np.float64),
                          sl.q.astype(np.float32).astype(np.float64))]:
        t = time.time()
        out = soe_ewald2d.soe_full(pos, q, sl.box, sl.alpha, s, w, kc=kc)
        v = {"E": out["E"], "E_parts": list(out["E_parts"]),
             "modes_full_lattice": int(len(out["modes"][0])),
             "fingerprint": fingerprint(pos, q), "oracle_seconds": time.time() - t}
        v.update(_values(out, idx))
        d[name] = v
    return d


JOBS = {"rbe_large": ("rbe_large_fullk.json", rbe_large_fullk),
        "confined": ("confined_fullk.json", confined_fullk)}


if __name__ == "__main__":
    names = sys.argv[1:] or list(JOBS)
    for name in names:
        fname, fn = JOBS[name]
        d = fn()
        with open(os.path.join(HERE, fname), "w") as fh:
            json.dump(d, fh, indent=0)
        print(fname, {k: v for k, v in d.items() if not isinstance(v, (list, dict))})
