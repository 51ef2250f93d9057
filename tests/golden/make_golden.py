"""Write the stored expected values used by the GPU tests.

Every value here is computed by the FP64 oracle (oracle/) from the seeded
workloads (workloads.py); nothing comes from the CUDA library.

  rbe_large_fullk.json   the full-k long-range energy (kc at Gaussian tail
                         1e-8, M = 16 conditioned SOE) of the N = 1e6
                         random-batch workload, i.e. the expectation of its
                         random-batch estimator; used as the energy scale of
                         the FP32 energy tolerance. The positions are rounded
                         to FP32 first, as the FP32 path sees them. A
                         fingerprint of the inputs is stored beside it.

Run: python tests/golden/make_golden.py   (a few minutes on 8 cores)
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


def fingerprint(pos, q):
    return [float(np.sum(pos[:, 0])), float(np.sum(pos[:, 2] * q)), int(pos.shape[0])]


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
    return {"workload": "rbe_large (seed 3), positions rounded to float32",
            "kc_tail": 1e-8, "M": 16, "soe": "conditioned",
            "E_fullk": out["E"], "modes_full_lattice": int(len(out["modes"][0])),
            "fingerprint": fingerprint(pos, sl.q), "oracle_seconds": time.time() - t}


if __name__ == "__main__":
    d = rbe_large_fullk()
    with open(os.path.join(HERE, "rbe_large_fullk.json"), "w") as fh:
        json.dump(d, fh, indent=1)
    print(d)
