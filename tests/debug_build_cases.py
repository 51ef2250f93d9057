"""Small and ragged cases run through the library (child process of
test_gpu_debug_build.py, with QSLAB_LIBRARY=debug so that the debug build
with its internal index checks is loaded). Every call must end with status 0
(no check fired) and the FP64 results must match the oracle to 1e-10.
Prints one line per case and "DEBUG-CASES OK" at the end."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import paper_2403_01521_gb300 as qs  # noqa: E402
import workloads  # noqa: E402
from oracle import lattice, soe_ewald2d  # noqa: E402


def close(a, b, tol):
    return np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1.0)


def main():
    lib = qs.load()
    assert os.path.basename(lib._name) == "libqslab_debug.so", lib._name
    soe = qs.load_soe(16)
    n_cases = 0
    for n in (1, 2, 3, 5, 17, 300, 2049, 5000):
        box = (12.0, 10.0, 6.0)
        if n == 1:
            sl = workloads.Slab("one", np.array([[2.0, 3.0, 1.0]]), np.array([0.0]), box, 0.5, 16)
        else:
            m = n + (n % 2)
            sl = workloads.uniform_slab(m, box, 100 + n, alpha=0.5)
            if m != n:               # odd n: drop a particle, keep the slab neutral
                sl.pos, sl.q = sl.pos[:n], sl.q[:n].copy()
                sl.q[0] -= sl.q.sum()
        kc = lattice.kcut_for_tail(0.5, 1e-8)
        for prec in ("fp64", "fp32c"):
            for rbe in (None, (40, 3)):
                slab = qs.QSlab(0, prec).configure(box, 0.5, soe, kcut=kc, rbe=rbe)
                dt = torch.float64 if prec == "fp64" else torch.float32
                pos = torch.tensor(sl.pos, device="cuda", dtype=dt)
                q = torch.tensor(sl.q, device="cuda", dtype=dt)
                e, phi, F = slab.compute(pos, q)
                st = slab.status()
                assert st == 0, (n, prec, rbe, st)
                if prec == "fp64":
                    if rbe is None:
                        ref = soe_ewald2d.soe_full(sl.pos, sl.q, box, 0.5, *soe, kc=kc)
                    else:
                        mx, my, _ = slab.sampled_modes()
                        ref = soe_ewald2d.soe_rbe(sl.pos, sl.q, box, 0.5, *soe, mx, my)
                    assert close(phi.cpu().numpy(), ref["phi"], 1e-10), (n, rbe)
                    assert close(F.cpu().numpy(), ref["F"], 1e-8), (n, rbe)
                slab.close()
                n_cases += 1
                print("case", n, prec, "rbe" if rbe else "full-k", "ok", flush=True)
    # a batched call with an empty slab and uneven slabs
    reps = [workloads.uniform_slab(n, (20.0, 20.0, 8.0), 200 + n, alpha=0.4) for n in (6, 0, 700, 2)]
    reps[1].pos = np.zeros((0, 3)); reps[1].q = np.zeros(0)
    off = np.concatenate([[0], np.cumsum([r.N for r in reps])]).astype(np.int64)
    boxes = np.array([r.box for r in reps])
    for prec in ("fp64", "fp32c"):
        dt = torch.float64 if prec == "fp64" else torch.float32
        slab = qs.QSlab(0, prec).configure(reps[0].box, 0.4, soe, rbe=(64, 9))
        pos = torch.tensor(np.concatenate([r.pos for r in reps]), device="cuda", dtype=dt)
        q = torch.tensor(np.concatenate([r.q for r in reps]), device="cuda", dtype=dt)
        slab.compute_batched(pos, q, off, boxes)
        assert slab.status() == 0, prec
        slab.close()
        n_cases += 1
        print("batched", prec, "ok", flush=True)
    print("DEBUG-CASES OK", n_cases, flush=True)


if __name__ == "__main__":
    main()
