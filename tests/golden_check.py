"""Helpers for the stored expected values under tests/golden/."""
import numpy as np


def fingerprint(pos, q):
    return [float(np.sum(pos[:, 0])), float(np.sum(pos[:, 2] * q)), int(pos.shape[0])]


def fingerprint_matches(gold, pos, q, rtol=1e-12):
    fp = fingerprint(pos, q)
    ref = gold["fingerprint"]
    return fp[2] == ref[2] and all(abs(a - b) <= rtol * max(abs(b), 1.0) for a, b in zip(fp[:2], ref[:2]))
