"""Seeded synthetic inputs for the quasi-2D slab workloads.

This module only draws particles (positions and charges) and states the
physical parameters of each workload. It holds none of the method's
arithmetic, so both the CUDA path and the FP64 oracle can take their inputs
from it without sharing code.

The paper measures on synthetic random ions only (Section 5.1: 50 cations and
50 anions uniform in a box; Section 5.2: 1:1 electrolytes between walls).
The recipes below have the shapes, sizes and value distributions of those
workloads, scaled to the sizes this library is measured at:

  small_full   N=1000, 500 of +1 and 500 of -1, uniform in 30 x 30 x 10,
               alpha=0.3, full k-sum with Gaussian tail <= 1e-8, M=16
  fp32_full    N=1e5 charges +-1 uniform in 100 x 100 x 20, alpha=0.25,
               full k-sum (tail 1e-8), M=16
  rbe_large    N=1e6 charges +-1 uniform in 400 x 400 x 50, alpha=0.1,
               P=200 importance-sampled k per call, M=16
  rbe_unbiased N=1e4 at the same density (40 x 40 x 50, alpha=0.1), for the
               mean-over-seeds check against the full k-sum
  replicas     512 slabs, N_r uniform on [500, 50000] (even), Lz_r uniform
               on [5, 40], Lx=Ly set by number density 0.05, charges +-1
  confined     N=2e5 in 200 x 200 x 2, z exponential from a randomly chosen
               wall with decay length 0.2 (redrawn above Lz), charges
               N(0,1) minus their mean, alpha=0.2, M=24, full k-sum
  cations_walls  n cations (+1) uniform in L x L x 30 between an uncharged
               bottom wall and a top wall of density -n/L^2 (Section 5.2's
               cation-only system: n = 436, L = 100, sigma_top = -0.0436),
               alpha=0.1, full k-sum
  electrolyte_walls  n/2 cations and n/2 anions uniform in L x L x 30
               between walls of density +-n/(2 L^2) (Section 5.2's 1:1
               electrolyte: n = 436, L = 100, sigma = +-0.0218), alpha=0.1

Every generator takes a seed and returns float64 numpy arrays; callers that
test a float32 path round them to float32 and feed the same rounded values to
both sides.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Slab:
    """One slab system: particles plus the parameters of its workload."""

    name: str
    pos: np.ndarray          # (N, 3) float64, x,y in [0,L), z in [0,Lz]
    q: np.ndarray            # (N,) float64, sums to zero unless walls are set
    box: tuple               # (Lx, Ly, Lz)
    alpha: float
    M: int                   # number of SOE terms
    tail: float = 1e-8       # Gaussian tail that sets the k cutoff (full k-sum)
    P: int = 0               # RBE batch size (0 = full k-sum)
    rc: float = 10.0         # real-space cutoff (used only for totals)
    walls: tuple = None      # (sigma_bot, sigma_top) uniform wall charge densities

    @property
    def N(self) -> int:
        return int(self.q.shape[0])


def _pm_charges(rng: np.random.Generator, n: int) -> np.ndarray:
    """n/2 charges of +1 and n/2 of -1 in random order (n even)."""
    if n % 2:
        raise ValueError("need an even particle count for +-1 neutrality")
    q = np.concatenate([np.ones(n // 2), -np.ones(n // 2)])
    rng.shuffle(q)
    return q


def uniform_slab(n: int, box, seed: int, name: str = "uniform",
                 alpha: float = 0.3, M: int = 16, P: int = 0,
                 tail: float = 1e-8, rc: float = 10.0) -> Slab:
    """n charges +-1 uniform in [0,Lx) x [0,Ly) x [0,Lz]."""
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = box
    pos = np.empty((n, 3))
    pos[:, 0] = rng.random(n) * Lx
    pos[:, 1] = rng.random(n) * Ly
    pos[:, 2] = rng.random(n) * Lz
    q = _pm_charges(rng, n)
    return Slab(name, pos, q, (float(Lx), float(Ly), float(Lz)), alpha, M,
                tail, P, rc)


def small_full(seed: int = 1, n: int = 1000) -> Slab:
    return uniform_slab(n, (30.0, 30.0, 10.0), seed, "small_full",
                        alpha=0.3, M=16)


def fp32_full(seed: int = 2, n: int = 100_000) -> Slab:
    return uniform_slab(n, (100.0, 100.0, 20.0), seed, "fp32_full",
                        alpha=0.25, M=16)


def rbe_large(seed: int = 3, n: int = 1_000_000, P: int = 200) -> Slab:
    return uniform_slab(n, (400.0, 400.0, 50.0), seed, "rbe_large",
                        alpha=0.1, M=16, P=P)


def rbe_unbiased(seed: int = 3, n: int = 10_000, P: int = 200) -> Slab:
    return uniform_slab(n, (40.0, 40.0, 50.0), seed, "rbe_unbiased",
                        alpha=0.1, M=16, P=P)


def confined(seed: int = 5, n: int = 200_000) -> Slab:
    """Strongly confined slab with charge layers at both walls."""
    rng = np.random.default_rng(seed)
    Lx = Ly = 200.0
    Lz = 2.0
    pos = np.empty((n, 3))
    pos[:, 0] = rng.random(n) * Lx
    pos[:, 1] = rng.random(n) * Ly
    d = rng.exponential(0.2, n)
    bad = d > Lz
    while bad.any():
        d[bad] = rng.exponential(0.2, int(bad.sum()))
        bad = d > Lz
    top = rng.random(n) < 0.5
    pos[:, 2] = np.where(top, Lz - d, d)
    q = rng.standard_normal(n)
    q -= q.mean()
    return Slab("confined", pos, q, (Lx, Ly, Lz), 0.2, 24)


def replicas(seed: int = 4, R: int = 512, nmin: int = 500, nmax: int = 50_000,
             density: float = 0.05):
    """R independent neutral slabs of uneven size (list of Slab)."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(R):
        n = int(rng.integers(nmin, nmax + 1))
        n -= n % 2
        Lz = float(rng.uniform(5.0, 40.0))
        L = math.sqrt(n / (density * Lz))
        sub = int(rng.integers(0, 2**31 - 1))
        out.append(uniform_slab(n, (L, L, Lz), sub, f"replica{r}",
                                alpha=0.25, M=16, P=200))
    return out


def tiny_neutral(n: int, box, seed: int) -> Slab:
    """A handful of +-1 charges, for brute-force checks."""
    return uniform_slab(n, box, seed, "tiny", alpha=0.5, M=16)


def cations_walls(seed: int = 6, n: int = 436, L: float = 100.0) -> Slab:
    """Cations only, neutralised by the top wall's charge."""
    rng = np.random.default_rng(seed)
    Lz = 30.0
    pos = np.column_stack([rng.random(n) * L, rng.random(n) * L, rng.random(n) * Lz])
    return Slab("cations_walls", pos, np.ones(n), (L, L, Lz), 0.1, 16,
                walls=(0.0, -n / (L * L)))


def electrolyte_walls(seed: int = 7, n: int = 436, L: float = 100.0) -> Slab:
    """1:1 electrolyte between oppositely charged walls."""
    rng = np.random.default_rng(seed)
    Lz = 30.0
    pos = np.column_stack([rng.random(n) * L, rng.random(n) * L, rng.random(n) * Lz])
    sig = n / (2 * L * L)
    return Slab("electrolyte_walls", pos, _pm_charges(rng, n), (L, L, Lz), 0.1, 16,
                walls=(sig, -sig))
