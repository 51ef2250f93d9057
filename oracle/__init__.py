"""FP64 CPU oracle for the SOE-Ewald2D / RBSE2D long-range path.

THIS PACKAGE IS TEST INFRASTRUCTURE. Only the tests, the smoke check of
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import or run
it. The CUDA library never links, imports or calls it, and it shares no code
with the library: it is a plain, slow, obviously correct restatement of the
paper (Gan, Gao, Liang, Xu, "Fast algorithm for quasi-2D Coulomb systems",
arXiv 2403.01521), in FP64.

Modules:
  lattice       k modes, H (Eqs. 4.5/4.6), h(k), Philox4x64-10 and the
                RBE k-sampler, the j = i constants (Eqs. 3.20, 3.25) and
                U_self (Eq. 2.12)
  ewald2d       exact Ewald2D long-range part (Lemma 2.1) with the erfc
                kernel, real-space sum (Eq. 2.10), brute image sums (Eq. 2.8),
                direct SOE pair sums (Eqs. 3.21, 3.26)
  soe_ewald2d   the sorted SOE recursion (Eqs. 3.27-3.30, Appendix E) for
                the full k-sum and for the random-batch estimator (Eq. 4.7)
  soe_check     SOE table checks (Eq. 3.1, Thm 3.2, Eq. 3.24)
  walls         charged walls at z = 0 and z = Lz: the particle-slab
                potential, forces and energy (Section 2.4, Thm 2.4)
  virial        the virial tensor W_ab = -dE/d eps_ab of the long-range
                energy (exact and SOE, full k-sum and random batch), of the
                particle-slab energy and of the real-space sum (pressure for
                the NPT ensemble, Section 4.3; the L_z-dependent constant of
                Thm 2.4's uniform-density case)
  md            Langevin dynamics (Section 4.3) with the short-range model of
                Section 5.2 (shifted-truncated LJ between particles and at
                the walls), BAOAB steps, Philox normal noise
  soe_recursion.c   the recursion itself, plain C99 + OpenMP

Every function is pinned by tests under tests/ against closed forms,
invariants, brute force or the paper's error bounds (see the test files).
"""
from . import ewald2d, lattice, md, soe_check, soe_ewald2d, virial, walls  # noqa: F401
from .ewald2d import ewald2d_longrange, image_sum_extrapolated, realspace, soe_pair_direct  # noqa: F401
from .soe_ewald2d import soe_full, soe_rbe, soe_rbe_seeded  # noqa: F401
