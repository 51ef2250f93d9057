// Internal declarations of the Langevin dynamics driver (qslab_md.cu):
// BAOAB steps of Section 4.3's Langevin equation with the forces of this
// library plus the short-range model of Section 5.2.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace qslab {

struct MDDev {
  double dt, mass;
  double c1, c2;            // Ornstein-Uhlenbeck step v <- c1 v + c2 xi
  double wall_eps, wall_sigma;
  double Lx, Ly, Lz;
  uint64_t seed;
};

// Block count of the per-particle MD kernels (for the partial-sum buffer).
int md_blocks(int64_t N);

// B A O A of one step: half kick with `force`, half drift, the
// Ornstein-Uhlenbeck step with the noise of step ctr[0], half drift; x and y
// wrapped into the box.
template <typename T>
void launch_md_begin(int64_t N, const MDDev& p, T* pos, T* vel, const T* force,
                     const uint64_t* ctr, cudaStream_t st);

// Total force = flr + frs + LJ walls into `force`; with kick, the closing
// half kick of vel and ctr[0] += 1. Per-block partial sums of the wall
// energy and (vel not NULL) the kinetic energy go to part[2][md_blocks(N)].
template <typename T>
void launch_md_end(int64_t N, const MDDev& p, const T* pos, T* vel, const T* flr, const T* frs,
                   T* force, double* part, uint64_t* ctr, bool kick, cudaStream_t st);

// energies[0..3] = e_lr, e_rs, wall energy, kinetic energy (fixed order).
void launch_md_energies(int64_t N, const double* part, const double* e_lr, const double* e_rs,
                        double* energies, cudaStream_t st);

}  // namespace qslab
