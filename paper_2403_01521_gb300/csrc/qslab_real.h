// Internal declarations of the real-space part (qslab_real.cu): the erfc
// sum of Eq. 2.10 over pairs within the cut-off rc, periodic in x and y.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace qslab {

struct RsGrid {
  int64_t N;
  int s;                    // cells of edge >= rc/s; (2s+1)^3 neighbour cells
  int ncx, ncy, ncz;        // cells (ncx, ncy >= 2s + 1)
  double Lx, Ly, Lz, hz;    // box and cell height in z
  double alpha, rc;
  double lj_eps, lj_sigma;  // shifted-truncated LJ between particles (eps = 0: none)
};
size_t rs_workspace_bytes(const RsGrid& g);
// phi, force (caller's order; may be NULL) and energy (device scalar, may be
// NULL) of the real-space sum; with lj_eps > 0 the force and energy include
// the LJ pairs (r < 2^(1/6) lj_sigma <= rc), phi does not. virial (device, 6
// doubles, or NULL): the pair virial (1/2) sum (F_ij)_a (r_ij)_b of the same
// pairs, as xx, yy, zz, xy, xz, yz. Returns the number of kernels launched.
template <typename T>
int launch_realspace(const RsGrid& g, const T* pos, const T* q, void* ws, unsigned* status,
                     double* energy, T* phi, T* force, cudaStream_t st, double* virial = nullptr);

}  // namespace qslab
