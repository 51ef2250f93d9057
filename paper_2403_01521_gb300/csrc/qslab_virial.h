// Internal declarations of the virial of the long-range energy
// (qslab_virial.cu): W_ab = -dE/d eps_ab under a strain of the particles,
// the lateral lattice and the charged walls, for the NPT ensemble (Section
// 4.3) and the L_z-dependent constant of the particle-slab potential (Thm 2.4).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "qslab_internal.h"

namespace qslab {

// Inputs of one virial pass; the sorted arrays, the mode tables and the
// forward carries are those of the long-range call just issued on the same
// stream (its workspace is still intact).
template <typename T>
struct VirArgs {
  ScanPlan plan;
  Reps rp;
  ModeTab<T> modes;
  PairTab pairs;
  double alpha;
  int rbe;                       // random-batch weights (else full k-sum, half plane)
  const T* zs;
  const T* dz;
  const T* qs;
  const typename PhaseT<T>::type* xh;
  const typename PhaseT<T>::type* yh;
  const float2* trig;            // FP32: [256] (cos, sin) of j/256 turns
  const Cplx<T>* carry;          // [2][nchunks][nstates][Kpad] (forward half used)
  const Cplx<T>* agg;            // pass A's aggregates, same layout (energy pass: backward half)
  const T* pos;                  // caller's order: N x 3, q: N, force: N x 3
  const T* q;
  const T* force;
  const double* energies;        // [R] energies of the call (particles and walls)
  const double* vdiag;           // [R][3] j = i lateral virial per unit sum q^2
  WallTab walls;
  double* virial;                // [R][6] output: xx, yy, zz, xy, xz, yz
};

// workspace bytes for virial_launch
size_t virial_workspace_bytes(const ScanPlan& plan, const Reps& rp);
// Issues the virial kernels on st; returns the number of kernels launched.
template <typename T>
int launch_virial(const VirArgs<T>& a, void* ws, cudaStream_t st);
// The k != 0 pair energy of every replica from forward sums only (the
// energy-only call): per mode, the sum over chunks of
// gam Re sum_beta c_beta S_beta, kept in ws. Uses a.plan, rp, modes, pairs,
// the sorted arrays, trig and the forward carries (virial_workspace_bytes of
// scratch). Returns the number of kernels launched.
template <typename T>
int launch_energy_pass(const VirArgs<T>& a, void* ws, cudaStream_t st);
// energies[r] += the replica's mode energies left in ws by launch_energy_pass
// (fixed order). Returns the number of kernels launched.
int launch_energy_add(const ScanPlan& plan, const Reps& rp, const void* ws, double* energies,
                      cudaStream_t st);

}  // namespace qslab
