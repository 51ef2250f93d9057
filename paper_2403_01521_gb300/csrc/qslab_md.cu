// Langevin dynamics of a slab electrolyte (Section 4.3's Langevin equation)
// in BAOAB splitting (Leimkuhler and Matthews 2013), with the particles held
// between the walls by the purely repulsive LJ walls of Section 5.2.
//
// One step: B (v += dt/2 F/m), A (x += dt/2 v), O (v <- c1 v + c2 xi,
// c1 = e^{-gamma dt/m}, c2 = sqrt((1 - c1^2) kT/m)), A, new forces, B.
// Noise xi of particle i at step n: Philox4x64-10 with counter
// (i, n, 0, tag), key (seed, 0); words (0, 1) and (2, 3) give two
// Box-Muller pairs, xi = (first pair, first of the second pair).
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "qslab_internal.h"
#include "qslab_math.cuh"
#include "qslab_md.h"

namespace qslab {

constexpr int kMdThreads = 256;
constexpr uint64_t kMdTag = 0x4D445331ull;

int md_blocks(int64_t N) {
  int64_t b = (N + kMdThreads - 1) / kMdThreads;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ double md_uniform53(uint64_t w) {
  return (double)(w >> 11) * 1.1102230246251565e-16;   // 2^-53
}

template <typename T>
__device__ __forceinline__ T md_wrap(T x, T L) {
  return x - L * floor(x / L);
}

template <typename T>
__global__ void __launch_bounds__(kMdThreads) md_begin_kernel(int64_t N, MDDev p, T* pos, T* vel,
                                                              const T* __restrict__ force,
                                                              const uint64_t* ctr) {
  const uint64_t step = ctr[0];
  const T h = (T)(0.5 * p.dt), m = (T)p.mass;
  const T Lx = (T)p.Lx, Ly = (T)p.Ly;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    T x[3], v[3];
    for (int d = 0; d < 3; ++d) {
      v[d] = vel[3 * i + d] + h * force[3 * i + d] / m;
      x[d] = pos[3 * i + d] + h * v[d];
    }
    x[0] = md_wrap(x[0], Lx);
    x[1] = md_wrap(x[1], Ly);
    U64x4 c;
    c.v[0] = (uint64_t)i; c.v[1] = step; c.v[2] = 0; c.v[3] = kMdTag;
    const U64x4 w = philox4x64_10(c, p.seed, 0ull);
    double xi[3];
    {
      const double r = sqrt(-2.0 * log(1.0 - md_uniform53(w.v[0])));
      const double th = 2.0 * 3.14159265358979323846 * md_uniform53(w.v[1]);
      xi[0] = r * cos(th);
      xi[1] = r * sin(th);
      const double r2 = sqrt(-2.0 * log(1.0 - md_uniform53(w.v[2])));
      const double th2 = 2.0 * 3.14159265358979323846 * md_uniform53(w.v[3]);
      xi[2] = r2 * cos(th2);
    }
    for (int d = 0; d < 3; ++d) {
      v[d] = (T)(p.c1 * (double)v[d] + p.c2 * xi[d]);
      x[d] = x[d] + h * v[d];
    }
    x[0] = md_wrap(x[0], Lx);
    x[1] = md_wrap(x[1], Ly);
    for (int d = 0; d < 3; ++d) {
      pos[3 * i + d] = x[d];
      vel[3 * i + d] = v[d];
    }
  }
}

// shifted-truncated LJ of the distance d to a wall: energy and -dU/dd
__device__ __forceinline__ void md_wall(double d, double eps, double sig, double& e, double& f) {
  e = 0.0;
  f = 0.0;
  if (eps > 0.0 && d < 1.122462048309373 * sig) {    // 2^(1/6) sigma
    const double s = sig / d;
    const double s6 = s * s * s * s * s * s;
    e = 4.0 * eps * (s6 * s6 - s6 + 0.25);
    f = 24.0 * eps * (2.0 * s6 * s6 - s6) / d;
  }
}

template <typename T>
__global__ void __launch_bounds__(kMdThreads) md_end_kernel(int64_t N, MDDev p,
                                                            const T* __restrict__ pos, T* vel,
                                                            const T* __restrict__ flr,
                                                            const T* __restrict__ frs, T* force,
                                                            double* part, uint64_t* ctr, int kick) {
  __shared__ double red[2][kMdThreads / 32];
  const T h = (T)(0.5 * p.dt), m = (T)p.mass;
  double ew = 0.0, ek = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double z = (double)pos[3 * i + 2];
    double eb, fb, et, ft;
    md_wall(z, p.wall_eps, p.wall_sigma, eb, fb);
    md_wall(p.Lz - z, p.wall_eps, p.wall_sigma, et, ft);
    ew += eb + et;
    T F[3];
    F[0] = flr[3 * i] + frs[3 * i];
    F[1] = flr[3 * i + 1] + frs[3 * i + 1];
    F[2] = flr[3 * i + 2] + frs[3 * i + 2] + (T)(fb - ft);
    for (int d = 0; d < 3; ++d) force[3 * i + d] = F[d];
    if (vel) {
      double k2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        T v = vel[3 * i + d];
        if (kick) {
          v = v + h * F[d] / m;
          vel[3 * i + d] = v;
        }
        k2 += (double)v * (double)v;
      }
      ek += 0.5 * p.mass * k2;
    }
  }
  for (int o = 16; o; o >>= 1) {
    ew += __shfl_xor_sync(0xffffffffu, ew, o);
    ek += __shfl_xor_sync(0xffffffffu, ek, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ew;
    red[1][threadIdx.x >> 5] = ek;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kMdThreads / 32; ++w) { a += red[0][w]; b += red[1][w]; }
    part[blockIdx.x] = a;
    part[gridDim.x + blockIdx.x] = b;
    if (kick && blockIdx.x == 0) ctr[0] += 1;   // md_begin of this step has completed
  }
}

__global__ void md_energies_kernel(int nb, const double* part, const double* e_lr,
                                   const double* e_rs, double* energies) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int j = 0; j < nb; ++j) { a += part[j]; b += part[nb + j]; }
  energies[0] = *e_lr;
  energies[1] = *e_rs;
  energies[2] = a;
  energies[3] = b;
}

template <typename T>
void launch_md_begin(int64_t N, const MDDev& p, T* pos, T* vel, const T* force,
                     const uint64_t* ctr, cudaStream_t st) {
  // the thermostat's normals are FP64 (Box-Muller), and an SM issues FP64 at
  // a small fraction of its FP32 rate: 64-thread blocks spread a small N
  // over as many SMs as possible (each particle's result is independent of
  // the thread that computes it)
  int64_t b = (N + 63) / 64;
  if (b > 152 * 16) b = 152 * 16;
  md_begin_kernel<T><<<(int)b, 64, 0, st>>>(N, p, pos, vel, force, ctr);
}

template <typename T>
void launch_md_end(int64_t N, const MDDev& p, const T* pos, T* vel, const T* flr, const T* frs,
                   T* force, double* part, uint64_t* ctr, bool kick, cudaStream_t st) {
  md_end_kernel<T><<<md_blocks(N), kMdThreads, 0, st>>>(N, p, pos, vel, flr, frs, force, part, ctr,
                                                        kick ? 1 : 0);
}

void launch_md_energies(int64_t N, const double* part, const double* e_lr, const double* e_rs,
                        double* energies, cudaStream_t st) {
  md_energies_kernel<<<1, 32, 0, st>>>(md_blocks(N), part, e_lr, e_rs, energies);
}

template void launch_md_begin<float>(int64_t, const MDDev&, float*, float*, const float*,
                                     const uint64_t*, cudaStream_t);
template void launch_md_begin<double>(int64_t, const MDDev&, double*, double*, const double*,
                                      const uint64_t*, cudaStream_t);
template void launch_md_end<float>(int64_t, const MDDev&, const float*, float*, const float*,
                                   const float*, float*, double*, uint64_t*, bool, cudaStream_t);
template void launch_md_end<double>(int64_t, const MDDev&, const double*, double*, const double*,
                                    const double*, double*, double*, uint64_t*, bool,
                                    cudaStream_t);

}  // namespace qslab
