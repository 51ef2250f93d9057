// Real-space part of the Ewald2D splitting (Eq. 2.10): the short-range
// potential phi_s,i = sum_j' sum_images q_j erfc(alpha |r_ij + M|)/|r_ij + M|
// and its forces, truncated at |r| <= rc (Section 2.3), with images
// M = (mx Lx, my Ly, 0) in x and y only.
//
// Cell list: the box is cut into ncx x ncy x ncz cells of edge >= rc
// (ncx, ncy >= 3, so that the 3 x 3 x 3 neighbouring cells of a cell are
// distinct images); particles are sorted by cell with the radix sort of
// qslab_sort.cu; one CTA per home cell streams the neighbouring cells through
// shared memory, each with the image shift of its periodic wrap.
// Every pair is evaluated from both ends (no atomics, deterministic sums).
#include <cstdint>
#include <cuda_runtime.h>

#include "qslab_internal.h"
#include "qslab_math.cuh"

namespace qslab {

template <typename T> struct RsRec { T x, y, z, q; };

__device__ __forceinline__ float rs_erfc(float x) { return erfcf(x); }
__device__ __forceinline__ double rs_erfc(double x) { return erfc(x); }
__device__ __forceinline__ float rs_exp_neg(float x) { return __expf(-x); }
__device__ __forceinline__ double rs_exp_neg(double x) { return exp(-x); }
__device__ __forceinline__ float rs_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double rs_sqrt(double x) { return sqrt(x); }

// box fraction of x in [0, 1)
__device__ __forceinline__ double rs_frac(double x, double L) {
  double f = x / L;
  f -= floor(f);
  return f < 1.0 ? f : 0.0;
}

template <typename T>
__global__ void rs_keys_kernel(RsGrid g, const T* __restrict__ pos, const T* __restrict__ q,
                               uint32_t* keys, uint32_t* vals, unsigned* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2], qi = q[i];
    unsigned flag = 0;
    if (!isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(qi)) flag = kStNonfinite;
    else if (!(z >= (T)0) || !((double)z <= g.Lz)) flag = kStZRange;
    if (flag) atomicOr(status, flag);
    int cx = 0, cy = 0, cz = 0;
    if (!flag) {
      cx = min((int)(rs_frac((double)x, g.Lx) * g.ncx), g.ncx - 1);
      cy = min((int)(rs_frac((double)y, g.Ly) * g.ncy), g.ncy - 1);
      cz = min((int)((double)z / g.hz), g.ncz - 1);
    }
    keys[i] = (uint32_t)((cz * g.ncy + cy) * g.ncx + cx);
    vals[i] = (uint32_t)i;
  }
}

// first and one-past-last sorted index of every non-empty cell
__global__ void rs_cells_kernel(int64_t N, const uint32_t* __restrict__ skeys, int32_t* cstart,
                                int32_t* cend) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = skeys[i];
    if (i == 0 || skeys[i - 1] != k) cstart[k] = (int32_t)i;
    if (i == N - 1 || skeys[i + 1] != k) cend[k] = (int32_t)(i + 1);
  }
}

// sorted records with x, y wrapped into the box
template <typename T>
__global__ void rs_gather_kernel(RsGrid g, const T* __restrict__ pos, const T* __restrict__ q,
                                 const uint32_t* __restrict__ perm, RsRec<T>* rec) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t o = perm[i];
    RsRec<T> r;
    r.x = (T)(rs_frac((double)pos[3 * (int64_t)o], g.Lx) * g.Lx);
    r.y = (T)(rs_frac((double)pos[3 * (int64_t)o + 1], g.Ly) * g.Ly);
    r.z = pos[3 * (int64_t)o + 2];
    r.q = q[o];
    rec[i] = r;
  }
}

constexpr int kRsThreads = 128;

// One CTA per home cell. For every tile of home particles (one per thread),
// the 27 neighbouring cells are streamed through shared memory in tiles of
// kRsThreads records, shifted by the image of their periodic wrap.
template <typename T>
__global__ void __launch_bounds__(kRsThreads) rs_pair_kernel(RsGrid g, const int32_t* __restrict__ cstart,
                                                           const int32_t* __restrict__ cend,
                                                           const RsRec<T>* __restrict__ rec,
                                                           const uint32_t* __restrict__ perm,
                                                           T* phi_out, T* force_out, double* ecell) {
  __shared__ RsRec<T> tile[kRsThreads];
  __shared__ double red[kRsThreads / 32];
  const int c = blockIdx.x;
  const int cx = c % g.ncx, cy = (c / g.ncx) % g.ncy, cz = c / (g.ncx * g.ncy);
  const int hs = cstart[c], he = cend[c];
  const T alpha = (T)g.alpha, rc2 = (T)(g.rc * g.rc);
  const T a2 = alpha * alpha;
  const T two_a_sqpi = (T)(2.0 * g.alpha / 1.7724538509055160);
  double e_acc = 0.0;
  for (int i0 = hs; i0 < he; i0 += kRsThreads) {
    const int i = i0 + threadIdx.x;
    const bool live = i < he;
    RsRec<T> ri{0, 0, 0, 0};
    if (live) ri = rec[i];
    T ph = 0, fx = 0, fy = 0, fz = 0;
    for (int dz = -1; dz <= 1; ++dz) {
      const int nz = cz + dz;
      if (nz < 0 || nz >= g.ncz) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        int ny = cy + dy;
        T sy = 0;
        if (ny < 0) { ny += g.ncy; sy = (T)(-g.Ly); }
        else if (ny >= g.ncy) { ny -= g.ncy; sy = (T)g.Ly; }
        for (int dx = -1; dx <= 1; ++dx) {
          int nx = cx + dx;
          T sx = 0;
          if (nx < 0) { nx += g.ncx; sx = (T)(-g.Lx); }
          else if (nx >= g.ncx) { nx -= g.ncx; sx = (T)g.Lx; }
          const int nc = (nz * g.ncy + ny) * g.ncx + nx;
          const int js = cstart[nc], je = cend[nc];
          for (int j0 = js; j0 < je; j0 += kRsThreads) {
            const int cntj = min(kRsThreads, je - j0);
            __syncthreads();
            if (threadIdx.x < cntj) {
              RsRec<T> rj = rec[j0 + threadIdx.x];
              rj.x += sx;
              rj.y += sy;
              tile[threadIdx.x] = rj;
            }
            __syncthreads();
            if (live) {
              for (int t = 0; t < cntj; ++t) {
                const RsRec<T> rj = tile[t];
                const T ddx = ri.x - rj.x, ddy = ri.y - rj.y, ddz = ri.z - rj.z;
                const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                if (r2 <= rc2 && (j0 + t != i || nc != c)) {
                  const T r = rs_sqrt(r2);
                  const T inv = (T)1 / r;
                  const T e = rs_erfc(alpha * r) * inv;          // erfc(a r)/r
                  const T g2 = two_a_sqpi * rs_exp_neg(a2 * r2);  // 2a/sqrt(pi) e^{-a^2 r^2}
                  const T fr = (e + g2) * inv * inv;             // -(d/dr)(erfc(a r)/r) / r
                  ph = fma(rj.q, e, ph);
                  const T w = rj.q * fr;
                  fx = fma(w, ddx, fx);
                  fy = fma(w, ddy, fy);
                  fz = fma(w, ddz, fz);
                }
              }
            }
          }
        }
      }
    }
    if (live) {
      const uint32_t o = perm[i];
      if (phi_out) phi_out[o] = ph;
      if (force_out) {
        force_out[3 * (int64_t)o] = ri.q * fx;
        force_out[3 * (int64_t)o + 1] = ri.q * fy;
        force_out[3 * (int64_t)o + 2] = ri.q * fz;
      }
      e_acc += 0.5 * (double)ri.q * (double)ph;
    }
  }
  for (int o = 16; o; o >>= 1) e_acc += __shfl_xor_sync(0xffffffffu, e_acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e_acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kRsThreads / 32; ++w) s += red[w];
    ecell[c] = s;
  }
}

// sum of the cells' energies in a fixed order (one CTA)
__global__ void rs_energy_kernel(int ncell, const double* ecell, double* energy) {
  __shared__ double red[32];
  double s = 0.0;
  for (int j = threadIdx.x; j < ncell; j += blockDim.x) s += ecell[j];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *energy = t;
  }
}

size_t rs_workspace_bytes(const RsGrid& g) {
  const int64_t ncell = (int64_t)g.ncx * g.ncy * g.ncz;
  auto a = [](size_t b) { return (b + 255) & ~size_t(255); };
  return a(sort_workspace_bytes(g.N, 4)) + 2 * a(4 * (size_t)ncell) + a(8 * (size_t)ncell) +
         a(sizeof(RsRec<double>) * (size_t)g.N);
}

template <typename T>
int launch_realspace(const RsGrid& g, const T* pos, const T* q, void* ws, unsigned* status,
                     double* energy, T* phi, T* force, cudaStream_t st) {
  const int64_t ncell = (int64_t)g.ncx * g.ncy * g.ncz;
  auto a = [](size_t b) { return (b + 255) & ~size_t(255); };
  char* p = static_cast<char*>(ws);
  SortWork sw;
  sort_bind_workspace(sw, p, g.N, 4);
  p += a(sort_workspace_bytes(g.N, 4));
  int32_t* cstart = reinterpret_cast<int32_t*>(p); p += a(4 * (size_t)ncell);
  int32_t* cend = reinterpret_cast<int32_t*>(p); p += a(4 * (size_t)ncell);
  double* ecell = reinterpret_cast<double*>(p); p += a(8 * (size_t)ncell);
  RsRec<T>* rec = reinterpret_cast<RsRec<T>*>(p);
  int blocks = (int)((g.N + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  rs_keys_kernel<T><<<blocks, 256, 0, st>>>(g, pos, q, static_cast<uint32_t*>(sw.keys[0]),
                                            sw.vals[0], status);
  int passes = 1;
  while (passes < 4 && (uint64_t)ncell > (1ull << (8 * passes))) ++passes;
  const int r = radix_sort(sw, g.N, 4, passes, 0, st);
  cudaMemsetAsync(cstart, 0, 4 * (size_t)ncell, st);
  cudaMemsetAsync(cend, 0, 4 * (size_t)ncell, st);
  rs_cells_kernel<<<blocks, 256, 0, st>>>(g.N, static_cast<const uint32_t*>(sw.keys[r]), cstart,
                                          cend);
  rs_gather_kernel<T><<<blocks, 256, 0, st>>>(g, pos, q, sw.vals[r], rec);
  rs_pair_kernel<T><<<(unsigned)ncell, kRsThreads, 0, st>>>(g, cstart, cend, rec, sw.vals[r], phi,
                                                            force, ecell);
  if (energy) rs_energy_kernel<<<1, 256, 0, st>>>((int)ncell, ecell, energy);
  return 3 + 3 * passes + (energy ? 2 : 1);
}

template int launch_realspace<float>(const RsGrid&, const float*, const float*, void*, unsigned*,
                                     double*, float*, float*, cudaStream_t);
template int launch_realspace<double>(const RsGrid&, const double*, const double*, void*,
                                      unsigned*, double*, double*, double*, cudaStream_t);

}  // namespace qslab
