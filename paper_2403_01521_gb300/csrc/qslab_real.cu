// Real-space part of the Ewald2D splitting (Eq. 2.10): the short-range
// potential phi_s,i = sum_j' sum_images q_j erfc(alpha |r_ij + M|)/|r_ij + M|
// and its forces, truncated at |r| <= rc (Section 2.3), with images
// M = (mx Lx, my Ly, 0) in x and y only.
//
// Cell list: the box is cut into ncx x ncy x ncz cells of edge >= rc/s
// (ncx, ncy >= 2s + 1, so that the (2s+1)^3 neighbouring cells of a cell
// are distinct images); particles are sorted by cell with the radix sort of
// qslab_sort.cu; CTAs take tiles of a home cell's particles and stream the
// neighbouring cells through shared memory, each with the image shift of its
// periodic wrap.
// Every pair is evaluated from both ends (no atomics, deterministic sums).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "qslab_internal.h"
#include "qslab_real.h"
#include "qslab_math.cuh"

namespace qslab {

template <typename T> struct RsRec { T x, y, z, q; };

// erfc(x) e^{x^2} for x >= 0 in FP32, branch-free: t P(2t - 1) with
// t = 1/(1 + x/2) (the approximate reciprocal, within 2 ulp) and P of degree
// 10 fitted by least squares in the relative error (fit_erfcx.py in the
// package; relative error 1.2e-8 in exact arithmetic, below 7e-7 evaluated
// in FP32).
__device__ __forceinline__ float rs_erfcx(float x) {
  const float t = __fdividef(1.0f, fmaf(0.5f, x, 1.0f));
  const float s = fmaf(2.0f, t, -1.0f);
  float p = 4.218412153e-05f;
  p = fmaf(p, s, -3.663383905e-05f);
  p = fmaf(p, s, -2.994463409e-04f);
  p = fmaf(p, s, 4.307417894e-04f);
  p = fmaf(p, s, 1.529219982e-03f);
  p = fmaf(p, s, -3.243504795e-03f);
  p = fmaf(p, s, -1.075165204e-02f);
  p = fmaf(p, s, 1.822168389e-02f);
  p = fmaf(p, s, 1.397357374e-01f);
  p = fmaf(p, s, 3.435803177e-01f);
  p = fmaf(p, s, 5.107913568e-01f);
  return t * p;
}

// erfc(a r) and e^{-a^2 r^2} of one pair: FP32 through erfcx and one fast
// exponential shared by both terms; FP64 with the library functions
__device__ __forceinline__ void rs_erfc_exp(float ar, float ar2, float& erfc_v, float& ex) {
  ex = __expf(-ar2);
  erfc_v = rs_erfcx(ar) * ex;
}
__device__ __forceinline__ void rs_erfc_exp(double ar, double ar2, double& erfc_v, double& ex) {
  ex = exp(-ar2);
  erfc_v = erfc(ar);
}
// 1/r from r^2: the FP32 reciprocal square root (a few ulp) on the FP32
// path, the exact FP64 operations on the FP64 path
__device__ __forceinline__ float rs_rinv(float r2) { return rsqrtf(r2); }
__device__ __forceinline__ double rs_rinv(double r2) { return 1.0 / sqrt(r2); }

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

// cstart[k] = first sorted index of cell k (= of the first cell >= k that
// is not empty; N for k = ncell), by binary search in the sorted keys, so
// that the cells of a row of the grid form one contiguous range
__global__ void rs_cells_kernel(int64_t N, int64_t ncell, const uint32_t* __restrict__ skeys,
                                int32_t* cstart) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= ncell;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = N;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)skeys[mid] < k) lo = mid + 1; else hi = mid;
    }
    cstart[k] = (int32_t)lo;
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

constexpr int kRsThreads = 64;   // home particles per CTA, one per thread
constexpr int kRsRow = 512;      // neighbour records staged in shared memory at once

// Grid (cell, part): CTA (c, y) takes the home tiles y, y + gridDim.y, ... of
// cell c (kRsThreads particles each, one per thread). Cells have edge
// >= rc/s; the (2s+1)^3 neighbouring cells are visited row by row: the
// cells of a row in x are consecutive keys, so a row is one or two
// contiguous ranges of sorted particles (two where it wraps around the box,
// each with its image shift). A row is staged in shared memory in one piece
// (kRsRow records at a time), padded to a multiple of 32 with records far
// outside any cut-off. Per group of 32 staged records every thread first
// marks those within rc of its particle in a 32-bit mask, then evaluates
// erfc and exp for the marked pairs only, so that the warp does not run the
// pair arithmetic for the candidates outside rc. A warp without a home
// particle only helps to stage the rows.
// VIR: also the pair virial (1/2) sum_{i,j} (F_ij)_a (r_ij)_b of the CTA's
// particles (Coulomb and LJ pairs) into vcell[cta][6] (xx, yy, zz, xy, xz, yz).
template <typename T, bool LJ, bool VIR>
__global__ void __launch_bounds__(kRsThreads) rs_pair_kernel(RsGrid g,
                                                           const int32_t* __restrict__ cstart,
                                                           const RsRec<T>* __restrict__ rec,
                                                           const uint32_t* __restrict__ perm,
                                                           T* phi_out, T* force_out, double* ecell,
                                                           double* vcell) {
  __shared__ RsRec<T> buf[kRsRow];
  __shared__ double red[kRsThreads / 32];
  __shared__ double vred[VIR ? 6 : 1][kRsThreads / 32];
  double v_acc[6] = {0, 0, 0, 0, 0, 0};
  const int c = blockIdx.x;
  const int S = g.s;
  const int cx = c % g.ncx, cy = (c / g.ncx) % g.ncy, cz = c / (g.ncx * g.ncy);
  const int hs = cstart[c], he = cstart[c + 1];
  const T alpha = (T)g.alpha, rc2 = (T)(g.rc * g.rc);
  const T a2 = alpha * alpha;
  const T two_a_sqpi = (T)(2.0 * g.alpha / 1.7724538509055160);
  // shifted-truncated LJ (the short-range model of Section 5.2), optional
  const T lj_s2 = (T)(g.lj_sigma * g.lj_sigma);
  const T lj_rc2 = (T)(1.2599210498948732 * g.lj_sigma * g.lj_sigma);   // (2^(1/6) sigma)^2
  const T lj_24e = (T)(24.0 * g.lj_eps), lj_4e = (T)(4.0 * g.lj_eps);
  const RsRec<T> far{(T)1e30, (T)1e30, (T)1e30, (T)0};
  double e_acc = 0.0;
  for (int i0 = hs + blockIdx.y * kRsThreads; i0 < he; i0 += gridDim.y * kRsThreads) {
    const int i = i0 + threadIdx.x;
    const bool live = i < he;
    const bool wlive = __ballot_sync(0xffffffffu, live) != 0u;   // warp-uniform
    RsRec<T> ri{(T)-1e30, (T)-1e30, (T)-1e30, (T)0};   // idle threads match nothing
    if (live) ri = rec[i];
    T ph = 0, fx = 0, fy = 0, fz = 0;
    T lx = 0, ly = 0, lz = 0, le = 0;       // LJ force and twice its energy share
    T vc[6] = {0, 0, 0, 0, 0, 0};           // sum_j q_j fr d_a d_b (VIR)
    T vl[6] = {0, 0, 0, 0, 0, 0};           // the same for the LJ pairs (VIR && LJ)
    for (int dz = -S; dz <= S; ++dz) {
      const int nz = cz + dz;
      if (nz < 0 || nz >= g.ncz) continue;
      for (int dy = -S; dy <= S; ++dy) {
        int ny = cy + dy;
        T sy = 0;
        if (ny < 0) { ny += g.ncy; sy = (T)(-g.Ly); }
        else if (ny >= g.ncy) { ny -= g.ncy; sy = (T)g.Ly; }
        const int row = (nz * g.ncy + ny) * g.ncx;
        // the row's cells [cx - S, cx + S] as up to two key ranges: records
        // [a0, a0 + n0) shifted by s0, then [a1, a1 + n1) shifted by s1
        const int lo = cx - S, hi = cx + S;
        int a0, n0, a1 = 0, n1 = 0;
        T s0 = 0, s1 = 0;
        if (lo < 0) {
          a0 = cstart[row + g.ncx + lo]; n0 = cstart[row + g.ncx] - a0; s0 = (T)(-g.Lx);
          a1 = cstart[row]; n1 = cstart[row + hi + 1] - a1;
        } else if (hi >= g.ncx) {
          a0 = cstart[row + lo]; n0 = cstart[row + g.ncx] - a0;
          a1 = cstart[row]; n1 = cstart[row + hi - g.ncx + 1] - a1; s1 = (T)g.Lx;
        } else {
          a0 = cstart[row + lo]; n0 = cstart[row + hi + 1] - a0;
        }
        const int nrow = n0 + n1;
        for (int b0 = 0; b0 < nrow; b0 += kRsRow) {
          const int cnt = min(kRsRow, nrow - b0);
          const int cpad = (cnt + 31) & ~31;
          __syncthreads();   // the previous records are no longer read
          for (int t = threadIdx.x; t < cpad; t += kRsThreads) {
            const int e = b0 + t;
            RsRec<T> rj = far;
            if (t < cnt) {
              if (e < n0) { rj = rec[a0 + e]; rj.x += s0; }
              else { rj = rec[a1 + (e - n0)]; rj.x += s1; }
              rj.y += sy;
            }
            buf[t] = rj;
          }
          __syncthreads();
          if (!wlive) continue;
          for (int t0 = 0; t0 < cpad; t0 += 32) {
            // phase 1: mark the records within rc; the particle itself
            // (r2 = 0) is left out (so would a distinct particle at the
            // same point be, whose pair energy is infinite)
            uint32_t m = 0u;
#pragma unroll
            for (int t = 0; t < 32; ++t) {
              const RsRec<T> rj = buf[t0 + t];
              const T ddx = ri.x - rj.x, ddy = ri.y - rj.y, ddz = ri.z - rj.z;
              const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
              m |= (r2 <= rc2 && r2 > (T)0) ? (1u << t) : 0u;
            }
            // phase 2: the pair terms of the marked records, two per step
            // (two independent dependency chains); an odd last record is
            // paired with itself at charge 0, which adds exact zeros
            while (m) {
              const int t1 = __ffs(m) - 1;
              m &= m - 1u;
              int t2 = t1;
              T qmul = (T)0;
              if (m) { t2 = __ffs(m) - 1; m &= m - 1u; qmul = (T)1; }
              const RsRec<T> rj1 = buf[t0 + t1];
              const RsRec<T> rj2 = buf[t0 + t2];
              const T dx1 = ri.x - rj1.x, dy1 = ri.y - rj1.y, dz1 = ri.z - rj1.z;
              const T dx2 = ri.x - rj2.x, dy2 = ri.y - rj2.y, dz2 = ri.z - rj2.z;
              const T r21 = dx1 * dx1 + dy1 * dy1 + dz1 * dz1;
              const T r22 = dx2 * dx2 + dy2 * dy2 + dz2 * dz2;
              const T inv1 = rs_rinv(r21), inv2 = rs_rinv(r22);
              const T r1 = r21 * inv1, r2b = r22 * inv2;
              T ec1, ex1, ec2, ex2;
              rs_erfc_exp(alpha * r1, a2 * r21, ec1, ex1);
              rs_erfc_exp(alpha * r2b, a2 * r22, ec2, ex2);
              const T e1 = ec1 * inv1, e2 = ec2 * inv2;
              const T fr1 = (e1 + two_a_sqpi * ex1) * inv1 * inv1;
              const T fr2 = (e2 + two_a_sqpi * ex2) * inv2 * inv2;
              const T q1 = rj1.q, q2 = rj2.q * qmul;
              ph = fma(q1, e1, ph);
              ph = fma(q2, e2, ph);
              const T w1 = q1 * fr1, w2 = q2 * fr2;
              fx = fma(w2, dx2, fma(w1, dx1, fx));
              fy = fma(w2, dy2, fma(w1, dy1, fy));
              fz = fma(w2, dz2, fma(w1, dz1, fz));
              if (VIR) {
                const T tx1 = w1 * dx1, ty1 = w1 * dy1, tz1 = w1 * dz1;
                const T tx2 = w2 * dx2, ty2 = w2 * dy2, tz2 = w2 * dz2;
                vc[0] = fma(tx2, dx2, fma(tx1, dx1, vc[0]));
                vc[1] = fma(ty2, dy2, fma(ty1, dy1, vc[1]));
                vc[2] = fma(tz2, dz2, fma(tz1, dz1, vc[2]));
                vc[3] = fma(tx2, dy2, fma(tx1, dy1, vc[3]));
                vc[4] = fma(tx2, dz2, fma(tx1, dz1, vc[4]));
                vc[5] = fma(ty2, dz2, fma(ty1, dz1, vc[5]));
              }
              if (LJ) {
                if (r21 < lj_rc2) {
                  const T s2 = lj_s2 / r21, s6 = s2 * s2 * s2;
                  const T f = lj_24e * (2 * s6 * s6 - s6) / r21;   // -(dU/dr)/r
                  lx = fma(f, dx1, lx); ly = fma(f, dy1, ly); lz = fma(f, dz1, lz);
                  le += lj_4e * (s6 * s6 - s6 + (T)0.25);
                  if (VIR) {
                    vl[0] = fma(f * dx1, dx1, vl[0]); vl[1] = fma(f * dy1, dy1, vl[1]);
                    vl[2] = fma(f * dz1, dz1, vl[2]); vl[3] = fma(f * dx1, dy1, vl[3]);
                    vl[4] = fma(f * dx1, dz1, vl[4]); vl[5] = fma(f * dy1, dz1, vl[5]);
                  }
                }
                if (qmul != (T)0 && r22 < lj_rc2) {
                  const T s2 = lj_s2 / r22, s6 = s2 * s2 * s2;
                  const T f = lj_24e * (2 * s6 * s6 - s6) / r22;
                  lx = fma(f, dx2, lx); ly = fma(f, dy2, ly); lz = fma(f, dz2, lz);
                  le += lj_4e * (s6 * s6 - s6 + (T)0.25);
                  if (VIR) {
                    vl[0] = fma(f * dx2, dx2, vl[0]); vl[1] = fma(f * dy2, dy2, vl[1]);
                    vl[2] = fma(f * dz2, dz2, vl[2]); vl[3] = fma(f * dx2, dy2, vl[3]);
                    vl[4] = fma(f * dx2, dz2, vl[4]); vl[5] = fma(f * dy2, dz2, vl[5]);
                  }
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
        force_out[3 * (int64_t)o] = fma(ri.q, fx, lx);
        force_out[3 * (int64_t)o + 1] = fma(ri.q, fy, ly);
        force_out[3 * (int64_t)o + 2] = fma(ri.q, fz, lz);
      }
      e_acc += 0.5 * (double)ri.q * (double)ph + 0.5 * (double)le;
      if (VIR)
        for (int k = 0; k < 6; ++k) v_acc[k] += 0.5 * ((double)ri.q * (double)vc[k] + (double)vl[k]);
    }
  }
  if (VIR) {
    for (int k = 0; k < 6; ++k) {
      double v = v_acc[k];
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) vred[k][threadIdx.x >> 5] = v;
    }
  }
  for (int o = 16; o; o >>= 1) e_acc += __shfl_xor_sync(0xffffffffu, e_acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e_acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kRsThreads / 32; ++w) s += red[w];
    ecell[(size_t)c * gridDim.y + blockIdx.y] = s;
    if (VIR) {
      // stored as xx, yy, zz, xy, xz, yz
      for (int k = 0; k < 6; ++k) {
        double t = 0.0;
        for (int w = 0; w < kRsThreads / 32; ++w) t += vred[k][w];
        vcell[((size_t)c * gridDim.y + blockIdx.y) * 6 + k] = t;
      }
    }
  }
}

// sum of the CTAs' virials in a fixed order (one CTA)
__global__ void rs_virial_kernel(int ncta, const double* vcell, double* virial) {
  __shared__ double red[6][32];
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int j = threadIdx.x; j < ncta; j += blockDim.x)
    for (int k = 0; k < 6; ++k) s[k] += vcell[(size_t)j * 6 + k];
  for (int k = 0; k < 6; ++k) {
    double v = s[k];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    virial[threadIdx.x] = t;
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

// CTAs per cell: about twice the mean occupancy over kRsThreads
static int rs_parts(const RsGrid& g) {
  const double ncell = (double)g.ncx * g.ncy * g.ncz;
  const double per = 2.0 * (double)g.N / ncell / kRsThreads;
  return (int)std::min(64.0, std::max(1.0, std::ceil(per)));
}

size_t rs_workspace_bytes(const RsGrid& g) {
  const int64_t ncell = (int64_t)g.ncx * g.ncy * g.ncz;
  auto a = [](size_t b) { return (b + 255) & ~size_t(255); };
  return a(sort_workspace_bytes(g.N, 4)) + a(4 * (size_t)(ncell + 1)) +
         a(8 * (size_t)ncell * rs_parts(g)) + a(sizeof(RsRec<double>) * (size_t)g.N) +
         a(6 * 8 * (size_t)ncell * rs_parts(g));
}

template <typename T>
int launch_realspace(const RsGrid& g, const T* pos, const T* q, void* ws, unsigned* status,
                     double* energy, T* phi, T* force, cudaStream_t st, double* virial) {
  const int64_t ncell = (int64_t)g.ncx * g.ncy * g.ncz;
  auto a = [](size_t b) { return (b + 255) & ~size_t(255); };
  char* p = static_cast<char*>(ws);
  SortWork sw;
  sort_bind_workspace(sw, p, g.N, 4);
  p += a(sort_workspace_bytes(g.N, 4));
  int32_t* cstart = reinterpret_cast<int32_t*>(p); p += a(4 * (size_t)(ncell + 1));
  const int parts = rs_parts(g);
  double* ecell = reinterpret_cast<double*>(p); p += a(8 * (size_t)ncell * parts);
  RsRec<T>* rec = reinterpret_cast<RsRec<T>*>(p);
  p += a(sizeof(RsRec<double>) * (size_t)g.N);
  double* vcell = reinterpret_cast<double*>(p);
  int blocks = (int)((g.N + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  rs_keys_kernel<T><<<blocks, 256, 0, st>>>(g, pos, q, static_cast<uint32_t*>(sw.keys[0]),
                                            sw.vals[0], status);
  int passes = 1;
  while (passes < 4 && (uint64_t)ncell > (1ull << (8 * passes))) ++passes;
  const int r = radix_sort(sw, g.N, 4, passes, 0, st);
  int cblocks = (int)((ncell + 1 + 255) / 256);
  if (cblocks > 152 * 16) cblocks = 152 * 16;
  rs_cells_kernel<<<cblocks, 256, 0, st>>>(g.N, ncell, static_cast<const uint32_t*>(sw.keys[r]),
                                           cstart);
  rs_gather_kernel<T><<<blocks, 256, 0, st>>>(g, pos, q, sw.vals[r], rec);
  const dim3 grid((unsigned)ncell, parts);
  if (virial) {
    if (g.lj_eps > 0.0)
      rs_pair_kernel<T, true, true><<<grid, kRsThreads, 0, st>>>(g, cstart, rec, sw.vals[r], phi,
                                                                 force, ecell, vcell);
    else
      rs_pair_kernel<T, false, true><<<grid, kRsThreads, 0, st>>>(g, cstart, rec, sw.vals[r], phi,
                                                                  force, ecell, vcell);
    rs_virial_kernel<<<1, 256, 0, st>>>((int)(ncell * parts), vcell, virial);
  } else if (g.lj_eps > 0.0) {
    rs_pair_kernel<T, true, false><<<grid, kRsThreads, 0, st>>>(g, cstart, rec, sw.vals[r], phi,
                                                                force, ecell, nullptr);
  } else {
    rs_pair_kernel<T, false, false><<<grid, kRsThreads, 0, st>>>(g, cstart, rec, sw.vals[r], phi,
                                                                 force, ecell, nullptr);
  }
  if (energy) rs_energy_kernel<<<1, 256, 0, st>>>((int)(ncell * parts), ecell, energy);
  return 3 + 3 * passes + (energy ? 2 : 1) + (virial ? 1 : 0);
}

template int launch_realspace<float>(const RsGrid&, const float*, const float*, void*, unsigned*,
                                     double*, float*, float*, cudaStream_t, double*);
template int launch_realspace<double>(const RsGrid&, const double*, const double*, void*,
                                      unsigned*, double*, double*, double*, cudaStream_t, double*);

}  // namespace qslab
