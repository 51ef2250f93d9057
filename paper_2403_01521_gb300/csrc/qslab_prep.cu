// qslab device kernels around the scans: input checks and sort keys, the
// sorted gather, the final combine with the energy reduction, and the mode
// tables (full k-sum list or the random-batch k-sampler).
#include <cstdint>
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "qslab_df.cuh"
#include "qslab_geom.cuh"
#include "qslab_internal.h"
#include "qslab_math.cuh"

namespace qslab {

namespace cg = cooperative_groups;

// ====================================================================== prep

template <typename T> struct KeyOf;
template <> struct KeyOf<float> {
  using type = uint32_t;
  __device__ static type key(float z) { return __float_as_uint(z == 0.0f ? 0.0f : z); }
};
template <> struct KeyOf<double> {
  using type = uint64_t;
  __device__ static type key(double z) {
    return (uint64_t)__double_as_longlong(z == 0.0 ? 0.0 : z);
  }
};

__device__ __forceinline__ double shfl_xor_cn(double v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}
__device__ __forceinline__ DF shfl_xor_cn(DF v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// One CTA per k-space chunk (chunks are contiguous in the caller's order as
// well): finiteness and z-range checks, the z keys, the replica index and
// the chunk's sums of q and |q| (csums[2c], csums[2c+1]; summed per replica
// in a fixed order by the neutrality check).
template <typename T>
__global__ void prepare_kernel(Reps rp, const T* __restrict__ pos, const T* __restrict__ q,
                               typename KeyOf<T>::type* keys, uint32_t* vals, int32_t* rid,
                               double* sums, unsigned* status) {
  __shared__ double red[2][32];
  const CRange ch = kchunk(rp, blockIdx.x);
  if (!QS_DCHECK(chunk_ok(rp, ch, rp.L), rp.status)) return;
  const double Lz = rp.info[ch.r].Lz;
  // the largest T not above Lz: z <= Lz exactly when z <= Lzlo
  T Lzlo = (T)Lz;
  if ((double)Lzlo > Lz) Lzlo = nextafter(Lzlo, (T)0);
  // the sums in the carry type: FP64, or double-float on the FP32 path
  // (whose FP32 charges sum exactly enough in it, without FP64 operations)
  using CN = typename CarryNum<T>::type;
  CN sq = cn_zero((CN*)nullptr), sa = sq;
  unsigned flags = 0;
  for (int t = threadIdx.x; t < ch.cnt; t += blockDim.x) {
    const int64_t i = ch.start + t;
    const T x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2], qi = q[i];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(qi)) flags |= kStNonfinite;
    else if (!(z >= (T)0) || !(z <= Lzlo)) flags |= kStZRange;
    keys[i] = KeyOf<T>::key(z);
    vals[i] = (uint32_t)i;
    if (rid) rid[i] = ch.r;
    sq = sq + qi;
    sa = sa + (T)fabs(qi);
  }
  if (flags) atomicOr(status, flags);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o; o >>= 1) {
    sq = sq + shfl_xor_cn(sq, o);
    sa = sa + shfl_xor_cn(sa, o);
  }
  if (lane == 0) { red[0][w] = cn_to_double(sq); red[1][w] = cn_to_double(sa); }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) { a += red[0][j]; b += red[1][j]; }
    sums[2 * blockIdx.x] = a;
    sums[2 * blockIdx.x + 1] = b;
  }
}

template <typename T>
void launch_prepare(const Reps& rp, const T* pos, const T* q, void* keys, uint32_t* vals,
                    int32_t* rid, double* sums, unsigned* status, cudaStream_t st) {
  prepare_kernel<T><<<rp.nchunks, chunk_threads(rp.L), 0, st>>>(
      rp, pos, q, static_cast<typename KeyOf<T>::type*>(keys), vals, rid, sums, status);
}

// One CTA per replica: the replica's sums of q and |q| from its chunks'
// partial sums (a fixed order), then the neutrality check.
__global__ void check_neutral_kernel(Reps rp, const double* sums, double tol, double sb0,
                                     double st0, unsigned* status, uint64_t* ctr) {
  __shared__ double red[2][32];
  const int r = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (ctr && r == 0 && threadIdx.x == 0) {
    const uint64_t c = ctr[0];
    ctr[1] = c;
    ctr[0] = c + 1;
  }
  const RepInfo& ri = rp.info[r];
  double sq = 0.0, sa = 0.0;
  for (int j = threadIdx.x; j < ri.nch; j += blockDim.x) {
    sq += sums[2 * (ri.c0 + j)];
    sa += sums[2 * (ri.c0 + j) + 1];
  }
  for (int o = 16; o; o >>= 1) {
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
  }
  if (lane == 0) { red[0][w] = sq; red[1][w] = sa; }
  __syncthreads();
  if (threadIdx.x == 0 && tol >= 0.0) {
    double a = 0.0, b = 0.0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) { a += red[0][j]; b += red[1][j]; }
    // particles and walls together (the neutrality condition of Section 2.4)
    const double ar = ri.area;
    const double net = a + ar * (sb0 + st0);
    const double mag = b + ar * (fabs(sb0) + fabs(st0));
    if (fabs(net) > tol * mag) atomicOr(status, kStNonneutral);
  }
}

void launch_check_neutral(const Reps& rp, const double* sums, double tol, double sb0,
                          double st0, unsigned* status, uint64_t* ctr, cudaStream_t st) {
  check_neutral_kernel<<<rp.R, 256, 0, st>>>(rp, sums, tol, sb0, st0, status, ctr);
}

__global__ void rep_keys_kernel(int64_t N, const uint32_t* __restrict__ perm,
                                const int32_t* __restrict__ rid, uint32_t* keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    keys[i] = (uint32_t)rid[perm[i] < (uint64_t)N ? perm[i] : 0];   // clamped as in the gather
}

void launch_rep_keys(int64_t N, const uint32_t* perm, const int32_t* rid, uint32_t* keys,
                     cudaStream_t st) {
  int blocks = (int)((N + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  rep_keys_kernel<<<blocks, 256, 0, st>>>(N, perm, rid, keys);
}

// ==================================================================== gather

// Fixed-point fraction x/L of a turn: floor(x 2^32/L) mod 2^32 (FP32 path,
// from the FP64 product with the scale k = 2^32/L and a round-down
// conversion) or frac(x/L) 2^64 (FP64 path, with ik = 1/L). One product per
// coordinate instead of an FP64 division.
__device__ __forceinline__ uint32_t to_fixed(float x, double k, double) {
  return (uint32_t)(uint64_t)__double2ll_rd((double)x * k);
}
__device__ __forceinline__ uint64_t to_fixed(double x, double, double ik) {
  double f = x * ik;
  f -= floor(f);
  if (!(f < 1.0)) f = 0.0;
  return (uint64_t)(f * 18446744073709551616.0);
}

template <typename T> struct KeyVal;
template <> struct KeyVal<float> {
  __device__ static float z(const void* keys, int64_t i) {
    return __uint_as_float(static_cast<const uint32_t*>(keys)[i]);
  }
};
template <> struct KeyVal<double> {
  __device__ static double z(const void* keys, int64_t i) {
    return __longlong_as_double((long long)static_cast<const uint64_t*>(keys)[i]);
  }
};

// One CTA per k-space chunk: the sorted SoA arrays, with dz = 0 at the first
// particle of every replica. zkeys (may be NULL): the sorted z keys of a
// single-slab call (the z values' own bits), read in order instead of
// gathering z from the positions.
template <typename T>
__global__ void gather_kernel(Reps rp, const T* __restrict__ pos, const T* __restrict__ q,
                              const uint32_t* __restrict__ perm, const void* zkeys, T* zs, T* dz,
                              T* qs, typename PhaseT<T>::type* xh, typename PhaseT<T>::type* yh,
                              int32_t* perm_out) {
  const CRange ch = kchunk(rp, blockIdx.x);
  if (!QS_DCHECK(chunk_ok(rp, ch, rp.L), rp.status)) return;
  const double Lx = rp.info[ch.r].Lx, Ly = rp.info[ch.r].Ly;
  const double kx = 4294967296.0 / Lx, ky = 4294967296.0 / Ly;   // FP32 path
  const double ikx = 1.0 / Lx, iky = 1.0 / Ly;                     // FP64 path
  for (int t = threadIdx.x; t < ch.cnt; t += blockDim.x) {
    const int64_t i = ch.start + t;
    uint32_t o = perm[i];
    if (!QS_DCHECK(o < (uint64_t)rp.N, rp.status)) continue;
    // a sort whose bounded wait gave up (status TIMEOUT) leaves indices
    // that may be out of range: clamp, so that the call stays in bounds
    if (o >= (uint64_t)rp.N) o = 0;
    const bool first = t == 0 && ch.first;
    T z, zp;
    if (zkeys) {
      z = KeyVal<T>::z(zkeys, i);
      zp = first ? z : KeyVal<T>::z(zkeys, i - 1);
    } else {
      z = pos[3 * (int64_t)o + 2];
      uint32_t op = first ? o : perm[i - 1];
      if (op >= (uint64_t)rp.N) op = 0;
      zp = first ? z : pos[3 * (int64_t)op + 2];
    }
    zs[i] = z;
    dz[i] = first ? (T)0 : z - zp;
    qs[i] = q[o];
    xh[i] = to_fixed(pos[3 * (int64_t)o], kx, ikx);
    yh[i] = to_fixed(pos[3 * (int64_t)o + 1], ky, iky);
    perm_out[i] = (int32_t)o;
  }
}

template <typename T>
void launch_gather(const Reps& rp, const T* pos, const T* q, const uint32_t* perm,
                   const void* zkeys, T* zs, T* dz, T* qs, typename PhaseT<T>::type* xh,
                   typename PhaseT<T>::type* yh, int32_t* perm_out, cudaStream_t st) {
  gather_kernel<T><<<rp.nchunks, chunk_threads(rp.L), 0, st>>>(rp, pos, q, perm, zkeys, zs, dz,
                                                                qs, xh, yh, perm_out);
}

// ================================================================== combine

// One CTA per k-space chunk: sums the mode ranges' partial outputs, adds the
// k = 0 term and the j = i constant of the chunk's replica, and with walls
// the particle-slab potential (Thm 2.4); scatters the potential and force to
// the caller's order and writes the chunk's energy
// sum_i q_i (phi_p-p,i / 2 + phi_p-s,i).
//
// Walls: phi_p-s = -2 pi [sb0 z + st0 (Lz - z)]
//                  + sum_w Re[e^{i k_w.rho} (Cb_w e^{-k z} + Ct_w e^{-k (Lz - z)})]
// with Cb_w = 4 pi c_bot,w / k (the 2 pi/(A k) of Thm 2.4, times A c_w for
// the cell integral, times 2 for the pair (m, -m)); F = -q grad phi_p-s.
template <typename T>
__global__ void combine_kernel(Reps rp, int nkr, const T* __restrict__ part,
                               const typename CarryNum<T>::type* __restrict__ phi0,
                               const typename CarryNum<T>::type* __restrict__ fz0,
                               const T* __restrict__ qs, const T* __restrict__ zs,
                               const typename PhaseT<T>::type* __restrict__ xh,
                               const typename PhaseT<T>::type* __restrict__ yh,
                               const __grid_constant__ WallTab W,
                               const int32_t* __restrict__ perm,
                               double* echunk, T* phi_out, T* force_out) {
  using PH = typename PhaseT<T>::type;
  __shared__ double red[32];
  // per-mode constants of this chunk's box: kx, ky, k, Cb (re, im), Ct (re, im)
  __shared__ T wk[kMaxWallModes][7];
  const CRange ch = kchunk(rp, blockIdx.x);
  if (!QS_DCHECK(chunk_ok(rp, ch, rp.L), rp.status)) return;
  const RepInfo& ri = rp.info[ch.r];
  const double diagq = ri.diagq;
  const double Lz = ri.Lz;
  const int nw = W.on ? W.nw : 0;
  for (int w = threadIdx.x; w < nw; w += blockDim.x) {
    const double kx = 6.283185307179586 * W.m[w][0] / ri.Lx;
    const double ky = 6.283185307179586 * W.m[w][1] / ri.Ly;
    const double k = sqrt(kx * kx + ky * ky);
    const double f = 12.566370614359172 / k;   // 4 pi / k
    wk[w][0] = (T)kx; wk[w][1] = (T)ky; wk[w][2] = (T)k;
    wk[w][3] = (T)(f * W.c[w][0]); wk[w][4] = (T)(f * W.c[w][1]);
    wk[w][5] = (T)(f * W.c[w][2]); wk[w][6] = (T)(f * W.c[w][3]);
  }
  __syncthreads();
  const int64_t N = rp.N;
  if constexpr (sizeof(T) == 4) {
    if (!W.on) {
      // FP32 path without walls: the sums in double-float (FP64 runs at
      // 1/76 of FP32 on this part), each output rounded once from them
      const DF dq = df_from(diagq);
      DF e2 = {0.0f, 0.0f};
      for (int t = threadIdx.x; t < ch.cnt; t += blockDim.x) {
        const int64_t i = ch.start + t;
        DF sp = {0.0f, 0.0f}, sx = sp, sy = sp, sz = sp;
        for (int r = 0; r < nkr; ++r) {
          const T* b = part + (size_t)r * 4 * N;
          sp = sp + (float)b[i];
          sx = sx + (float)b[N + i];
          sy = sy + (float)b[2 * N + i];
          sz = sz + (float)b[3 * N + i];
        }
        const float qq = (float)qs[i];
        const DF q2 = df_from(qq);
        const DF ph = sp + reinterpret_cast<const DF*>(phi0)[i] + q2 * dq;
        const DF fz = sz * q2 + reinterpret_cast<const DF*>(fz0)[i];
        const int32_t o = perm[i];
        if (!QS_DCHECK(o >= 0 && o < rp.N, rp.status)) continue;
        if (phi_out) phi_out[o] = (T)df_to_float(ph);
        if (force_out) {
          force_out[3 * (int64_t)o] = (T)df_to_float(sx * q2);
          force_out[3 * (int64_t)o + 1] = (T)df_to_float(sy * q2);
          force_out[3 * (int64_t)o + 2] = (T)df_to_float(fz);
        }
        const DF qp = q2 * ph;
        e2 = e2 + DF{0.5f * qp.hi, 0.5f * qp.lo};
      }
      for (int o = 16; o; o >>= 1)
        e2 = e2 + DF{__shfl_xor_sync(0xffffffffu, e2.hi, o), __shfl_xor_sync(0xffffffffu, e2.lo, o)};
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = df_to_double(e2);
      __syncthreads();
      if (threadIdx.x == 0) {
        double s = 0;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) s += red[j];
        echunk[blockIdx.x] = s;
      }
      return;
    }
  }
  double e = 0.0;
  for (int t = threadIdx.x; t < ch.cnt; t += blockDim.x) {
    const int64_t i = ch.start + t;
    double ph = 0, fx = 0, fy = 0, fz = 0;
    for (int r = 0; r < nkr; ++r) {
      const T* b = part + (size_t)r * 4 * N;
      ph += (double)b[i];
      fx += (double)b[N + i];
      fy += (double)b[2 * N + i];
      fz += (double)b[3 * N + i];
    }
    const double qq = (double)qs[i];
    ph += cn_to_double(phi0[i]) + qq * diagq;
    fx *= qq; fy *= qq;
    fz = fz * qq + cn_to_double(fz0[i]);
    double pw = 0.0;
    if (W.on) {
      const double z = (double)zs[i];
      pw = -6.283185307179586 * (W.sb0 * z + W.st0 * (Lz - z));
      double gz = 6.283185307179586 * (W.sb0 - W.st0);   // field along z
      T pm = 0, gx = 0, gy = 0, gzm = 0;
      if (nw) {
        const T zb = (T)z, zt = (T)(Lz - z);
        const PH px = xh[i], py = yh[i];
        for (int w = 0; w < nw; ++w) {
          T cs, sn;
          sincos_turns((PH)((PH)(int64_t)W.m[w][0] * px + (PH)(int64_t)W.m[w][1] * py), cs, sn);
          const T k = wk[w][2];
          const T eb = exp_neg(k * zb), et = exp_neg(k * zt);
          const T ar = wk[w][3] * eb + wk[w][5] * et;    // Cb e^{-k z} + Ct e^{-k (Lz - z)}
          const T ai = wk[w][4] * eb + wk[w][6] * et;
          const T br = k * (wk[w][5] * et - wk[w][3] * eb);   // its z-derivative
          const T bi = k * (wk[w][6] * et - wk[w][4] * eb);
          pm += cs * ar - sn * ai;                        // Re[e^{i k.rho} a]
          const T im = sn * ar + cs * ai;                 // Im[e^{i k.rho} a]
          gx += wk[w][0] * im;                            // -d/dx of Re[...]
          gy += wk[w][1] * im;
          gzm -= cs * br - sn * bi;                       // -d/dz of Re[...]
        }
      }
      pw += (double)pm;
      gz += (double)gzm;
      fx += qq * (double)gx;
      fy += qq * (double)gy;
      fz += qq * gz;
    }
    const int32_t o = perm[i];
    if (!QS_DCHECK(o >= 0 && o < rp.N, rp.status)) continue;
    if (phi_out) phi_out[o] = (T)(ph + pw);
    if (force_out) {
      force_out[3 * (int64_t)o] = (T)fx;
      force_out[3 * (int64_t)o + 1] = (T)fy;
      force_out[3 * (int64_t)o + 2] = (T)fz;
    }
    e += qq * (0.5 * ph + pw);
  }
  for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) s += red[j];
    echunk[blockIdx.x] = s;
  }
}

// One warp per replica: the sum of its chunks' energies in a fixed order
// (deterministic).
__global__ void energy_rep_kernel(Reps rp, const double* echunk, double* energies) {
  const int rep = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (rep >= rp.R) return;   // whole warps leave together
  const RepInfo& ri = rp.info[rep];
  double s = 0.0;
  for (int j = lane; j < ri.nch; j += 32) s += echunk[ri.c0 + j];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) energies[rep] = s;
}

template <typename T>
void launch_combine(const Reps& rp, int nkr, const T* part, const void* phi0v,
                    const void* fz0v, const T* qs, const T* zs,
                    const typename PhaseT<T>::type* xh, const typename PhaseT<T>::type* yh,
                    const WallTab& W, const int32_t* perm, double* echunk,
                    T* phi_out, T* force_out, double* energies, cudaStream_t st) {
  using CN = typename CarryNum<T>::type;
  const CN* phi0 = static_cast<const CN*>(phi0v);
  const CN* fz0 = static_cast<const CN*>(fz0v);
  combine_kernel<T><<<rp.nchunks, chunk_threads(rp.L), 0, st>>>(
      rp, nkr, part, phi0, fz0, qs, zs, xh, yh, W, perm, echunk, phi_out, force_out);
  if (energies) {
    const int64_t thr = (int64_t)rp.R * 32;
    energy_rep_kernel<<<(unsigned)((thr + 255) / 256), 256, 0, st>>>(rp, echunk, energies);
  }
}

// ========================================================= random-batch modes

__device__ int upper_index(const double* cdf, int n, double u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (u < cdf[mid]) hi = mid; else lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ double uniform53(uint64_t w) {
  return (double)(w >> 11) * 1.1102230246251565e-16;   // 2^-53
}

// Fill the mode tables, per (mode, replica). Full k-sum: (mx, my) from
// the replica's half-plane list, weight 2 (k and -k), gam = (pi/A) C_k 2.
// Random batch: (mx, my) drawn here (Philox4x64-10 with counter
// (m, attempt, call, tag + replica * 2^32) and key (seed, 0); words 0,1 then
// 2,3 are inverted through the replica's per-axis cumulative tables; the
// origin is rejected), gam = (pi/A) (H/P) 2 alpha/(sqrt(pi) k) (Eq. 4.7 with
// 4.9: the Gaussian of C_k cancels against e^{k^2/(4 alpha^2)}).
// A group of G lanes serves one mode: every lane finds the mode and its
// constants (the same values), lane g takes pairs g, g + G, ..., and the
// group sums the pair terms with shuffles, so that each warp issues a few
// pairs' FP64 work instead of all of them.
template <typename T, int G>
__global__ void __launch_bounds__(64) mode_coef_kernel(Reps rp, int npc, const int32_t* list,
                                                       int rbe, uint64_t seed, const uint64_t* ctr,
                                                       const double* cdf, PairTab pr, double alpha,
                                                       ModeTab<T> mt, int32_t* sampled) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = tid / G, g = tid % G;
  const int rep = blockIdx.y;
  const int Kpad = rp.Kpad;
  if (m >= Kpad) return;                  // whole groups: Kpad G is a multiple of the block
  const unsigned gmask = (G == 32 ? 0xffffffffu : ((1u << G) - 1u)) << ((threadIdx.x & 31) & ~(G - 1));
  const RepInfo& ri = rp.info[rep];
  const int K = ri.K;
  const double Lx = ri.Lx, Ly = ri.Ly;
  const size_t mg = (size_t)rep * Kpad + m;
  const size_t ks = (size_t)rp.R * Kpad;
  const double pi = 3.14159265358979323846;
  const double sqpi = 1.7724538509055160;
  int mx = 0, my = 0;
  if (m < K) {
    if (rbe == 0) {
      mx = list[2 * ((size_t)ri.list0 + m)];
      my = list[2 * ((size_t)ri.list0 + m) + 1];
    } else if (rbe == 2) {
      mx = sampled[2 * ((size_t)rep * K + m)];
      my = sampled[2 * ((size_t)rep * K + m) + 1];
    } else {
      const double* cdfx = cdf + ri.cdfx0;
      const double* cdfy = cdf + ri.cdfy0;
      const uint64_t counter = ctr[1];
      for (uint64_t attempt = 0; attempt < 64; ++attempt) {
        U64x4 c;
        c.v[0] = (uint64_t)m; c.v[1] = attempt; c.v[2] = counter;
        c.v[3] = 0x52424531ull + ((uint64_t)rep << 32);
        const U64x4 r = philox4x64_10(c, seed, 0ull);
        const int ax = upper_index(cdfx, ri.nx, uniform53(r.v[0])) - ri.mxmax;
        const int ay = upper_index(cdfy, ri.ny, uniform53(r.v[1])) - ri.mymax;
        if (ax != 0 || ay != 0) { mx = ax; my = ay; break; }
        const int bx = upper_index(cdfx, ri.nx, uniform53(r.v[2])) - ri.mxmax;
        const int by = upper_index(cdfy, ri.ny, uniform53(r.v[3])) - ri.mymax;
        if (bx != 0 || by != 0) { mx = bx; my = by; break; }
      }
      if (sampled && g == 0) {
        sampled[2 * ((size_t)rep * K + m)] = mx;
        sampled[2 * ((size_t)rep * K + m) + 1] = my;
      }
    }
  }
  const bool live = (m < K) && (mx != 0 || my != 0);
  const double kx = 2 * pi * mx / Lx, ky = 2 * pi * my / Ly;
  const double k = live ? sqrt(kx * kx + ky * ky) : 1.0;
  double gam = 0.0;
  if (live) {
    gam = rbe ? pi / (Lx * Ly) * (ri.H / K) * 2.0 * alpha / (sqpi * k)
              : pi / (Lx * Ly) * 2.0 * (2.0 * alpha * exp(-k * k / (4.0 * alpha * alpha)) / (sqpi * k));
  }
  double ckk = 0.0, sY = 0.0, sZ = 0.0;
  for (int p = g; p < npc; p += G) {
    double cr = 0, ci = 0, br = 0, bi = 0;
    if (p < pr.np) {
      const double ar = pr.a_re[p], ai = pr.a_im[p];
      const double wr = pr.w_re[p], wi = pr.w_im[p];
      const double dr = ar * ar - ai * ai - k * k, di = 2 * ar * ai;   // a^2 - k^2
      const double rdd = 1.0 / (dr * dr + di * di);
      const double qr = (wr * dr + wi * di) * rdd, qi = (wi * dr - wr * di) * rdd;  // w/(a^2-k^2)
      ckk += pr.mult[p] * 2.0 * (ar * qr - ai * qi);     // sum over both nodes of 2 a w/(a^2-k^2)
      cr = -2.0 * k * qr * pr.mult[p] * gam;             // m_p gam c_{k,p}
      ci = -2.0 * k * qi * pr.mult[p] * gam;
      br = cr * ar - ci * ai;                            // times a_p
      bi = cr * ai + ci * ar;
      // the kernels remove the j = i term with sY and sZ; summing the
      // coefficients as the kernels see them (rounded to T) makes that
      // removal exact up to one rounding of sY (rounded one by one, the
      // mismatch would leave a bias of q_i^2 times it in every potential)
      sY += (double)(T)cr;
      sZ += (double)(T)br;
    }
    mt.cp[((size_t)0 * npc + p) * ks + mg] = (T)cr;
    mt.cp[((size_t)1 * npc + p) * ks + mg] = (T)ci;
    mt.cp[((size_t)2 * npc + p) * ks + mg] = (T)br;
    mt.cp[((size_t)3 * npc + p) * ks + mg] = (T)bi;
  }
  for (int o = G >> 1; o; o >>= 1) {
    ckk += __shfl_xor_sync(gmask, ckk, o, G);
    sY += __shfl_xor_sync(gmask, sY, o, G);
    sZ += __shfl_xor_sync(gmask, sZ, o, G);
  }
  if (g != 0) return;
  const double ck = gam * ckk;
  mt.mx[mg] = mx;
  mt.my[mg] = my;
  mt.kx[mg] = (T)kx;
  mt.ky[mg] = (T)ky;
  mt.kk[mg] = (T)k;
  mt.ck[mg] = (T)ck;
  mt.ckk[mg] = (T)(ck * k);
  mt.sY[mg] = (T)((double)(T)ck + sY);
  mt.sZ[mg] = (T)((double)(T)(ck * k) + sZ);
}

// ================================================= Metropolis k-sampler

constexpr int kMhBlock = 1024;          // chain steps prepared per round
constexpr int kMhWin = 8;               // earlier states with precomputed decisions
constexpr int kMhCluster = 8;           // CTAs per replica drawing the proposals
constexpr int kMhThreads = 512;         // 4 roles x 4 groups of 32 lanes
constexpr int kMhSlots = 128;           // items per pass of the role warps
static_assert(kMhBlock <= kMhSlots * kMhCluster, "one pass covers a CTA's proposals");
constexpr uint64_t kMhTag = 0x4D484731ull;

// One proposal of App. G from two words: Box-Muller normals (u1 = 1 -
// uniform53(w0) in (0, 1], u2 = uniform53(w1)) scaled by the standard
// deviations alpha L/(sqrt(2) pi), rounded half away from zero. The three
// pieces are separate so that different warps can compute them.
__device__ __forceinline__ double mh_radius(uint64_t w0) {
  const double u1 = 1.0 - uniform53(w0);
  return sqrt(-2.0 * log(u1));
}
__device__ __forceinline__ double mh_angle(uint64_t w1) {
  return 2.0 * 3.14159265358979323846 * uniform53(w1);
}
__device__ __forceinline__ void mh_round(double sdx, double sdy, double r, double c, double s,
                                         int& mx, int& my) {
  mx = (int)round(sdx * r * c);
  my = (int)round(sdy * r * s);
}
__device__ __forceinline__ void mh_propose(uint64_t w0, uint64_t w1, double sdx, double sdy,
                                           int& mx, int& my) {
  const double r = mh_radius(w0), th = mh_angle(w1);
  mh_round(sdx, sdy, r, cos(th), sin(th), mx, my);
}

// log[H(m)/q(m)] from the replica's per-axis tables. A Box-Muller normal is
// at most sqrt(2 * 53 ln 2) < 8.58 standard deviations from 0, so |m| stays
// within the tables' range 6.438 alpha L / pi + 1; the clamp only guards
// the memory access.
__device__ __forceinline__ double mh_log_weight(const double* lwx, const double* lwy,
                                                int mxmax, int mymax, int mx, int my) {
  const int ix = min(max(mx, -mxmax), mxmax) + mxmax;
  const int iy = min(max(my, -mymax), mymax) + mymax;
  return lwx[ix] + lwy[iy];
}

// The chain within a round after its first acceptance, as a scan. With the
// decision bits of the kMhWin states before each step, the state after step
// t is t - o(t) for an offset o in 0..kMhWin - 1, or kMhWin steps back
// (o = kMhFar), and step t maps o(t - 1) to o(t): 0 when the step accepts
// from offset o(t - 1) (bit o(t - 1) of its decisions), o(t - 1) + 1 when it
// rejects (always for the origin); kMhFar stays kMhFar, where the decision
// needs the FP64 test (the state is kMhWin or more steps back). A step is a
// map on the kMhWin + 1 offsets, packed as nibbles, and the maps compose
// associatively, so a block-wide scan gives every step's offset.
constexpr int kMhFar = kMhWin;
using MhMap = unsigned long long;
constexpr MhMap kMhId = 0x876543210ull;
static_assert(kMhWin == 8, "nine nibbles");
__device__ __forceinline__ int mh_at(MhMap f, int o) { return (int)((f >> (4 * o)) & 0xFull); }
__device__ __forceinline__ MhMap mh_then(MhMap f, MhMap g) {   // f first, then g
  MhMap h = 0;
#pragma unroll
  for (int o = 0; o <= kMhFar; ++o) h |= (MhMap)mh_at(g, mh_at(f, o)) << (4 * o);
  return h;
}
__device__ __forceinline__ MhMap mh_step_map(bool origin, unsigned bits) {
  MhMap f = (MhMap)kMhFar << (4 * kMhFar);
#pragma unroll
  for (int o = 0; o < kMhFar; ++o) {
    const int out = (!origin && ((bits >> o) & 1u)) ? 0 : o + 1;
    f |= (MhMap)out << (4 * o);
  }
  return f;
}
// keep the state after chain step `step` (0-based) when step + 1 is a
// multiple of thin, as output (step + 1) / thin - 1 of the replica
__device__ __forceinline__ void mh_keep(int64_t step, int thin, int rep, int P, int x, int y,
                                        int32_t* sampled) {
  const int64_t eta = step + 1;
  if (thin == 1 || eta % thin == 0) {
    const size_t j = (size_t)rep * P + (size_t)(eta / thin - 1);
    sampled[2 * j] = x;
    sampled[2 * j + 1] = y;
  }
}

// One cluster of kMhCluster CTAs per replica. The proposals do not depend
// on the chain's state (App. G), so all CTAs of the cluster draw kMhBlock of
// them at a time (proposal, its log-weight and log u; CTA r takes steps
// r, r + kMhCluster, ...) straight into the shared memory of the cluster's
// first CTA. Within a CTA the FP64 work of a proposal is split by role over
// warps that sit on different SM sub-partitions (warp w has role w mod 4):
// role 0 the radius sqrt(-2 ln u1), role 1 cos and sin of the angle, role 2
// log u; a combine step then rounds the normals and looks up the weights.
// The first CTA also draws the start attempt 0's two candidates this way.
// After a cluster barrier the first CTA runs the chain: the origin is
// rejected (h = 0 there), any other proposal accepted when d >= 0 or
// log u < d, d the log acceptance ratio. The chain's state is always an
// earlier proposal of the round (or the state it entered the round with),
// so the CTA first decides in parallel, for every step t and each of the
// kMhWin steps j before it, whether t would be accepted from state j (the
// same FP64 operations with lw = log-weight of j). Thread 0 fixes the start
// state (searching attempts 1..63 itself only if both candidates are the
// origin) and takes the steps up to the round's first acceptance; the
// states after it come from a block scan of the steps' offset maps (see
// mh_step_map), and thread 0 decides step by step again only after kMhWin
// rejections in a row.
// Counters: start attempts (a, 1, ctr[1], tag + rep 2^32), steps
// (eta - 1, 0, ctr[1], tag + rep 2^32), key (seed, 0).
__global__ void __cluster_dims__(kMhCluster, 1, 1) __launch_bounds__(kMhThreads)
mh_chain_kernel(Reps rp, int P, int thin, uint64_t seed, const uint64_t* ctr, const double* cdf,
                double alpha, int32_t* sampled) {
  __shared__ int32_t spx[kMhBlock], spy[kMhBlock];
  __shared__ double slw[kMhBlock], slu[kMhBlock];
  __shared__ uint8_t sacc[kMhBlock];      // bit w: accepted from state t - 1 - w
  __shared__ double ir[kMhSlots], ic[kMhSlots], isn[kMhSlots], iu[kMhSlots];
  __shared__ int32_t cand[2][2];          // start attempt 0's candidates (first CTA)
  __shared__ MhMap s_wmap[kMhThreads / 32], s_wpre[kMhThreads / 32];
  __shared__ int s_ta, s_tf, s_end;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const bool lead = rank == 0;
  // the first CTA's arrays, which every CTA of the cluster fills
  int32_t* lpx = cluster.map_shared_rank(spx, 0);
  int32_t* lpy = cluster.map_shared_rank(spy, 0);
  double* llw = cluster.map_shared_rank(slw, 0);
  double* llu = cluster.map_shared_rank(slu, 0);
  const int rep = blockIdx.x / kMhCluster;
  const RepInfo& ri = rp.info[rep];
  const double pi = 3.14159265358979323846;
  const double sdx = alpha * ri.Lx / (sqrt(2.0) * pi);
  const double sdy = alpha * ri.Ly / (sqrt(2.0) * pi);
  const double* lwx = cdf + ri.cdfx0 + ri.nx + ri.ny;
  const double* lwy = cdf + ri.cdfy0 + ri.nx + ri.ny;
  const uint64_t counter = ctr[1];
  const uint64_t tag = kMhTag + ((uint64_t)rep << 32);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int role = warp & 3, slot = (warp >> 2) * 32 + lane;
  int cx = 1, cy = 0;         // chain state (thread 0 of the first CTA)
  double lw = 0.0;
  const int64_t n = (int64_t)P * thin;
  for (int64_t b0 = 0; b0 < n; b0 += kMhBlock) {
    const int cnt = (int)min((int64_t)kMhBlock, n - b0);
    // the first CTA has finished the previous round's chain
    if (b0 > 0) cluster.sync();
    // items: this CTA's proposals t = rank + kMhCluster i, then (first CTA,
    // first round) the two start candidates
    const int m = cnt > rank ? (cnt - rank + kMhCluster - 1) / kMhCluster : 0;
    const int items = m + (lead && b0 == 0 ? 2 : 0);
    for (int i0 = 0; i0 < items; i0 += kMhSlots) {
      const int i = i0 + slot;
      if (i < items && role < 3) {
        U64x4 c;
        if (i < m) { c.v[0] = (uint64_t)(b0 + rank + kMhCluster * i); c.v[1] = 0; }
        else { c.v[0] = 0; c.v[1] = 1; }
        c.v[2] = counter; c.v[3] = tag;
        const U64x4 w = philox4x64_10(c, seed, 0ull);
        const bool second = i >= m && i - m == 1;      // words 2, 3 of attempt 0
        const uint64_t w0 = second ? w.v[2] : w.v[0], w1 = second ? w.v[3] : w.v[1];
        if (role == 0) {
          ir[slot] = mh_radius(w0);
        } else if (role == 1) {
          const double th = mh_angle(w1);
          ic[slot] = cos(th);
          isn[slot] = sin(th);
        } else if (i < m) {
          iu[slot] = log(uniform53(w.v[2]));     // -inf for u = 0
        }
      }
      __syncthreads();
      if (threadIdx.x < kMhSlots && i0 + (int)threadIdx.x < items) {
        const int j = threadIdx.x, it = i0 + j;
        int px, py;
        mh_round(sdx, sdy, ir[j], ic[j], isn[j], px, py);
        if (it < m) {
          const int t = rank + kMhCluster * it;
          lpx[t] = px;
          lpy[t] = py;
          llw[t] = mh_log_weight(lwx, lwy, ri.mxmax, ri.mymax, px, py);
          llu[t] = iu[j];
        } else {
          cand[it - m][0] = px;
          cand[it - m][1] = py;
        }
      }
      __syncthreads();
    }
    cluster.sync();             // the round's proposals are in the first CTA
    if (!lead) continue;
    // decisions from the kMhWin states before each step: groups of kMhWin
    // lanes per step, one ballot per warp (the loop bound is warp-uniform)
    for (int e0 = 0; e0 < cnt * kMhWin; e0 += blockDim.x) {
      const int e = e0 + threadIdx.x;
      const int t = e / kMhWin, j = t - 1 - e % kMhWin;
      bool acc = false;
      if (e < cnt * kMhWin && j >= 0) {
        const double d = slw[t] - slw[j];
        acc = d >= 0.0 || slu[t] < d;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, acc);
      if (e < cnt * kMhWin && lane % kMhWin == 0)
        sacc[t] = (uint8_t)((bal >> lane) & ((1u << kMhWin) - 1u));
    }
    __syncthreads();
    // (1) thread 0: the steps from the round's entry state up to the first
    // acceptance (FP64 tests against the entry log-weight)
    if (threadIdx.x == 0) {
      if (b0 == 0) {
        // the start: the first candidate that is not the origin
        bool found = false;
        for (int k = 0; k < 2 && !found; ++k) {
          if (cand[k][0] != 0 || cand[k][1] != 0) { cx = cand[k][0]; cy = cand[k][1]; found = true; }
        }
        for (uint64_t a = 1; a < 64 && !found; ++a) {
          U64x4 c;
          c.v[0] = a; c.v[1] = 1; c.v[2] = counter; c.v[3] = tag;
          const U64x4 w = philox4x64_10(c, seed, 0ull);
          int px, py;
          mh_propose(w.v[0], w.v[1], sdx, sdy, px, py);
          if (px != 0 || py != 0) { cx = px; cy = py; found = true; break; }
          mh_propose(w.v[2], w.v[3], sdx, sdy, px, py);
          if (px != 0 || py != 0) { cx = px; cy = py; found = true; }
        }
        lw = mh_log_weight(lwx, lwy, ri.mxmax, ri.mymax, cx, cy);
      }
      int ta = cnt;
      for (int t = 0; t < cnt; ++t) {
        if (spx[t] != 0 || spy[t] != 0) {
          const double d = slw[t] - lw;
          if (d >= 0.0 || slu[t] < d) { ta = t; break; }
        }
        mh_keep(b0 + t, thin, rep, P, cx, cy, sampled);
      }
      if (ta < cnt) mh_keep(b0 + ta, thin, rep, P, spx[ta], spy[ta], sampled);
      s_ta = ta;
      s_tf = cnt;
      s_end = ta;
    }
    __syncthreads();
    const int ta = s_ta;
    if (ta < cnt) {             // the same for every thread
      // (2) offsets of the steps (ta, cnt) by a block scan of their maps;
      // thread i takes steps ta + 1 + 2i and ta + 2 + 2i
      const int nit = cnt - ta - 1;
      const int k0 = 2 * (int)threadIdx.x;
      const int t0 = ta + 1 + k0, t1 = t0 + 1;
      const MhMap f0 = k0 < nit ? mh_step_map(spx[t0] == 0 && spy[t0] == 0, sacc[t0]) : kMhId;
      const MhMap f1 = k0 + 1 < nit ? mh_step_map(spx[t1] == 0 && spy[t1] == 0, sacc[t1]) : kMhId;
      MhMap F = mh_then(f0, f1);
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const MhMap o = __shfl_up_sync(0xffffffffu, F, d);
        if (lane >= d) F = mh_then(o, F);
      }
      MhMap Ex = __shfl_up_sync(0xffffffffu, F, 1);   // this thread's prefix in its warp
      if (lane == 0) Ex = kMhId;
      if (lane == 31) s_wmap[warp] = F;
      __syncthreads();
      if (warp == 0) {
        const int nw = (int)(blockDim.x >> 5);
        MhMap G = lane < nw ? s_wmap[lane] : kMhId;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const MhMap o = __shfl_up_sync(0xffffffffu, G, d);
          if (lane >= d) G = mh_then(o, G);
        }
        if (lane < nw) s_wpre[lane] = G;       // inclusive over warps
      }
      __syncthreads();
      // (3) the offset entering each of this thread's steps, and the first
      // step entered at kMhFar (from there on thread 0 decides)
      int oin0 = mh_at(warp > 0 ? s_wpre[warp - 1] : kMhId, 0);
      oin0 = mh_at(Ex, oin0);
      const int o0 = mh_at(f0, oin0), o1 = mh_at(f1, o0);
      if (k0 < nit && oin0 == kMhFar) atomicMin(&s_tf, t0);
      else if (k0 + 1 < nit && o0 == kMhFar) atomicMin(&s_tf, t1);
      __syncthreads();
      const int tf = s_tf;
      // (4) the kept states of the steps before tf, and the round's end state
      if (k0 < nit && t0 < tf) {
        mh_keep(b0 + t0, thin, rep, P, spx[t0 - o0], spy[t0 - o0], sampled);
        if (t0 == cnt - 1) s_end = t0 - o0;
      }
      if (k0 + 1 < nit && t1 < tf) {
        mh_keep(b0 + t1, thin, rep, P, spx[t1 - o1], spy[t1 - o1], sampled);
        if (t1 == cnt - 1) s_end = t1 - o1;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int jc = s_end;
        if (tf < cnt) {
          // (5) from tf on: the state is kMhWin steps back; decide step by
          // step with the decision bits where they reach, else in FP64
          jc = tf - 1 - kMhFar;
          cx = spx[jc];
          cy = spy[jc];
          for (int t = tf; t < cnt; ++t) {
            if (spx[t] != 0 || spy[t] != 0) {
              const int dist = t - 1 - jc;
              bool acc;
              if (dist < kMhWin) {
                acc = (sacc[t] >> dist) & 1u;
              } else {
                const double d = slw[t] - slw[jc];
                acc = d >= 0.0 || slu[t] < d;
              }
              if (acc) { cx = spx[t]; cy = spy[t]; jc = t; }
            }
            mh_keep(b0 + t, thin, rep, P, cx, cy, sampled);
          }
        }
        cx = spx[jc];
        cy = spy[jc];
        lw = slw[jc];
      }
    }
    __syncthreads();
  }
}

void launch_mh_chain(const Reps& rp, int P, int thin, uint64_t seed, const uint64_t* ctr,
                     const double* cdf, double alpha, int32_t* sampled, cudaStream_t st) {
  mh_chain_kernel<<<rp.R * kMhCluster, kMhThreads, 0, st>>>(rp, P, thin, seed, ctr, cdf, alpha,
                                                            sampled);
}

template <typename T>
void launch_mode_coef(const Reps& rp, int npc, const int32_t* list, int rbe, uint64_t seed,
                      const uint64_t* ctr, const double* cdf, const PairTab& pairs,
                      double alpha, ModeTab<T> modes, int32_t* sampled, cudaStream_t st) {
  // Kpad is a multiple of 32, so Kpad G threads fill 64-thread blocks exactly
  if (npc <= 4) {
    dim3 grid(rp.Kpad * 4 / 64, rp.R);
    mode_coef_kernel<T, 4><<<grid, 64, 0, st>>>(rp, npc, list, rbe, seed, ctr, cdf, pairs, alpha,
                                                modes, sampled);
  } else if (npc <= 8) {
    dim3 grid(rp.Kpad * 8 / 64, rp.R);
    mode_coef_kernel<T, 8><<<grid, 64, 0, st>>>(rp, npc, list, rbe, seed, ctr, cdf, pairs, alpha,
                                                modes, sampled);
  } else {
    dim3 grid(rp.Kpad * 16 / 64, rp.R);
    mode_coef_kernel<T, 16><<<grid, 64, 0, st>>>(rp, npc, list, rbe, seed, ctr, cdf, pairs,
                                                 alpha, modes, sampled);
  }
}

// ============================================================ instantiations
#define QSLAB_INST(T, PH)                                                                        \
  template void launch_prepare<T>(const Reps&, const T*, const T*, void*, uint32_t*, int32_t*,   \
                                  double*, unsigned*, cudaStream_t);                             \
  template void launch_gather<T>(const Reps&, const T*, const T*, const uint32_t*, const void*,  \
                                 T*, T*, T*, PH*, PH*, int32_t*, cudaStream_t);                  \
  template void launch_combine<T>(const Reps&, int, const T*, const void*, const void*,          \
                                  const T*, const T*, const PH*, const PH*, const WallTab&,       \
                                  const int32_t*, double*, T*, T*, double*, cudaStream_t);       \
  template void launch_mode_coef<T>(const Reps&, int, const int32_t*, int, uint64_t,             \
                                    const uint64_t*, const double*, const PairTab&, double,      \
                                    ModeTab<T>, int32_t*, cudaStream_t);
QSLAB_INST(float, uint32_t)
QSLAB_INST(double, uint64_t)
#undef QSLAB_INST

}  // namespace qslab
