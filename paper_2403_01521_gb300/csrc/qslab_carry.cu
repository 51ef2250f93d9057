// Chunk-to-chunk decays and the carries of the k != 0 scans: the states
// entering every chunk, from the chunk aggregates of pass A, by a linear
// recurrence over the chunks of each replica (Eqs. 3.28-3.30 applied to
// whole chunks). Also the pair decays of the k = 0 chunks.
#include <cstdint>
#include <cuda_runtime.h>

#include "qslab_df.cuh"
#include "qslab_geom.cuh"
#include "qslab_internal.h"
#include "qslab_math.cuh"

namespace qslab {

// --------------------------------------------------- chunk-to-chunk decays
// All decays between chunk reference points are computed in FP64 by these
// parallel kernels and stored in the carry type (FP64, or double-float on the
// FP32 path), so that the sequential chains below only multiply and add.
//   pair decays  pdec[dir][c][p]: forward e^{-a_p (z_end(c) - z_end(c-1))},
//                backward e^{-a_p (z_start(c+1) - z_start(c))}
//   mode decays  kdec[dir][c][m]: the same with beta = |k_m|
//   group pair decays gpd[dir][g][p]: the product over a carry group
// All are 1 (gap 0) where the chain of a replica starts, whose carry is 0.
// zero_chunks = 0: k-space chunks (L), 1: k = 0 chunks (L0)
template <typename T>
__device__ __forceinline__ void pair_decay_at(const Reps& rp, int zero_chunks, int np, const T* zs,
                                              const PairTab& pairs,
                                              Cplx<typename CarryNum<T>::type>* pdec,
                                              typename CarryNum<T>::type* gaps, int e) {
  using CN = typename CarryNum<T>::type;
  const int nch = zero_chunks ? rp.nzchunks : rp.nchunks;
  const int dir = e / (nch * np);
  const int r = e - dir * nch * np;
  const int c = r / np, p = r - c * np;
  const CRange ch = zero_chunks ? zchunk(rp, c) : kchunk(rp, c);
  const double gap = chunk_gap(zs, ch, dir, zero_chunks ? rp.L0 : rp.L);
  const Cplx<double> d = cexp_neg(pairs.a_re[p], pairs.a_im[p], gap);
  pdec[e] = Cplx<CN>{cn_from(d.re, (CN*)nullptr), cn_from(d.im, (CN*)nullptr)};
  if (gaps && p == 0) gaps[dir * nch + c] = cn_from(gap, (CN*)nullptr);
}

template <typename T>
__global__ void pair_decay_kernel(Reps rp, int zero_chunks, int np, const T* zs, PairTab pairs,
                                  Cplx<typename CarryNum<T>::type>* pdec,
                                  typename CarryNum<T>::type* gaps) {
  const int nch = zero_chunks ? rp.nzchunks : rp.nchunks;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < 2 * nch * np) pair_decay_at<T>(rp, zero_chunks, np, zs, pairs, pdec, gaps, e);
}

// Decay of a pair state across a whole carry group [ca, cb) of k-space
// chunks, in the group's chain order: forward z_end(cb-1) - z_end(ca-1),
// backward z_start(cb) - z_start(ca); 0 for the group where the chain starts.
template <typename T>
__device__ __forceinline__ void group_pair_decay_at(const Reps& rp, int np, const T* zs,
                                                    const PairTab& pairs,
                                                    Cplx<typename CarryNum<T>::type>* gpd, int e) {
  using CN = typename CarryNum<T>::type;
  const int NG = rp.ngroups;
  const int dir = e / (NG * np);
  const int r = e - dir * NG * np;
  const int grp = r / np, p = r - grp * np;
  const RepInfo& ri = rp.info[rp.group_rep[grp]];
  const int ca = rp.gstart[grp], cb = rp.gstart[grp + 1];
  double span = 0.0;
  if (dir == 0) {
    if (ca > ri.c0) {
      const CRange last = kchunk(rp, cb - 1);
      span = (double)zs[last.start + last.cnt - 1] - (double)zs[kchunk(rp, ca).start - 1];
    }
  } else if (cb < ri.c0 + ri.nch) {
    span = (double)zs[kchunk(rp, cb).start] - (double)zs[kchunk(rp, ca).start];
  }
  const Cplx<double> d = cexp_neg(pairs.a_re[p], pairs.a_im[p], span);
  gpd[e] = Cplx<CN>{cn_from(d.re, (CN*)nullptr), cn_from(d.im, (CN*)nullptr)};
}

// e^{-x} in FP64 for x >= 0: the Taylor series to x^11 when x < 1/16
// (truncation below 2e-21), the library exp otherwise.
__device__ __forceinline__ double exp_neg_small(double x) {
  if (x >= 0.0625) return exp(-x);
  double r = -1.0 / 39916800.0;
  r = fma(r, x, 1.0 / 3628800.0);
  r = fma(r, x, -1.0 / 362880.0);
  r = fma(r, x, 1.0 / 40320.0);
  r = fma(r, x, -1.0 / 5040.0);
  r = fma(r, x, 1.0 / 720.0);
  r = fma(r, x, -1.0 / 120.0);
  r = fma(r, x, 1.0 / 24.0);
  r = fma(r, x, -1.0 / 6.0);
  r = fma(r, x, 0.5);
  r = fma(r, x, -1.0);
  return fma(r, x, 1.0);
}

// e^{-x} in double-float for 0 <= x < 1/16: the Taylor series to x^12
// (truncation below 5e-20 relative) by Horner's rule in double-float
// arithmetic, whose ~48 bits match the carries' (this replaces ~13 FP64
// operations per decay, on a part where FP64 runs at 1/76 of FP32).
// the coefficients (-1)^n / n!, n = 12 .. 0, split as hi = the FP32 rounding
// of the FP64 value and lo = the FP32 rounding of the remainder
__device__ constexpr float kExpNegDF[13][2] = {
    {2.0876755879584152e-09f, 1.1082839809204342e-16f},
    {-2.5052107943679403e-08f, -4.4176230446483665e-16f},
    {2.755731998149713e-07f, -7.575112209051195e-15f},
    {-2.7557318844628753e-06f, -3.793571224297229e-14f},
    {2.4801587642286904e-05f, -3.40699609366682e-13f},
    {-0.00019841270113829523f, 2.725596874933456e-12f},
    {0.0013888889225199819f, -3.3631094437103215e-11f},
    {-0.008333333767950535f, 4.34617203337595e-10f},
    {0.0416666679084301f, -1.2417634698280722e-09f},
    {-0.1666666716337204f, 4.967053879312289e-09f},
    {0.5f, 0.0f},
    {-1.0f, 0.0f},
    {1.0f, 0.0f}};

__device__ __forceinline__ DF exp_neg_small_df(DF x) {
  DF r = {kExpNegDF[0][0], kExpNegDF[0][1]};
#pragma unroll
  for (int n = 1; n < 13; ++n) r = r * x + DF{kExpNegDF[n][0], kExpNegDF[n][1]};
  return r;
}

// the gap between two chunk reference points as an exact double-float
// (the difference of two FP32 values)
__device__ __forceinline__ DF chunk_gap_df(const float* zs, const CRange& ch, int dir, int L) {
  if (dir == 0) {
    if (ch.first) return DF{0.0f, 0.0f};
    return df_two_sum(zs[ch.start + ch.cnt - 1], -zs[ch.start - 1]);
  }
  if (ch.last) return DF{0.0f, 0.0f};
  return df_two_sum(zs[ch.start + L], -zs[ch.start]);
}

template <typename T>
__device__ __forceinline__ void mode_decay_at(const Reps& rp, const T* zs, const T* kk,
                                              typename CarryNum<T>::type* kdec, int64_t e) {
  using CN = typename CarryNum<T>::type;
  const int64_t per_dir = (int64_t)rp.nchunks * rp.Kpad;
  const int dir = (int)(e / per_dir);
  const int64_t r = e - (int64_t)dir * per_dir;
  const int c = (int)(r / rp.Kpad), m = (int)(r - (int64_t)c * rp.Kpad);
  const CRange ch = kchunk(rp, c);
  if constexpr (sizeof(T) == 4) {
    const DF x = df_from((float)kk[(size_t)ch.r * rp.Kpad + m]) * chunk_gap_df(zs, ch, dir, rp.L);
    if (x.hi < 0.0625f) {
      kdec[e] = exp_neg_small_df(x);
      return;
    }
    kdec[e] = cn_from(exp(-df_to_double(x)), (CN*)nullptr);
  } else {
    const double x = (double)kk[(size_t)ch.r * rp.Kpad + m] * chunk_gap(zs, ch, dir, rp.L);
    kdec[e] = cn_from(exp_neg_small(x), (CN*)nullptr);
  }
}

// The three decay tables of the k-space carries in one launch: pair decays
// on [0, ne), group pair decays on [ne, ne + nge), mode decays after them.
template <typename T>
__global__ void kspace_decay_kernel(Reps rp, int np, const T* zs, const T* kk, PairTab pairs,
                                    Cplx<typename CarryNum<T>::type>* pdec,
                                    Cplx<typename CarryNum<T>::type>* gpd,
                                    typename CarryNum<T>::type* kdec) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // group decays only serve the three-phase chains
  const int64_t ne = (int64_t)2 * rp.nchunks * np, nge = rp.kflat ? 0 : (int64_t)2 * rp.ngroups * np;
  const int64_t nk = (int64_t)2 * rp.nchunks * rp.Kpad;
  if (e < ne) pair_decay_at<T>(rp, 0, np, zs, pairs, pdec, nullptr, (int)e);
  else if (e < ne + nge) group_pair_decay_at<T>(rp, np, zs, pairs, gpd, (int)(e - ne));
  else if (e < ne + nge + nk) mode_decay_at<T>(rp, zs, kk, kdec, e - ne - nge);
}

// ------------------------------------------------------------------ carries
// carry_in[c+1] = D_c carry_in[c] + A_c over the chunks of a replica
// (forward; mirrored backward), one chain per (replica, direction, state,
// mode), in the carry type. The chunks of a replica are cut into groups,
// and the chains run in three parallel phases: (1) every group composes its
// output from a zero input, A_g (for beta = k also its decay D_g, the
// product of the chunks' real decays; a pair's D_g is the closed form of
// group_pair_decay_at); (2) a short chain over the replica's groups
// gives each group's input; (3) every group replays its chunks from that
// input and writes the carries. Depth 2g + G instead of G g for G groups of
// g chunks; the last group of a chain needs no phase 1. Loads and stores
// are coalesced across modes and issued in batches.

template <typename T>
struct CarryCtx {
  Reps rp;
  int S, np;
  size_t cs;        // stride between chunks in agg/carry (S * Kpad)
  size_t dirstride; // nchunks * S * Kpad
};

// phase 1 (replay = false) and phase 3 (replay = true); thread = (dir, state, group, mode)
template <typename T>
__global__ void carry_group_kernel(CarryCtx<T> X, const Cplx<T>* __restrict__ agg,
                                   Cplx<T>* __restrict__ carry,
                                   const Cplx<typename CarryNum<T>::type>* __restrict__ pdec,
                                   const typename CarryNum<T>::type* __restrict__ kdec,
                                   typename CarryNum<T>::type* __restrict__ gkD,
                                   Cplx<typename CarryNum<T>::type>* __restrict__ gA, bool replay) {
  using CN = typename CarryNum<T>::type;
  const int Kpad = X.rp.Kpad, NG = X.rp.ngroups;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per_dir = (int64_t)X.S * NG * Kpad;
  if (e >= 2 * per_dir) return;
  const int dir = (int)(e / per_dir);
  int64_t r = e - dir * per_dir;
  const int st = (int)(r / ((int64_t)NG * Kpad));
  r -= (int64_t)st * NG * Kpad;
  const int grp = (int)(r / Kpad), m = (int)(r - (int64_t)grp * Kpad);
  if (!replay) {
    const RepInfo& ri = X.rp.info[X.rp.group_rep[grp]];
    if (grp == (dir == 0 ? ri.g0 + ri.ng - 1 : ri.g0)) return;   // last in its chain
  }
  const size_t gidx = (((size_t)dir * X.S + st) * NG + grp) * Kpad + m;
  const CN zero = cn_zero((CN*)nullptr);
  CN cr = zero, ci = zero, pk = cn_from(1.0, (CN*)nullptr);
  if (replay && !X.rp.kflat) { cr = gA[gidx].re; ci = gA[gidx].im; }
  const int ca = X.rp.gstart[grp], cb = X.rp.gstart[grp + 1];
  const int len = cb - ca;
  const int cfirst = dir == 0 ? ca : cb - 1;
  const int64_t cstep = dir == 0 ? 1 : -1;
  const Cplx<T>* A = agg + dir * X.dirstride + (size_t)cfirst * X.cs + (size_t)st * Kpad + m;
  Cplx<T>* C = carry + dir * X.dirstride + (size_t)cfirst * X.cs + (size_t)st * Kpad + m;
  const int64_t astep = cstep * (int64_t)X.cs;
  constexpr int B = 4;
  if (st == 0) {
    // beta = k: real decays
    const CN* D = kdec + ((size_t)dir * X.rp.nchunks + cfirst) * Kpad + m;
    const int64_t dstep = cstep * Kpad;
    for (int jb = 0; jb < len; jb += B) {
      Cplx<T> a[B];
      CN d[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        if (jb + u < len) { a[u] = A[(jb + u) * astep]; d[u] = D[(jb + u) * dstep]; }
        else { a[u] = Cplx<T>{0, 0}; d[u] = zero; }
      }
#pragma unroll
      for (int u = 0; u < B; ++u) {
        if (jb + u < len) {
          if (replay) C[(jb + u) * astep] = Cplx<T>{cn_to_t(cr), cn_to_t(ci)};
          cr = d[u] * cr + cn_from_t(a[u].re, (CN*)nullptr);
          ci = d[u] * ci + cn_from_t(a[u].im, (CN*)nullptr);
          if (!replay) pk = d[u] * pk;
        }
      }
    }
  } else {
    const Cplx<CN>* D = pdec + ((size_t)dir * X.rp.nchunks + cfirst) * X.np + ((st - 1) >> 1);
    const int64_t dstep = cstep * X.np;
    for (int jb = 0; jb < len; jb += B) {
      Cplx<T> a[B];
      Cplx<CN> d[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        if (jb + u < len) { a[u] = A[(jb + u) * astep]; d[u] = D[(jb + u) * dstep]; }
        else { a[u] = Cplx<T>{0, 0}; d[u] = Cplx<CN>{zero, zero}; }
      }
#pragma unroll
      for (int u = 0; u < B; ++u) {
        if (jb + u < len) {
          if (replay) C[(jb + u) * astep] = Cplx<T>{cn_to_t(cr), cn_to_t(ci)};
          const CN nr = d[u].re * cr - d[u].im * ci + cn_from_t(a[u].re, (CN*)nullptr);
          const CN ni = d[u].re * ci + d[u].im * cr + cn_from_t(a[u].im, (CN*)nullptr);
          cr = nr; ci = ni;
        }
      }
    }
  }
  if (!replay) {
    gA[gidx] = Cplx<CN>{cr, ci};
    if (st == 0) gkD[((size_t)dir * NG + grp) * Kpad + m] = pk;
  }
}

// phase 2: thread = (dir, state, replica, mode); turns gA into each group's
// input. The transfers of up to 8 groups are loaded before they are used.
template <typename T>
__global__ void carry_chain_kernel(CarryCtx<T> X,
                                   const typename CarryNum<T>::type* __restrict__ gkD,
                                   const Cplx<typename CarryNum<T>::type>* __restrict__ gpd,
                                   Cplx<typename CarryNum<T>::type>* __restrict__ gA) {
  using CN = typename CarryNum<T>::type;
  const int Kpad = X.rp.Kpad, NG = X.rp.ngroups, R = X.rp.R;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per_dir = (int64_t)X.S * R * Kpad;
  if (e >= 2 * per_dir) return;
  const int dir = (int)(e / per_dir);
  int64_t r = e - dir * per_dir;
  const int st = (int)(r / ((int64_t)R * Kpad));
  r -= (int64_t)st * R * Kpad;
  const int rep = (int)(r / Kpad), m = (int)(r - (int64_t)rep * Kpad);
  const int g0 = X.rp.info[rep].g0, ng = X.rp.info[rep].ng;
  const CN zero = cn_zero((CN*)nullptr);
  CN cr = zero, ci = zero;
  const int p = (st - 1) >> 1;
  constexpr int B = 8;
  for (int jb = 0; jb < ng; jb += B) {
    Cplx<CN> d[B], a[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int j = jb + u;
      d[u] = Cplx<CN>{zero, zero};
      a[u] = Cplx<CN>{zero, zero};
      if (j < ng - 1) {
        const int grp = dir == 0 ? g0 + j : g0 + ng - 1 - j;
        a[u] = gA[(((size_t)dir * X.S + st) * NG + grp) * Kpad + m];
        if (st == 0) d[u].re = gkD[((size_t)dir * NG + grp) * Kpad + m];
        else d[u] = gpd[((size_t)dir * NG + grp) * X.np + p];
      }
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int j = jb + u;
      if (j < ng) {
        const int grp = dir == 0 ? g0 + j : g0 + ng - 1 - j;
        gA[(((size_t)dir * X.S + st) * NG + grp) * Kpad + m] = Cplx<CN>{cr, ci};
        if (j < ng - 1) {
          const CN nr = d[u].re * cr - d[u].im * ci + a[u].re;
          const CN ni = d[u].re * ci + d[u].im * cr + a[u].im;
          cr = nr; ci = ni;
        }
      }
    }
  }
}

// Views of the decay and transfer tables: pdec [2][nchunks][np] complex,
// kdec [2][nchunks][Kpad], gkD [2][ngroups][Kpad], gpd [2][ngroups][np]
// complex, gA [2][S][ngroups][Kpad] complex, all in the carry type.
template <typename T>
struct DecayViews {
  using CN = typename CarryNum<T>::type;
  Cplx<CN>* pdec;
  CN* kdec;
  CN* gkD;
  Cplx<CN>* gpd;
  Cplx<CN>* gA;
};

template <typename T>
DecayViews<T> decay_views(const ScanPlan& pl, const Reps& rp, void* dec) {
  using CN = typename CarryNum<T>::type;
  DecayViews<T> v;
  char* p = static_cast<char*>(dec);
  auto take = [&p](size_t b) { char* r = p; p += (b + 255) & ~size_t(255); return r; };
  v.pdec = reinterpret_cast<Cplx<CN>*>(take(sizeof(Cplx<CN>) * 2 * (size_t)rp.nchunks * pl.np));
  v.kdec = reinterpret_cast<CN*>(take(sizeof(CN) * 2 * (size_t)rp.nchunks * rp.Kpad));
  v.gkD = reinterpret_cast<CN*>(take(sizeof(CN) * 2 * (size_t)rp.ngroups * rp.Kpad));
  v.gpd = reinterpret_cast<Cplx<CN>*>(take(sizeof(Cplx<CN>) * 2 * (size_t)rp.ngroups * pl.np));
  v.gA = reinterpret_cast<Cplx<CN>*>(
      take(sizeof(Cplx<CN>) * 2 * (size_t)pl.nstates * rp.ngroups * rp.Kpad));
  return v;
}

size_t kspace_decay_bytes(const ScanPlan& pl, const Reps& rp, int fp64) {
  const size_t cn = fp64 ? sizeof(double) : sizeof(DF);
  return 2 * cn * 2 * (size_t)rp.nchunks * pl.np + cn * 2 * (size_t)rp.nchunks * rp.Kpad +
         cn * 2 * (size_t)rp.ngroups * rp.Kpad + 2 * cn * 2 * (size_t)rp.ngroups * pl.np +
         2 * cn * 2 * (size_t)pl.nstates * rp.ngroups * rp.Kpad + 5 * 256;
}

template <typename T>
void launch_kspace_carries(const ScanPlan& pl, const Reps& rp, const PairTab& pairs, const T* zs,
                           const T* kk, const Cplx<T>* agg, Cplx<T>* carry, void* dec,
                           cudaStream_t st) {
  const DecayViews<T> v = decay_views<T>(pl, rp, dec);
  const int64_t nall = (int64_t)2 * rp.nchunks * pl.np +
                       (rp.kflat ? 0 : (int64_t)2 * rp.ngroups * pl.np) +
                       (int64_t)2 * rp.nchunks * rp.Kpad;
  // 64-thread blocks: each thread's FP64 exponentials go to as many SMs as
  // possible (an SM issues FP64 at a small fraction of its FP32 rate)
  kspace_decay_kernel<T><<<(unsigned)((nall + 63) / 64), 64, 0, st>>>(
      rp, pl.np, zs, kk, pairs, v.pdec, v.gpd, v.kdec);
  CarryCtx<T> X;
  X.rp = rp;
  X.S = pl.nstates;
  X.np = pl.np;
  X.cs = (size_t)pl.nstates * rp.Kpad;
  X.dirstride = (size_t)rp.nchunks * pl.nstates * rp.Kpad;
  const int64_t ng = (int64_t)2 * X.S * rp.ngroups * rp.Kpad;
  if (rp.kflat) {
    // one group per chain: the replay from zero is the whole scan
    carry_group_kernel<T><<<(unsigned)((ng + 127) / 128), 128, 0, st>>>(
        X, agg, carry, v.pdec, v.kdec, v.gkD, v.gA, true);
    return;
  }
  carry_group_kernel<T><<<(unsigned)((ng + 127) / 128), 128, 0, st>>>(
      X, agg, carry, v.pdec, v.kdec, v.gkD, v.gA, false);
  const int64_t nt = (int64_t)2 * X.S * rp.R * rp.Kpad;
  carry_chain_kernel<T><<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(X, v.gkD, v.gpd, v.gA);
  carry_group_kernel<T><<<(unsigned)((ng + 127) / 128), 128, 0, st>>>(
      X, agg, carry, v.pdec, v.kdec, v.gkD, v.gA, true);
}

template <typename T>
void launch_pair_decay(const Reps& rp, int zero_chunks, int np, const T* zs, const PairTab& pairs,
                       void* pdec, void* gaps, cudaStream_t st) {
  using CN = typename CarryNum<T>::type;
  const int nch = zero_chunks ? rp.nzchunks : rp.nchunks;
  const int ne = 2 * nch * np;
  pair_decay_kernel<T><<<(ne + 63) / 64, 64, 0, st>>>(
      rp, zero_chunks, np, zs, pairs, static_cast<Cplx<CN>*>(pdec), static_cast<CN*>(gaps));
}

// ============================================================ instantiations
template void launch_kspace_carries<float>(const ScanPlan&, const Reps&, const PairTab&,
                                           const float*, const float*, const Cplx<float>*,
                                           Cplx<float>*, void*, cudaStream_t);
template void launch_kspace_carries<double>(const ScanPlan&, const Reps&, const PairTab&,
                                            const double*, const double*, const Cplx<double>*,
                                            Cplx<double>*, void*, cudaStream_t);
template void launch_pair_decay<float>(const Reps&, int, int, const float*, const PairTab&, void*,
                                       void*, cudaStream_t);
template void launch_pair_decay<double>(const Reps&, int, int, const double*, const PairTab&,
                                        void*, void*, cudaStream_t);

}  // namespace qslab
