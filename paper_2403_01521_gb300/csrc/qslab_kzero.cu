// The k = 0 term of the SOE-Ewald2D long-range part (Eq. 3.26 and its z
// derivative): FP64 (or double-float) prefix sums for the |z| part and SOE
// scans over the z-sorted particles for the exponential part.
#include <cstdint>
#include <cuda_runtime.h>

#include "qslab_df.cuh"
#include "qslab_geom.cuh"
#include "qslab_internal.h"
#include "qslab_math.cuh"

namespace qslab {

// ================================================================ k = 0 term
// Pair sums of g0_SOE(|z_ij|) (Eq. 3.26) and of its derivative (Eq. E.6):
//   sum_{j != i} q_j g0(|z_ij|) = c1 sum_j q_j |z_ij|
//        + sum_l (w_l/sqrt(pi)) [ (1/alpha) S_l - (2/s_l) H_l ]
//   sum_{j != i} q_j g0'(|z_ij|) sgn(z_i - z_j) = c1 (Q< - Q>)
//        + sum_l (w_l/sqrt(pi)) [ -(2/s_l + s_l)(S_l^f - S_l^b) + 2 alpha (H_l^f - H_l^b) ]
// with S_l = sum_j q_j e^{-a_l |z_ij|} and H_l = sum_j q_j |z_ij| e^{-a_l |z_ij|}
// split into j < i (f) and j > i (b), c1 = sum_l 2 w_l/(s_l sqrt(pi)). The
// |z| sums come from FP64 prefix sums of q and q z (they cancel heavily).
// S and H are scanned in the path precision T, per chunk of L0 particles
// with FP64 carries between chunks; H is carried without cancellation:
//   H_i = d_i (H_{i-1} + dz_i S_{i-1}),  S_i = d_i S_{i-1} + q_i  (inclusive).
// One thread per (chunk, SOE pair representative); the lanes of a chunk sit
// in one warp and are summed by shuffles.

struct K0Params {
  Reps rp;
  int npad;          // lanes per chunk (power of two >= np, at least 4)
  double alpha, c1;
};

// acc + a b, with the product kept exact on the double-float path
__device__ __forceinline__ double cn_add_prod(double acc, double a, double b) { return fma(a, b, acc); }
__device__ __forceinline__ DF cn_add_prod(DF acc, float a, float b) {
  const float p = a * b;
  const DF pr = df_fast_two_sum(p, fmaf(a, b, -p));
  return acc + pr;
}
__device__ __forceinline__ double cn_add(double acc, double a) { return acc + a; }
__device__ __forceinline__ DF cn_add(DF acc, float a) { return acc + a; }

// Chunks per CTA of the k = 0 aggregate and final kernels: kK0Cpb * npad
// threads, the npad lanes of a chunk inside one warp. Each chunk's z, q
// and dz are staged in shared memory first, so that the sequential loops
// below read no global memory.
constexpr int kK0Cpb = 8;

__device__ __forceinline__ double shfl_xor_cn(double v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}
__device__ __forceinline__ DF shfl_xor_cn(DF v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ double shfl_up_cn(double v, int o, int w) {
  return __shfl_up_sync(0xffffffffu, v, o, w);
}
__device__ __forceinline__ DF shfl_up_cn(DF v, int o, int w) {
  return {__shfl_up_sync(0xffffffffu, v.hi, o, w), __shfl_up_sync(0xffffffffu, v.lo, o, w)};
}

template <typename T>
__global__ void kzero_aggregate_kernel(K0Params Q, PairTab pr, const T* zs,
                                       const T* qs, Cplx<T>* agg,
                                       typename CarryNum<T>::type* csum) {
  using CN = typename CarryNum<T>::type;
  extern __shared__ __align__(16) char kag_raw[];   // [kK0Cpb][2][L0] of T
  const int lanes = Q.npad, L0 = Q.rp.L0;
  const int lc = threadIdx.x / lanes, p = threadIdx.x % lanes;
  const int c = blockIdx.x * kK0Cpb + lc;
  T* zl = reinterpret_cast<T*>(kag_raw) + (size_t)lc * 2 * L0;
  T* ql = zl + L0;
  const bool valid = c < Q.rp.nzchunks;
  CRange ch{0, 0, 0, false, false};
  if (valid) ch = zchunk(Q.rp, c);
  const int64_t start = ch.start;
  const int cnt = ch.cnt;
  for (int t = p; t < cnt; t += lanes) { zl[t] = zs[start + t]; ql[t] = qs[start + t]; }
  __syncwarp();
  const T zst = cnt ? zl[0] : (T)0, zen = cnt ? zl[cnt - 1] : (T)0;
  const bool act = valid && p < pr.np;
  const T ar = act ? (T)pr.a_re[p] : (T)0, ai = act ? (T)pr.a_im[p] : (T)0;
  Cplx<T> sf{0, 0}, hf{0, 0}, sb{0, 0}, hb{0, 0};
  if (act) {
    for (int t = 0; t < cnt; ++t) {
      const T z = zl[t], qq = ql[t];
      const T xf = zen - z, xb = z - zst;
      const Cplx<T> ef = cexp_neg(ar, ai, xf);
      const Cplx<T> eb = cexp_neg(ar, ai, xb);
      sf.re = fma(qq, ef.re, sf.re); sf.im = fma(qq, ef.im, sf.im);
      hf.re = fma(qq * xf, ef.re, hf.re); hf.im = fma(qq * xf, ef.im, hf.im);
      sb.re = fma(qq, eb.re, sb.re); sb.im = fma(qq, eb.im, sb.im);
      hb.re = fma(qq * xb, eb.re, hb.re); hb.im = fma(qq * xb, eb.im, hb.im);
    }
    Cplx<T>* a = agg + ((size_t)c * lanes + p) * 4;
    a[0] = sf; a[1] = hf; a[2] = sb; a[3] = hb;
  }
  // chunk sums of q and q z: a segment per lane, then a butterfly over the
  // chunk's lanes (fixed order: deterministic)
  const int seg = (cnt + lanes - 1) / lanes;
  const int ta = min(cnt, p * seg), tb = min(cnt, ta + seg);
  CN q0 = cn_zero((CN*)nullptr), q1 = cn_zero((CN*)nullptr);
  for (int t = ta; t < tb; ++t) { q0 = cn_add(q0, ql[t]); q1 = cn_add_prod(q1, ql[t], zl[t]); }
  for (int o = lanes >> 1; o; o >>= 1) {
    q0 = q0 + shfl_xor_cn(q0, o);
    q1 = q1 + shfl_xor_cn(q1, o);
  }
  if (valid && p == 0) { csum[2 * c] = q0; csum[2 * c + 1] = q1; }
}

// Carries of the k = 0 scans, one CTA per replica. The per-chunk update of
// a pair's state (S, H) is affine, S' = d S + S_c, H' = d (H + g S) + H_c
// (d the chunk's decay, g its gap), and so is any run of chunks:
// (S, H) -> (D S + A_S, D (H + G S) + A_H). The replica's chunks are cut
// into kK0Group groups per (direction, pair) chain; (1) every thread
// composes its group's transfer (D, G, A_S, A_H) from the chunk aggregates,
// (2) one thread per chain runs the short chain over the groups in shared
// memory, (3) every thread replays its group from its input and writes the
// carry entering each chunk. The last warp does the same for the chunk sums
// of q and q z (per-chunk prefixes and the replica's totals).
constexpr int kK0Chains = 512;   // (direction, pair, group) threads per CTA

template <typename CN>
struct K0Transfer {
  CN Dr, Di, G, Sr, Si, Hr, Hi;
};
template <typename CN>
struct K0State {
  CN Sr, Si, Hr, Hi;
};

__host__ __device__ inline int kzero_groups(int npad) { return kK0Chains / (2 * npad); }

template <typename T>
__global__ void __launch_bounds__(kK0Chains + 32) kzero_carry_kernel(K0Params Q, PairTab pr, const typename CarryNum<T>::type* gaps,
                                   const Cplx<T>* agg,
                                   const Cplx<typename CarryNum<T>::type>* pdec,
                                   typename CarryNum<T>::type* carry,
                                   const typename CarryNum<T>::type* csum,
                                   typename CarryNum<T>::type* cpre,
                                   typename CarryNum<T>::type* rtot) {
  using CN = typename CarryNum<T>::type;
  extern __shared__ __align__(16) char k0c_raw[];
  const int G = kzero_groups(Q.npad);
  K0Transfer<CN>* tr = reinterpret_cast<K0Transfer<CN>*>(k0c_raw);          // [2 npad G]
  K0State<CN>* in = reinterpret_cast<K0State<CN>*>(tr + kK0Chains);         // [2 npad G]
  CN* qsum = reinterpret_cast<CN*>(in + kK0Chains);                         // [32][2]
  const CN zero = cn_zero((CN*)nullptr), one = cn_from(1.0, (CN*)nullptr);
  const int rep = blockIdx.x;
  const int z0 = Q.rp.info[rep].z0, nz = Q.rp.info[rep].nz;
  const int nch = Q.rp.nzchunks;
  const int np = pr.np;
  const int e = threadIdx.x;
  const int g = (nz + G - 1) / G;            // chunks per chain group
  const int gq = (nz + 31) / 32;             // chunks per prefix group
  // chain threads: e = (dir * npad + p) * G + grp
  const bool chain = e < kK0Chains;
  const int dir = chain ? e / (Q.npad * G) : 0;
  const int p = chain ? (e / G) % Q.npad : 0;
  const int grp = chain ? e % G : 0;
  const bool act = chain && p < np;
  // the group's chunks in chain order: forward ascending, backward descending
  const int gpos = dir == 0 ? grp : G - 1 - grp;          // position along the chain
  const int ja = gpos * g, jb = min(nz, ja + g);          // replica-local chunk range
  const int q = e - kK0Chains;                            // prefix lane (0..31)
  const int qa = q * gq, qb = min(nz, qa + gq);

  // the chunk aggregates, decay and gap of chunk c for this chain
  auto load_step = [&](int c, Cplx<T>& as, Cplx<T>& ah, Cplx<CN>& d, CN& dz) {
    const Cplx<T>* a = agg + ((size_t)c * Q.npad + p) * 4 + 2 * dir;
    as = a[0];
    ah = a[1];
    d = pdec[((size_t)dir * nch + c) * np + p];
    dz = gaps[dir * nch + c];
  };
  constexpr int B = 4;   // loads in flight per thread (bounded by 96 registers)
  // ---- phase 1: compose the group's transfer from a zero input
  if (act) {
    CN Dr = one, Di = zero, Gs = zero, sr = zero, si = zero, hr = zero, hi = zero;
    for (int j0 = ja; j0 < jb; j0 += B) {
      Cplx<T> as[B], ah[B];
      Cplx<CN> d[B];
      CN dz[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const int j = j0 + u;
        if (j < jb) load_step(dir == 0 ? z0 + j : z0 + nz - 1 - j, as[u], ah[u], d[u], dz[u]);
      }
#pragma unroll
      for (int u = 0; u < B; ++u) {
        if (j0 + u < jb) {
          const CN tr_ = hr + dz[u] * sr, ti_ = hi + dz[u] * si;
          const CN nhr = d[u].re * tr_ - d[u].im * ti_ + cn_from_t(ah[u].re, (CN*)nullptr);
          const CN nhi = d[u].re * ti_ + d[u].im * tr_ + cn_from_t(ah[u].im, (CN*)nullptr);
          const CN nsr = d[u].re * sr - d[u].im * si + cn_from_t(as[u].re, (CN*)nullptr);
          const CN nsi = d[u].re * si + d[u].im * sr + cn_from_t(as[u].im, (CN*)nullptr);
          sr = nsr; si = nsi; hr = nhr; hi = nhi;
          const CN nDr = d[u].re * Dr - d[u].im * Di;
          const CN nDi = d[u].re * Di + d[u].im * Dr;
          Dr = nDr; Di = nDi;
          Gs = Gs + dz[u];
        }
      }
    }
    tr[e] = K0Transfer<CN>{Dr, Di, Gs, sr, si, hr, hi};
  } else if (!chain && q < 32) {
    CN a = zero, b = zero;
    for (int j = qa; j < qb; ++j) { a = a + csum[2 * (z0 + j)]; b = b + csum[2 * (z0 + j) + 1]; }
    qsum[2 * q] = a;
    qsum[2 * q + 1] = b;
  }
  __syncthreads();
  // ---- phase 2: chain over the groups (thread of group 0 of each chain)
  if (act && grp == 0) {
    CN sr = zero, si = zero, hr = zero, hi = zero;
    for (int gg = 0; gg < G; ++gg) {
      // group at chain position gg is thread index with grp' such that
      // gpos(grp') = gg
      const int gidx = dir == 0 ? gg : G - 1 - gg;
      const int t = (dir * Q.npad + p) * G + gidx;
      in[t] = K0State<CN>{sr, si, hr, hi};
      const K0Transfer<CN> x = tr[t];
      const CN tr_ = hr + x.G * sr, ti_ = hi + x.G * si;
      const CN nhr = x.Dr * tr_ - x.Di * ti_ + x.Hr;
      const CN nhi = x.Dr * ti_ + x.Di * tr_ + x.Hi;
      const CN nsr = x.Dr * sr - x.Di * si + x.Sr;
      const CN nsi = x.Dr * si + x.Di * sr + x.Si;
      sr = nsr; si = nsi; hr = nhr; hi = nhi;
    }
  } else if (!chain && q == 0) {
    CN a = zero, b = zero;
    for (int j = 0; j < 32; ++j) {
      const CN na = a + qsum[2 * j], nb = b + qsum[2 * j + 1];
      qsum[2 * j] = a;
      qsum[2 * j + 1] = b;
      a = na; b = nb;
    }
    rtot[2 * rep] = a;
    rtot[2 * rep + 1] = b;
  }
  __syncthreads();
  // ---- phase 3: replay every group from its input, writing the carries
  if (act) {
    const K0State<CN> s0 = in[e];
    CN sr = s0.Sr, si = s0.Si, hr = s0.Hr, hi = s0.Hi;
    for (int j0 = ja; j0 < jb; j0 += B) {
      Cplx<T> as[B], ah[B];
      Cplx<CN> d[B];
      CN dz[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const int j = j0 + u;
        if (j < jb) load_step(dir == 0 ? z0 + j : z0 + nz - 1 - j, as[u], ah[u], d[u], dz[u]);
      }
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const int j = j0 + u;
        if (j < jb) {
          const int c = dir == 0 ? z0 + j : z0 + nz - 1 - j;
          CN* out = carry + (((size_t)dir * nch + c) * Q.npad + p) * 4;
          out[0] = sr; out[1] = si; out[2] = hr; out[3] = hi;
          const CN tr_ = hr + dz[u] * sr, ti_ = hi + dz[u] * si;
          const CN nhr = d[u].re * tr_ - d[u].im * ti_ + cn_from_t(ah[u].re, (CN*)nullptr);
          const CN nhi = d[u].re * ti_ + d[u].im * tr_ + cn_from_t(ah[u].im, (CN*)nullptr);
          const CN nsr = d[u].re * sr - d[u].im * si + cn_from_t(as[u].re, (CN*)nullptr);
          const CN nsi = d[u].re * si + d[u].im * sr + cn_from_t(as[u].im, (CN*)nullptr);
          sr = nsr; si = nsi; hr = nhr; hi = nhi;
        }
      }
    }
  } else if (!chain && q < 32) {
    CN a = qsum[2 * q], b = qsum[2 * q + 1];
    for (int j = qa; j < qb; ++j) {
      const int c = z0 + j;
      cpre[2 * c] = a;
      cpre[2 * c + 1] = b;
      a = a + csum[2 * c];
      b = b + csum[2 * c + 1];
    }
  }
}

inline size_t kzero_carry_smem(int fp64) {
  const size_t cn = fp64 ? sizeof(double) : sizeof(DF);
  return (size_t)kK0Chains * (7 + 4) * cn + 64 * cn;
}

template <typename T>
__global__ void kzero_final_kernel(K0Params Q, PairTab pr, const T* zs,
                                   const T* dz, const T* qs,
                                   const typename CarryNum<T>::type* carry,
                                   const typename CarryNum<T>::type* cpre,
                                   const typename CarryNum<T>::type* rtot,
                                   typename CarryNum<T>::type* phi0,
                                   typename CarryNum<T>::type* fz0) {
  using CN = typename CarryNum<T>::type;
  // per chunk: z, q, dz [L0 + 1] and the potential / derivative sums [L0][2]
  extern __shared__ __align__(16) char ksm_raw[];
  const int lanes = Q.npad;
  const int L0 = Q.rp.L0;
  const int nch = Q.rp.nzchunks;
  const int64_t N = Q.rp.N;
  const int lc = threadIdx.x / lanes, p = threadIdx.x % lanes;
  const int c = blockIdx.x * kK0Cpb + lc;
  T* zl = reinterpret_cast<T*>(ksm_raw) + (size_t)lc * (5 * L0 + 3);
  T* ql = zl + (L0 + 1);
  T* dzl = ql + (L0 + 1);
  T* acc = dzl + (L0 + 1);
  const bool valid = c < nch;
  CRange ch{0, 0, 0, false, false};
  if (valid) ch = zchunk(Q.rp, c);
  const int64_t start = ch.start;
  const int cnt = ch.cnt;
  // stage the chunk; dz[cnt] is the next particle's (the backward scan's
  // first decay; 0 past the replica's end, where its carry is 0)
  for (int t = p; t <= cnt && valid; t += lanes) {
    const int64_t i = start + t;
    if (t < cnt) { zl[t] = zs[i]; ql[t] = qs[i]; }
    dzl[t] = i < N ? dz[i] : (T)0;
  }
  for (int t = p; t < L0; t += lanes) { acc[2 * t] = 0; acc[2 * t + 1] = 0; }
  __syncwarp();
  const bool act = valid && p < pr.np;
  const double sq = 1.7724538509055160;   // sqrt(pi)
  T cwr = 0, cwi = 0, isr = 0, isi = 0, csr = 0, csi = 0, ar = 1, ai = 0;
  if (act) {
    // multiplicity times w_p/sqrt(pi), 1/s_p and 2/s_p + s_p
    const double sr_ = pr.s_re[p], si_ = pr.s_im[p];
    const double den = sr_ * sr_ + si_ * si_;
    cwr = (T)(pr.mult[p] * pr.w_re[p] / sq); cwi = (T)(pr.mult[p] * pr.w_im[p] / sq);
    isr = (T)(sr_ / den); isi = (T)(-si_ / den);
    csr = (T)(2 * sr_ / den + sr_); csi = (T)(-2 * si_ / den + si_);
    ar = (T)pr.a_re[p]; ai = (T)pr.a_im[p];
  }
  const T alpha = (T)Q.alpha, ialpha = (T)(1.0 / Q.alpha);
  for (int dir = 0; dir < 2; ++dir) {
    T sr = 0, si = 0, hr = 0, hi = 0;
    if (act) {
      const CN* in = carry + (((size_t)dir * nch + c) * Q.npad + p) * 4;
      sr = cn_to_t(in[0]); si = cn_to_t(in[1]); hr = cn_to_t(in[2]); hi = cn_to_t(in[3]);
    }
    // every lane runs L0 steps so that the shuffles below see the whole warp
    for (int n = 0; n < L0; ++n) {
      const bool live = n < cnt;
      const int t = dir == 0 ? n : cnt - 1 - n;
      T pot = 0, der = 0;
      if (act && live) {
        const T qq = ql[t];
        const T dzi = dzl[dir == 0 ? t : t + 1];
        const Cplx<T> d = cexp_neg(ar, ai, dzi);
        // H first (uses the previous inclusive S), then S
        const T tr = fma(dzi, sr, hr), ti = fma(dzi, si, hi);
        hr = d.re * tr - d.im * ti; hi = fma(d.re, ti, d.im * tr);
        const T nsr = fma(d.re, sr, fma(-d.im, si, qq));
        const T nsi = fma(d.re, si, d.im * sr);
        sr = nsr; si = nsi;
        // exclusive S (j != i): S - q_i ; H has no j = i term
        const T xr = sr - qq, xi = si;
        // pot part: cw [ (1/alpha) S - 2 (1/s) H ]
        const T ur = xr * ialpha - 2 * (isr * hr - isi * hi);
        const T ui = xi * ialpha - 2 * (isr * hi + isi * hr);
        pot = cwr * ur - cwi * ui;
        // der part: cw [ -(2/s + s) S + 2 alpha H ] with sign +/- by direction
        const T vr = -(csr * xr - csi * xi) + 2 * alpha * hr;
        const T vi = -(csr * xi + csi * xr) + 2 * alpha * hi;
        der = (dir == 0 ? (T)1 : (T)-1) * (cwr * vr - cwi * vi);
      }
      for (int o = lanes >> 1; o; o >>= 1) {
        pot += __shfl_xor_sync(0xffffffffu, pot, o);
        der += __shfl_xor_sync(0xffffffffu, der, o);
      }
      if (p == 0 && live) { acc[2 * t] += pot; acc[2 * t + 1] += der; }
    }
  }
  __syncwarp();
  // sum_j q_j |z_i - z_j| = z_i (Q< - Q>) - P< + P>, from prefix sums in the
  // carry type (the terms cancel heavily); the result stays in the carry
  // type and the combine kernel widens it to FP64. Each lane takes a segment
  // of the chunk: its sums, an exclusive scan over the lanes, then the
  // segment's particles in order.
  const int seg = (cnt + lanes - 1) / lanes;
  const int ta = min(cnt, p * seg), tb = min(cnt, ta + seg);
  CN sq0 = cn_zero((CN*)nullptr), sq1 = cn_zero((CN*)nullptr);
  for (int t = ta; t < tb; ++t) { sq0 = cn_add(sq0, ql[t]); sq1 = cn_add_prod(sq1, ql[t], zl[t]); }
  for (int o = 1; o < lanes; o <<= 1) {   // inclusive scan over the chunk's lanes
    const CN u0 = shfl_up_cn(sq0, o, lanes), u1 = shfl_up_cn(sq1, o, lanes);
    if (p >= o) { sq0 = u0 + sq0; sq1 = u1 + sq1; }
  }
  CN e0 = shfl_up_cn(sq0, 1, lanes), e1 = shfl_up_cn(sq1, 1, lanes);   // exclusive
  if (p == 0) { e0 = cn_zero((CN*)nullptr); e1 = cn_zero((CN*)nullptr); }
  if (valid) {
    CN Ql = cpre[2 * c] + e0, Pl = cpre[2 * c + 1] + e1;
    const CN Qt = rtot[2 * ch.r], Pt = rtot[2 * ch.r + 1];
    const CN c1 = cn_from(Q.c1, (CN*)nullptr);
    const CN pre = cn_from(2.0 * 3.14159265358979323846 / Q.rp.info[ch.r].area, (CN*)nullptr);
    for (int t = ta; t < tb; ++t) {
      const int64_t i = start + t;
      const T zt = zl[t], qt = ql[t];
      const CN zc = cn_from_t(zt, (CN*)nullptr);
      const CN Qg = Qt - Ql - cn_from_t(qt, (CN*)nullptr);
      const CN Pg = cn_add_prod(Pt - Pl, -qt, zt);
      const CN lin = zc * (Ql - Qg) - Pl + Pg;
      const CN pot = c1 * lin + cn_from_t(acc[2 * t], (CN*)nullptr);
      const CN der = c1 * (Ql - Qg) + cn_from_t(acc[2 * t + 1], (CN*)nullptr);
      phi0[i] = -(pre * pot);
      fz0[i] = pre * der * cn_from_t(qt, (CN*)nullptr);
      Ql = cn_add(Ql, qt);
      Pl = cn_add_prod(Pl, qt, zt);
    }
  }
}

inline int kzero_lanes(int np) {
  int npad = 4;                 // at least 4 lanes per chunk: 8 chunks fill a warp multiple
  while (npad < np) npad <<= 1;
  return npad;
}

template <typename T>
void launch_kzero(const Reps& rp, const PairTab& pairs, double alpha, const T* zs,
                  const T* dz, const T* qs, double* work, void* phi0v, void* fz0v,
                  cudaStream_t st) {
  using CN = typename CarryNum<T>::type;
  K0Params Q;
  Q.rp = rp;
  Q.alpha = alpha;
  const int npad = kzero_lanes(pairs.np);
  Q.npad = npad;
  double c1 = 0.0;
  for (int p = 0; p < pairs.np; ++p) {
    // c1 = sum over nodes of 2 w/(s sqrt(pi)) = sum over representatives of mult 2 Re(w/s)/sqrt(pi)
    const double den = pairs.s_re[p] * pairs.s_re[p] + pairs.s_im[p] * pairs.s_im[p];
    const double re = (pairs.w_re[p] * pairs.s_re[p] + pairs.w_im[p] * pairs.s_im[p]) / den;
    c1 += pairs.mult[p] * 2.0 * re / 1.7724538509055160;
  }
  Q.c1 = c1;
  const int nch = rp.nzchunks;
  // work layout: agg [nch][npad][4] Cplx<T>, csum [nch][2] CN,
  // pdec [2][nch][np] Cplx<CN>, carry [2][nch][npad][4] CN, cpre [nch][2] CN,
  // rtot [R][2] CN, gaps [2][nch] CN
  char* w = reinterpret_cast<char*>(work);
  auto take = [&w](size_t b) { char* r = w; w += (b + 255) & ~size_t(255); return r; };
  Cplx<T>* agg = reinterpret_cast<Cplx<T>*>(take(sizeof(Cplx<T>) * (size_t)nch * npad * 4));
  CN* csum = reinterpret_cast<CN*>(take(sizeof(CN) * (size_t)nch * 2));
  Cplx<CN>* pdec = reinterpret_cast<Cplx<CN>*>(take(sizeof(Cplx<CN>) * (size_t)2 * nch * pairs.np));
  CN* carry = reinterpret_cast<CN*>(take(sizeof(CN) * (size_t)2 * nch * npad * 4));
  CN* cpre = reinterpret_cast<CN*>(take(sizeof(CN) * (size_t)nch * 2));
  CN* rtot = reinterpret_cast<CN*>(take(sizeof(CN) * (size_t)rp.R * 2));
  CN* gaps = reinterpret_cast<CN*>(take(sizeof(CN) * (size_t)2 * nch));
  CN* phi0 = static_cast<CN*>(phi0v);
  CN* fz0 = static_cast<CN*>(fz0v);
  const int nblk = (nch + kK0Cpb - 1) / kK0Cpb;
  const int thr = npad * kK0Cpb;      // whole warps for npad >= 4
  const size_t sma = (size_t)kK0Cpb * 2 * rp.L0 * sizeof(T);
  cudaFuncSetAttribute(kzero_aggregate_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sma);
  kzero_aggregate_kernel<T><<<nblk, thr, sma, st>>>(Q, pairs, zs, qs, agg, csum);
  launch_pair_decay<T>(rp, 1, pairs.np, zs, pairs, pdec, gaps, st);
  const size_t smc = kzero_carry_smem(sizeof(T) == 8);
  cudaFuncSetAttribute(kzero_carry_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
  kzero_carry_kernel<T><<<rp.R, kK0Chains + 32, smc, st>>>(Q, pairs, gaps, agg, pdec, carry, csum,
                                                           cpre, rtot);
  const size_t smf = (size_t)kK0Cpb * (5 * rp.L0 + 3) * sizeof(T);
  cudaFuncSetAttribute(kzero_final_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf);
  kzero_final_kernel<T><<<nblk, thr, smf, st>>>(Q, pairs, zs, dz, qs, carry, cpre, rtot, phi0,
                                                fz0);
}

size_t kzero_work_doubles(int nzchunks, int R, int np) {
  const int npad = kzero_lanes(np);
  // in 8-byte units (a double-float takes one), with room for the 256-byte
  // alignment of each of the 7 arrays
  return (size_t)nzchunks * npad * 4 * 2 + (size_t)nzchunks * 2 +
         (size_t)2 * nzchunks * kMaxPairs * 2 + (size_t)2 * nzchunks * npad * 4 +
         (size_t)nzchunks * 2 + (size_t)R * 2 + (size_t)2 * nzchunks + 7 * 32 + 64;
}

// ============================================================ instantiations
template void launch_kzero<float>(const Reps&, const PairTab&, double, const float*, const float*,
                                  const float*, double*, void*, void*, cudaStream_t);
template void launch_kzero<double>(const Reps&, const PairTab&, double, const double*,
                                   const double*, const double*, double*, void*, void*,
                                   cudaStream_t);

}  // namespace qslab
