// The k = 0 term of the SOE-Ewald2D long-range part (Eq. 3.26 and its z
// derivative): prefix sums for the |z| part (FP64 on the FP64 path,
// double-float on the FP32 path) and SOE scans over the z-sorted particles
// for the exponential part (within a chunk in the path precision, FP32 on
// the FP32 path; carries between chunks in FP64 or double-float).
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
// |z| sums come from prefix sums of q and q z in the carry type (FP64, or
// double-float on the FP32 path: they cancel heavily). S and H are scanned
// in the path precision T, per chunk of L0 particles, with carries between
// chunks in the carry type; H is carried without cancellation:
//   H_i = d_i (H_{i-1} + dz_i S_{i-1}),  S_i = d_i S_{i-1} + q_i  (inclusive).
// One thread per (chunk, SOE pair representative); the lanes of a chunk sit
// in one warp and are summed by shuffles.

struct K0Params {
  Reps rp;
  int npad;          // lanes per chunk (power of two >= np, at least 4)
  double alpha, c1;
  // per pair representative (host-computed, so that no lane divides in
  // FP64): multiplicity w/sqrt(pi), 1/s and 2/s + s, real and imaginary parts
  double cw[2][kMaxPairs], is[2][kMaxPairs], cs[2][kMaxPairs];
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
constexpr int kK0Batch = 8;     // steps whose decays the final kernel computes ahead

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
  bool valid = c < Q.rp.nzchunks;
  CRange ch{0, 0, 0, false, false};
  if (valid) {
    ch = zchunk(Q.rp, c);
    // debug builds: a chunk outside the arrays is left out
    if (!QS_DCHECK(chunk_ok(Q.rp, ch, Q.rp.L0), Q.rp.status)) {
      valid = false;
      ch = CRange{0, 0, 0, false, false};
    }
  }
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

// Carries of the k = 0 scans. The per-chunk update of a pair's state
// (S, H) is affine, S' = d S + S_c, H' = d (H + g S) + H_c (d the chunk's
// decay, g its gap), and so is any run of chunks:
// (S, H) -> (D S + A_S, D (H + G S) + A_H). A slab's k = 0 chunks are cut
// into about sqrt(nz) groups of about sqrt(nz) chunks, and the chains run in
// three parallel phases as the k-space carries do: (1) every (direction,
// group, pair) composes its group's transfer (D, G, A_S, A_H) from the chunk
// aggregates (kzero_group_kernel), (2) one thread per (direction, slab,
// pair) chains the groups (kzero_chain_kernel), (3) every group replays its
// chunks from its input and writes the carry entering each chunk. The chunk
// sums of q and q z go through the same three phases (per-chunk prefixes
// and the slab's totals). Lanes run over the pairs of one group, so that
// their loads are contiguous.
template <typename CN>
struct K0Transfer {
  CN Dr, Di, G, Sr, Si, Hr, Hi;
};
template <typename CN>
struct K0State {
  CN Sr, Si, Hr, Hi;
};

template <typename T>
struct K0Carry {
  using CN = typename CarryNum<T>::type;
  const CN* gaps;              // [2][nch]
  const Cplx<T>* agg;          // [nch][npad][4]
  const Cplx<CN>* pdec;        // [2][nch][np]
  const CN* csum;              // [nch][2]
  K0Transfer<CN>* ztr;         // [2][NZG][npad]
  K0State<CN>* zin;            // [2][NZG][npad]
  CN* zq;                      // [NZG][2] group sums, then group inputs
  CN* carry;                   // [2][nch][npad][4]
  CN* cpre;                    // [nch][2]
  CN* rtot;                    // [R][2]
};

// one chunk of a pair chain: S' = d S + S_c, H' = d (H + g S) + H_c
template <typename CN, typename T>
__device__ __forceinline__ void k0_step(CN& sr, CN& si, CN& hr, CN& hi, const Cplx<CN>& d,
                                        const CN& g, const Cplx<T>& as, const Cplx<T>& ah) {
  const CN tr = hr + g * sr, ti = hi + g * si;
  const CN nhr = d.re * tr - d.im * ti + cn_from_t(ah.re, (CN*)nullptr);
  const CN nhi = d.re * ti + d.im * tr + cn_from_t(ah.im, (CN*)nullptr);
  const CN nsr = d.re * sr - d.im * si + cn_from_t(as.re, (CN*)nullptr);
  const CN nsi = d.re * si + d.im * sr + cn_from_t(as.im, (CN*)nullptr);
  sr = nsr; si = nsi; hr = nhr; hi = nhi;
}

// phases 1 (replay = false) and 3 (replay = true)
template <typename T>
__global__ void kzero_group_kernel(K0Params Q, PairTab pr, K0Carry<T> W, bool replay) {
  using CN = typename CarryNum<T>::type;
  const CN zero = cn_zero((CN*)nullptr), one = cn_from(1.0, (CN*)nullptr);
  const int NZG = Q.rp.nzgroups, npad = Q.npad, np = pr.np;
  const int nch = Q.rp.nzchunks;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int npair = 2 * NZG * npad;
  if (e < npair) {
    const int p = e % npad, rest = e / npad;
    const int grp = rest % NZG, dir = rest / NZG;
    if (p >= np) return;
    if (!replay) {
      const RepInfo& ri = Q.rp.info[Q.rp.zgroup_rep[grp]];
      if (grp == (dir == 0 ? ri.zg0 + ri.nzg - 1 : ri.zg0)) return;   // last in its chain
    }
    const int ca = Q.rp.zgstart[grp], cb = Q.rp.zgstart[grp + 1], len = cb - ca;
    const size_t ti = ((size_t)dir * NZG + grp) * npad + p;
    CN sr = zero, si = zero, hr = zero, hi = zero, Dr = one, Di = zero, Gs = zero;
    if (replay && !Q.rp.zflat) {
      const K0State<CN> x = W.zin[ti];
      sr = x.Sr; si = x.Si; hr = x.Hr; hi = x.Hi;
    }
    constexpr int B = 8;
    for (int j0 = 0; j0 < len; j0 += B) {
      Cplx<T> as[B], ah[B];
      Cplx<CN> d[B];
      CN dz[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        if (j0 + u < len) {
          const int c = dir == 0 ? ca + j0 + u : cb - 1 - (j0 + u);
          const Cplx<T>* a = W.agg + ((size_t)c * npad + p) * 4 + 2 * dir;
          as[u] = a[0];
          ah[u] = a[1];
          d[u] = W.pdec[((size_t)dir * nch + c) * np + p];
          dz[u] = W.gaps[dir * nch + c];
        }
      }
#pragma unroll
      for (int u = 0; u < B; ++u) {
        if (j0 + u < len) {
          if (replay) {
            const int c = dir == 0 ? ca + j0 + u : cb - 1 - (j0 + u);
            CN* out = W.carry + (((size_t)dir * nch + c) * npad + p) * 4;
            out[0] = sr; out[1] = si; out[2] = hr; out[3] = hi;
          }
          k0_step(sr, si, hr, hi, d[u], dz[u], as[u], ah[u]);
          if (!replay) {
            const CN nDr = d[u].re * Dr - d[u].im * Di;
            const CN nDi = d[u].re * Di + d[u].im * Dr;
            Dr = nDr; Di = nDi;
            Gs = Gs + dz[u];
          }
        }
      }
    }
    if (!replay) W.ztr[ti] = K0Transfer<CN>{Dr, Di, Gs, sr, si, hr, hi};
  } else if (e < npair + NZG) {
    const int grp = e - npair;
    const int ca = Q.rp.zgstart[grp], cb = Q.rp.zgstart[grp + 1];
    // a replica with one group starts from zero and ends at its totals
    CN a = zero, b = zero;
    if (replay && !Q.rp.zflat) { a = W.zq[2 * grp]; b = W.zq[2 * grp + 1]; }
    constexpr int B = 8;        // loads issued ahead of the dependent sums
    for (int c0 = ca; c0 < cb; c0 += B) {
      CN s0[B], s1[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        if (c0 + u < cb) { s0[u] = W.csum[2 * (c0 + u)]; s1[u] = W.csum[2 * (c0 + u) + 1]; }
      }
#pragma unroll
      for (int u = 0; u < B; ++u) {
        if (c0 + u < cb) {
          if (replay) { W.cpre[2 * (c0 + u)] = a; W.cpre[2 * (c0 + u) + 1] = b; }
          a = a + s0[u];
          b = b + s1[u];
        }
      }
    }
    if (!replay) {
      W.zq[2 * grp] = a;
      W.zq[2 * grp + 1] = b;
    } else {
      if (Q.rp.zflat) {
        const int rep = Q.rp.zgroup_rep[grp];
        W.rtot[2 * rep] = a;
        W.rtot[2 * rep + 1] = b;
      }
    }
  }
}

// phase 2: thread = (direction, slab, pair), plus one thread per slab for
// the sums of q and q z
template <typename T>
__global__ void kzero_chain_kernel(K0Params Q, PairTab pr, K0Carry<T> W) {
  using CN = typename CarryNum<T>::type;
  const CN zero = cn_zero((CN*)nullptr);
  const int NZG = Q.rp.nzgroups, npad = Q.npad, R = Q.rp.R;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int npair = 2 * R * npad;
  if (e < npair) {
    const int p = e % npad, rest = e / npad;
    const int rep = rest % R, dir = rest / R;
    if (p >= pr.np) return;
    const int g0 = Q.rp.info[rep].zg0, ng = Q.rp.info[rep].nzg;
    CN sr = zero, si = zero, hr = zero, hi = zero;
    constexpr int B = 4;
    for (int j0 = 0; j0 < ng; j0 += B) {
      K0Transfer<CN> x[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const int j = j0 + u;
        if (j < ng - 1) {
          const int grp = dir == 0 ? g0 + j : g0 + ng - 1 - j;
          x[u] = W.ztr[((size_t)dir * NZG + grp) * npad + p];
        }
      }
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const int j = j0 + u;
        if (j < ng) {
          const int grp = dir == 0 ? g0 + j : g0 + ng - 1 - j;
          W.zin[((size_t)dir * NZG + grp) * npad + p] = K0State<CN>{sr, si, hr, hi};
          if (j < ng - 1) {
            const CN tr = hr + x[u].G * sr, ti = hi + x[u].G * si;
            const CN nhr = x[u].Dr * tr - x[u].Di * ti + x[u].Hr;
            const CN nhi = x[u].Dr * ti + x[u].Di * tr + x[u].Hi;
            const CN nsr = x[u].Dr * sr - x[u].Di * si + x[u].Sr;
            const CN nsi = x[u].Dr * si + x[u].Di * sr + x[u].Si;
            sr = nsr; si = nsi; hr = nhr; hi = nhi;
          }
        }
      }
    }
  } else if (e < npair + R) {
    const int rep = e - npair;
    const int g0 = Q.rp.info[rep].zg0, ng = Q.rp.info[rep].nzg;
    CN a = zero, b = zero;
    for (int j = 0; j < ng; ++j) {
      const int grp = g0 + j;
      const CN na = a + W.zq[2 * grp], nb = b + W.zq[2 * grp + 1];
      W.zq[2 * grp] = a;
      W.zq[2 * grp + 1] = b;
      a = na; b = nb;
    }
    W.rtot[2 * rep] = a;
    W.rtot[2 * rep + 1] = b;
  }
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
  // per chunk: z, q, dz [L0 + 1] and the potential / derivative sums
  // [2 directions][L0][2]; 2 npad lanes per chunk, lane = dir npad + pair,
  // so that the two directions' scans run side by side
  extern __shared__ __align__(16) char ksm_raw[];
  const int lanes = Q.npad, w2 = 2 * Q.npad;
  const int L0 = Q.rp.L0;
  const int nch = Q.rp.nzchunks;
  const int64_t N = Q.rp.N;
  const int lc = threadIdx.x / w2, lq = threadIdx.x % w2;
  const int dir = lq / lanes, p = lq % lanes;
  const int c = blockIdx.x * kK0Cpb + lc;
  T* zl = reinterpret_cast<T*>(ksm_raw) + (size_t)lc * (7 * L0 + 3);
  T* ql = zl + (L0 + 1);
  T* dzl = ql + (L0 + 1);
  T* accd = dzl + (L0 + 1);             // [dir][L0][2]
  bool valid = c < nch;
  CRange ch{0, 0, 0, false, false};
  if (valid) {
    ch = zchunk(Q.rp, c);
    // debug builds: a chunk outside the arrays is left out
    if (!QS_DCHECK(chunk_ok(Q.rp, ch, L0), Q.rp.status)) {
      valid = false;
      ch = CRange{0, 0, 0, false, false};
    }
  }
  const int64_t start = ch.start;
  const int cnt = ch.cnt;
  // stage the chunk; dz[cnt] is the next particle's (the backward scan's
  // first decay; 0 past the replica's end, where its carry is 0)
  for (int t = lq; t <= cnt && valid; t += w2) {
    const int64_t i = start + t;
    if (t < cnt) { zl[t] = zs[i]; ql[t] = qs[i]; }
    dzl[t] = i < N ? dz[i] : (T)0;
  }
  for (int t = lq; t < 4 * L0; t += w2) accd[t] = 0;
  __syncwarp();
  const bool act = valid && p < pr.np;
  T cwr = 0, cwi = 0, isr = 0, isi = 0, csr = 0, csi = 0, ar = 1, ai = 0;
  if (act) {
    cwr = (T)Q.cw[0][p]; cwi = (T)Q.cw[1][p];
    isr = (T)Q.is[0][p]; isi = (T)Q.is[1][p];
    csr = (T)Q.cs[0][p]; csi = (T)Q.cs[1][p];
    ar = (T)pr.a_re[p]; ai = (T)pr.a_im[p];
  }
  const T alpha = (T)Q.alpha, ialpha = (T)(1.0 / Q.alpha);
  T* acc = accd + (size_t)dir * 2 * L0;
  {
    T sr = 0, si = 0, hr = 0, hi = 0;
    if (act) {
      const CN* in = carry + (((size_t)dir * nch + c) * Q.npad + p) * 4;
      sr = cn_to_t(in[0]); si = cn_to_t(in[1]); hr = cn_to_t(in[2]); hi = cn_to_t(in[3]);
    }
    // every lane runs L0 steps so that the shuffles below see the whole
    // warp; the decays of a batch of steps are computed first (they do not
    // depend on the states), then the batch's dependent updates
    for (int n0 = 0; n0 < L0; n0 += kK0Batch) {
      Cplx<T> dd[kK0Batch];
#pragma unroll
      for (int u = 0; u < kK0Batch; ++u) {
        const int n = n0 + u;
        dd[u] = Cplx<T>{0, 0};
        if (act && n < cnt) dd[u] = cexp_neg(ar, ai, dzl[dir == 0 ? n : cnt - n]);
      }
#pragma unroll
      for (int u = 0; u < kK0Batch; ++u) {
        const int n = n0 + u;
        if (n >= L0) break;       // the same for every lane
        const bool live = n < cnt;
        const int t = dir == 0 ? n : cnt - 1 - n;
        T pot = 0, der = 0;
        if (act && live) {
          const T qq = ql[t];
          const T dzi = dzl[dir == 0 ? t : t + 1];
          const Cplx<T> d = dd[u];
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
        // sum over the direction's pair lanes (offsets below npad stay in it)
        for (int o = lanes >> 1; o; o >>= 1) {
          pot += __shfl_xor_sync(0xffffffffu, pot, o);
          der += __shfl_xor_sync(0xffffffffu, der, o);
        }
        if (p == 0 && live) { acc[2 * t] = pot; acc[2 * t + 1] = der; }
      }
    }
  }
  __syncwarp();
  // sum_j q_j |z_i - z_j| = z_i (Q< - Q>) - P< + P>, from prefix sums in the
  // carry type (the terms cancel heavily); the result stays in the carry
  // type and the combine kernel widens it to FP64. Each lane takes a segment
  // of the chunk: its sums, an exclusive scan over the lanes, then the
  // segment's particles in order. The backward lanes repeat the forward
  // lanes' scan in their own half of the chunk's lanes and write nothing.
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
  if (valid && dir == 0) {
    CN Ql = cpre[2 * c] + e0, Pl = cpre[2 * c + 1] + e1;
    const CN Qt = rtot[2 * ch.r], Pt = rtot[2 * ch.r + 1];
    const CN c1 = cn_from(Q.c1, (CN*)nullptr);
    const CN pre = cn_from(Q.rp.info[ch.r].k0pre, (CN*)nullptr);
    for (int t = ta; t < tb; ++t) {
      const int64_t i = start + t;
      const T zt = zl[t], qt = ql[t];
      const CN zc = cn_from_t(zt, (CN*)nullptr);
      const CN Qg = Qt - Ql - cn_from_t(qt, (CN*)nullptr);
      const CN Pg = cn_add_prod(Pt - Pl, -qt, zt);
      const CN lin = zc * (Ql - Qg) - Pl + Pg;
      // the two directions' sums, forward first
      const T ep = accd[2 * t] + accd[2 * L0 + 2 * t];
      const T ed = accd[2 * t + 1] + accd[2 * L0 + 2 * t + 1];
      const CN pot = c1 * lin + cn_from_t(ep, (CN*)nullptr);
      const CN der = c1 * (Ql - Qg) + cn_from_t(ed, (CN*)nullptr);
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
  for (int p = 0; p < kMaxPairs; ++p) {
    Q.cw[0][p] = Q.cw[1][p] = Q.is[0][p] = Q.is[1][p] = Q.cs[0][p] = Q.cs[1][p] = 0.0;
    if (p >= pairs.np) continue;
    // multiplicity times w_p/sqrt(pi), 1/s_p and 2/s_p + s_p
    const double sr = pairs.s_re[p], si = pairs.s_im[p];
    const double den = sr * sr + si * si;
    Q.cw[0][p] = pairs.mult[p] * pairs.w_re[p] / 1.7724538509055160;
    Q.cw[1][p] = pairs.mult[p] * pairs.w_im[p] / 1.7724538509055160;
    Q.is[0][p] = sr / den;
    Q.is[1][p] = -si / den;
    Q.cs[0][p] = 2 * sr / den + sr;
    Q.cs[1][p] = -2 * si / den + si;
  }
  for (int p = 0; p < pairs.np; ++p) {
    // c1 = sum over nodes of 2 w/(s sqrt(pi)) = sum over representatives of mult 2 Re(w/s)/sqrt(pi)
    const double den = pairs.s_re[p] * pairs.s_re[p] + pairs.s_im[p] * pairs.s_im[p];
    const double re = (pairs.w_re[p] * pairs.s_re[p] + pairs.w_im[p] * pairs.s_im[p]) / den;
    c1 += pairs.mult[p] * 2.0 * re / 1.7724538509055160;
  }
  Q.c1 = c1;
  const int nch = rp.nzchunks;
  const int NZG = rp.nzgroups;
  // work layout: agg [nch][npad][4] Cplx<T>, csum [nch][2] CN,
  // pdec [2][nch][np] Cplx<CN>, carry [2][nch][npad][4] CN, cpre [nch][2] CN,
  // rtot [R][2] CN, gaps [2][nch] CN, ztr [2][NZG][npad] K0Transfer,
  // zin [2][NZG][npad] K0State, zq [NZG][2] CN
  char* w = reinterpret_cast<char*>(work);
  auto take = [&w](size_t b) { char* r = w; w += (b + 255) & ~size_t(255); return r; };
  Cplx<T>* agg = reinterpret_cast<Cplx<T>*>(take(sizeof(Cplx<T>) * (size_t)nch * npad * 4));
  CN* csum = reinterpret_cast<CN*>(take(sizeof(CN) * (size_t)nch * 2));
  Cplx<CN>* pdec = reinterpret_cast<Cplx<CN>*>(take(sizeof(Cplx<CN>) * (size_t)2 * nch * pairs.np));
  CN* carry = reinterpret_cast<CN*>(take(sizeof(CN) * (size_t)2 * nch * npad * 4));
  CN* cpre = reinterpret_cast<CN*>(take(sizeof(CN) * (size_t)nch * 2));
  CN* rtot = reinterpret_cast<CN*>(take(sizeof(CN) * (size_t)rp.R * 2));
  CN* gaps = reinterpret_cast<CN*>(take(sizeof(CN) * (size_t)2 * nch));
  K0Carry<T> W;
  W.gaps = gaps;
  W.agg = agg;
  W.pdec = pdec;
  W.csum = csum;
  W.ztr = reinterpret_cast<K0Transfer<CN>*>(take(sizeof(K0Transfer<CN>) * (size_t)2 * NZG * npad));
  W.zin = reinterpret_cast<K0State<CN>*>(take(sizeof(K0State<CN>) * (size_t)2 * NZG * npad));
  W.zq = reinterpret_cast<CN*>(take(sizeof(CN) * (size_t)NZG * 2));
  W.carry = carry;
  W.cpre = cpre;
  W.rtot = rtot;
  CN* phi0 = static_cast<CN*>(phi0v);
  CN* fz0 = static_cast<CN*>(fz0v);
  const int nblk = (nch + kK0Cpb - 1) / kK0Cpb;
  const int thr = npad * kK0Cpb;      // whole warps for npad >= 4
  const size_t sma = (size_t)kK0Cpb * 2 * rp.L0 * sizeof(T);
  cudaFuncSetAttribute(kzero_aggregate_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sma);
  kzero_aggregate_kernel<T><<<nblk, thr, sma, st>>>(Q, pairs, zs, qs, agg, csum);
  launch_pair_decay<T>(rp, 1, pairs.np, zs, pairs, pdec, gaps, st);
  const int ng1 = 2 * NZG * npad + NZG;
  if (!rp.zflat) {
    kzero_group_kernel<T><<<(ng1 + 127) / 128, 128, 0, st>>>(Q, pairs, W, false);
    const int ng2 = 2 * rp.R * npad + rp.R;
    kzero_chain_kernel<T><<<(ng2 + 127) / 128, 128, 0, st>>>(Q, pairs, W);
  }
  // with one group per replica this replay from zero is the whole scan
  kzero_group_kernel<T><<<(ng1 + 127) / 128, 128, 0, st>>>(Q, pairs, W, true);
  const size_t smf = (size_t)kK0Cpb * (7 * rp.L0 + 3) * sizeof(T);
  cudaFuncSetAttribute(kzero_final_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf);
  kzero_final_kernel<T><<<nblk, 2 * thr, smf, st>>>(Q, pairs, zs, dz, qs, carry, cpre, rtot, phi0,
                                                fz0);
}

size_t kzero_work_doubles(int nzchunks, int nzgroups, int R, int np) {
  const int npad = kzero_lanes(np);
  // in 8-byte units (a double-float takes one), with room for the 256-byte
  // alignment of each of the 10 arrays
  return (size_t)nzchunks * npad * 4 * 2 + (size_t)nzchunks * 2 +
         (size_t)2 * nzchunks * kMaxPairs * 2 + (size_t)2 * nzchunks * npad * 4 +
         (size_t)nzchunks * 2 + (size_t)R * 2 + (size_t)2 * nzchunks +
         (size_t)2 * nzgroups * npad * (7 + 4) + (size_t)nzgroups * 2 + 10 * 32 + 64;
}

// ============================================================ instantiations
template void launch_kzero<float>(const Reps&, const PairTab&, double, const float*, const float*,
                                  const float*, double*, void*, void*, cudaStream_t);
template void launch_kzero<double>(const Reps&, const PairTab&, double, const double*,
                                   const double*, const double*, double*, void*, void*,
                                   cudaStream_t);

}  // namespace qslab
