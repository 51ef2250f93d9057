// qslab device kernels: input checks and sort keys, the sorted gather, the
// k != 0 SOE scans (chunk aggregates, carries, bidirectional recurrences with
// the fused potential/force gather), the k = 0 term, the final combine and
// the random-batch k-sampler.
//
// Method: Gan, Gao, Liang, Xu, "Fast algorithm for quasi-2D Coulomb systems".
// For a mode k and beta in {k, alpha s_1, ..., alpha s_M} the pair sums over
// j < i and j > i of u_j e^{-beta |z_i - z_j|}, u_j = q_j e^{-i k.rho_j}, are
// first-order linear recurrences over the z-sorted particles (Eqs. 3.28-3.30,
// Remark 3.3). Forces need both directions (Appendix E). Here the sorted
// particles are cut into chunks of L; one CTA owns one chunk and a range of
// modes, one thread one mode:
//   pass A   chunk aggregates sum_j u_j e^{-beta(z_end - z_j)} (forward) and
//            sum_j u_j e^{-beta(z_j - z_start)} (backward), by dot products
//            with k-independent exponential tables kept in shared memory;
//   carries  an FP64 recurrence over chunks per (mode, beta, direction);
//   pass B   the recurrences over the chunk from the carried state, with the
//            gather of Eq. 3.21 / Appendix E fused: per particle and mode the
//            potential and force contributions are formed, summed over the
//            warp's 32 modes by shuffles and over warps in shared memory.
// SOE nodes come in conjugate pairs; one representative a_p per pair drives
// two complex states, fed by the real inputs q cos(k.rho) and q sin(k.rho),
// whose combination 2 Re(c F(a)) - 2i Re(c F(b)) equals the pair's
// contribution (the conjugate partner needs no scan of its own).
#include <cstdint>
#include <cuda_runtime.h>

#include "qslab_df.cuh"
#include "qslab_geom.cuh"
#include "qslab_internal.h"
#include "qslab_math.cuh"

namespace qslab {

// ============================================================ k != 0 scans

// Shared-memory layout of one chunk: L particle records (plus one more whose
// dz belongs to the next chunk's first particle), the exponential tables in
// particle-major order (all pairs of one particle are contiguous), and in
// pass B the per-warp output slots.
template <typename T>
struct __align__(4 * sizeof(T)) Rec {
  typename PhaseT<T>::type xh, yh;   // fixed-point x/Lx, y/Ly
  T q, dz;
};

template <typename T>
struct ChunkSmem {
  Cplx<T>* tab;   // pass B: [L+1][NP] decays; pass A: [L][2][NP] (E_f, E_b)
  Rec<T>* rec;    // [L+1]
  T* zl;          // [L]
  float2* trig;   // FP32 path: [256] (cos, sin) of j/256 turns
  T* slots;       // pass B: [W][L][4]
  T* idle;        // pass B: [W][32] write targets of lanes that hold no output
};
constexpr int kTrig = 256;

__host__ __device__ inline size_t align_up(size_t x) { return (x + 31) & ~size_t(31); }

template <typename T>
__host__ __device__ inline size_t chunk_smem_bytes(int L, int NP, int W, bool passB) {
  size_t b = 0;
  b += align_up(sizeof(Cplx<T>) * (size_t)NP * (passB ? (L + 1) : 2 * L));
  b += align_up(sizeof(Rec<T>) * (L + 1));
  b += align_up(sizeof(T) * L);
  b += align_up(sizeof(float2) * kTrig);
  if (passB) b += align_up(sizeof(T) * (size_t)W * L * 4) + align_up(sizeof(T) * (size_t)W * kWarp);
  return b;
}

template <typename T>
__device__ inline ChunkSmem<T> carve(char* base, int L, int NP, int W, bool passB) {
  ChunkSmem<T> s;
  char* p = base;
  s.tab = reinterpret_cast<Cplx<T>*>(p);
  p += align_up(sizeof(Cplx<T>) * (size_t)NP * (passB ? (L + 1) : 2 * L));
  s.rec = reinterpret_cast<Rec<T>*>(p); p += align_up(sizeof(Rec<T>) * (L + 1));
  s.zl = reinterpret_cast<T*>(p); p += align_up(sizeof(T) * L);
  s.trig = reinterpret_cast<float2*>(p); p += align_up(sizeof(float2) * kTrig);
  s.slots = passB ? reinterpret_cast<T*>(p) : nullptr;
  if (passB) p += align_up(sizeof(T) * (size_t)W * L * 4);
  s.idle = passB ? reinterpret_cast<T*>(p) : nullptr;
  return s;
}

template <typename T>
struct KParams {
  ScanPlan plan;
  Reps rp;
  ModeTab<T> modes;
  size_t kstride;   // R * Kpad: stride between the planes of modes.cp
  const T* zs;
  const T* dz;
  const T* qs;
  const typename PhaseT<T>::type* xh;
  const typename PhaseT<T>::type* yh;
  const float2* trig;  // [256] (cos, sin) of j/256 turns (FP32 path)
  Cplx<T>* agg;     // [2][nchunks][nstates][Kpad]
  Cplx<T>* carry;   // same layout
  T* part;          // [nkr][4][N]
};

// Per-thread (per-mode) coefficients.
template <typename T, int NP>
struct ModeCoef {
  int32_t mx, my;
  T kx, ky, kk, ck, ckk, sY, sZ;
  T cpr[NP], cpi[NP], cbr[NP], cbi[NP];
};

template <typename T, int NP>
__device__ __forceinline__ void load_mode(const ModeTab<T>& mt, size_t kstride, size_t m,
                                          ModeCoef<T, NP>& c) {
  c.mx = mt.mx[m]; c.my = mt.my[m];
  c.kx = mt.kx[m]; c.ky = mt.ky[m]; c.kk = mt.kk[m];
  c.ck = mt.ck[m]; c.ckk = mt.ckk[m]; c.sY = mt.sY[m]; c.sZ = mt.sZ[m];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    c.cpr[p] = mt.cp[(0 * NP + p) * kstride + m];
    c.cpi[p] = mt.cp[(1 * NP + p) * kstride + m];
    c.cbr[p] = mt.cp[(2 * NP + p) * kstride + m];
    c.cbi[p] = mt.cp[(3 * NP + p) * kstride + m];
  }
}

// Load the chunk's particles into shared memory.
template <typename T>
__device__ inline void load_chunk(const KParams<T>& P, ChunkSmem<T>& s,
                                  int64_t start, int cnt) {
  const int64_t N = P.rp.N;
  for (int t = threadIdx.x; t <= cnt; t += blockDim.x) {
    const int64_t i = start + t;
    Rec<T> r;
    r.dz = (i < N) ? P.dz[i] : (T)0;
    if (t < cnt) {
      r.xh = P.xh[i];
      r.yh = P.yh[i];
      r.q = P.qs[i];
      s.zl[t] = P.zs[i];
    } else {
      r.xh = 0; r.yh = 0; r.q = 0;
    }
    s.rec[t] = r;
  }
  if (P.trig)
    for (int t = threadIdx.x; t < kTrig; t += blockDim.x) s.trig[t] = P.trig[t];
}

// ------------------------------------------------------------------ pass A
// the two table entries of a pair (16 bytes on the FP32 path: one load)
__device__ __forceinline__ void load_pair(const Cplx<float>* e, Cplx<float>& a, Cplx<float>& b) {
  const float4 v = *reinterpret_cast<const float4*>(e);
  a = Cplx<float>{v.x, v.y};
  b = Cplx<float>{v.z, v.w};
}
__device__ __forceinline__ void load_pair(const Cplx<double>* e, Cplx<double>& a,
                                          Cplx<double>& b) {
  a = e[0];
  b = e[1];
}

template <typename T, int NP>
__global__ void kspace_aggregate_kernel(KParams<T> P, PairTab pairs) {
  extern __shared__ __align__(32) char smem[];
  const ScanPlan& pl = P.plan;
  const int c = blockIdx.x;
  const CRange ch = kchunk(P.rp, c);
  if (!QS_DCHECK(chunk_ok(P.rp, ch, P.rp.L), P.rp.status)) return;
  const int64_t start = ch.start;
  const int cnt = ch.cnt;
  const int Kpad = P.rp.Kpad;
  ChunkSmem<T> s = carve<T>(smem, P.rp.L, NP, 0, false);
  load_chunk<T>(P, s, start, cnt);
  __syncthreads();
  // E tables: [t][p][0] = e^{-a_p (z_end - z_t)}, [t][p][1] = e^{-a_p (z_t - z_start)}
  // (a pair's two entries adjacent: one 16-byte load on the FP32 path)
  const T zend = s.zl[cnt - 1], zst = s.zl[0];
  for (int e = threadIdx.x; e < NP * cnt; e += blockDim.x) {
    const int t = e / NP, p = e - t * NP;
    const T ar = (T)pairs.a_re[p], ai = (T)pairs.a_im[p];
    s.tab[2 * (t * NP + p)] = cexp_neg(ar, ai, zend - s.zl[t]);
    s.tab[2 * (t * NP + p) + 1] = cexp_neg(ar, ai, s.zl[t] - zst);
  }
  __syncthreads();
  const int m = blockIdx.y * pl.KR + threadIdx.x;
  ModeCoef<T, NP> mc;
  load_mode<T, NP>(P.modes, P.kstride, (size_t)ch.r * Kpad + m, mc);
  Cplx<T> f0 = {0, 0}, b0 = {0, 0};
  Cplx<T> fa[NP], fb[NP], ba[NP], bb[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) fa[p] = fb[p] = ba[p] = bb[p] = Cplx<T>{0, 0};
  for (int t = 0; t < cnt; ++t) {
    const Rec<T> r = s.rec[t];
    T cs, sn;
    phase_cs(phase_turns(mc.mx, mc.my, r.xh, r.yh), s.trig, cs, sn);
    const T a = r.q * cs, b = r.q * sn;   // u = a - i b
    const T zt = s.zl[t];
    const T ef = exp_neg_term(mc.kk * (zend - zt));
    const T eb = exp_neg_term(mc.kk * (zt - zst));
    f0.re = fma(ef, a, f0.re); f0.im = fma(-ef, b, f0.im);
    b0.re = fma(eb, a, b0.re); b0.im = fma(-eb, b, b0.im);
    const Cplx<T>* Et = s.tab + 2 * t * NP;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      Cplx<T> Ef, Eb;
      load_pair(Et + 2 * p, Ef, Eb);
      fa[p].re = fma(Ef.re, a, fa[p].re); fa[p].im = fma(Ef.im, a, fa[p].im);
      fb[p].re = fma(Ef.re, b, fb[p].re); fb[p].im = fma(Ef.im, b, fb[p].im);
      ba[p].re = fma(Eb.re, a, ba[p].re); ba[p].im = fma(Eb.im, a, ba[p].im);
      bb[p].re = fma(Eb.re, b, bb[p].re); bb[p].im = fma(Eb.im, b, bb[p].im);
    }
  }
  const int S = pl.nstates;
  const size_t dirstride = (size_t)P.rp.nchunks * S * Kpad;
  Cplx<T>* af = P.agg + ((size_t)c * S) * Kpad + m;
  Cplx<T>* ab = af + dirstride;
  af[0] = f0;
  ab[0] = b0;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    af[(size_t)(1 + 2 * p) * Kpad] = fa[p];
    af[(size_t)(2 + 2 * p) * Kpad] = fb[p];
    ab[(size_t)(1 + 2 * p) * Kpad] = ba[p];
    ab[(size_t)(2 + 2 * p) * Kpad] = bb[p];
  }
}

// ------------------------------------------------ pass A on the tensor cores
// On the FP32 path the chunk aggregates are one matrix product per chunk:
// rows (mode, a | b), a = q cos(k.rho) and b = q sin(k.rho) of each particle;
// columns (direction, pair, re | im) of the exponential tables
// E_f(t, p) = e^{-a_p (z_end - z_t)} and E_b(t, p) = e^{-a_p (z_t - z_start)};
// the sum runs over the chunk's particles t. It runs as mma.sync m16n8k8
// TF32 products at FP32-level accuracy: each operand x = x_hi + x_lo with
// x_hi = x rounded to 11 significant bits (exact in TF32) and x_lo = x - x_hi
// (exact) rounded to TF32, and the product as a_hi b_hi + a_hi b_lo +
// a_lo b_hi (the dropped a_lo b_lo is below 2^-22 of it). Eight k-steps (64
// particles) accumulate in the MMA's FP32 accumulators and are then added to
// FP32 sums in registers: measured RMS error 3.5e-8 of sum |a E| over 480
// particles, as for sequential FP32 FMAs (one accumulator over all 60
// k-steps: 2.5e-7). The beta = k term, whose exponent depends on the mode,
// stays scalar.
//
// A warp owns 32 modes and runs them in passes over the chunk of MT m-tiles
// of 8 modes (two halves of 16 up to 8 pairs, four quarters of 8 above):
// rows g = the a-state and g + 8 = the b-state of mode g. A lane
// (group g = lane / 4, q4 = lane % 4) forms the phases of its m-tiles' mode g
// at particles k0 + q4 and k0 + q4 + 4 of each k-step, which are exactly its
// A-fragment entries; its accumulators hold columns 2 q4, 2 q4 + 1 of each
// n-tile: the (re, im) of one (direction, pair) for the a- and the b-state.
// The E table rows have a stride of 4 NP + 8 floats, so that the B-fragment
// loads (row k0 + q4 (+4), column 8 j + g) hit 32 different banks.

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// x = hi + lo, both TF32: hi by Dekker's split with 2^13 + 1 (x rounded to
// its 11 leading significant bits, exact in TF32; FP32 pipe operations, for
// |x| < 4e34), lo = x - hi (exact) rounded to TF32 (measured 3% faster than
// rounding hi with the conversion instruction as well)
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  const float c = __fmul_rn(x, 8193.0f);
  const float h = __fsub_rn(c, __fsub_rn(c, x));
  hi = __float_as_uint(h);
  lo = tf32_rna(__fsub_rn(x, h));
}
// d += a b (16 x 8 x 8, TF32 inputs, FP32 accumulation)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// shared memory of the tensor-core pass A: E table [L8][4 NP + 8] (L8: L
// rounded up to whole k-steps of 8), records [L + 1], z [L], sin/cos table
__host__ __device__ inline size_t tc_agg_smem_bytes(int L, int NP) {
  const size_t L8 = ((size_t)L + 7) & ~(size_t)7;
  return align_up(sizeof(float) * L8 * (4 * NP + 8)) + align_up(sizeof(Rec<float>) * (L + 1)) +
         align_up(sizeof(float) * L) + align_up(sizeof(float2) * kTrig);
}

template <int NP>
__global__ void kspace_aggregate_tc_kernel(KParams<float> P, PairTab pairs) {
  extern __shared__ __align__(32) char smem[];
  constexpr int NC = 4 * NP;        // columns: direction, pair, re | im
  constexpr int NS = NC + 8;        // E table row stride (floats)
  constexpr int NT = NC / 8;        // n-tiles
  constexpr int KB = 8;             // k-steps accumulated in the MMA before an FP32 add
  // m-tiles (8 modes each) in flight per pass over the chunk: two up to 8
  // pairs, one above (register budget)
  constexpr int MT = NP <= 8 ? 2 : 1, MB = 8 * MT;
  const ScanPlan& pl = P.plan;
  const int c = blockIdx.x;
  const int L = P.rp.L, Kpad = P.rp.Kpad;
  const CRange ch = kchunk(P.rp, c);
  if (!QS_DCHECK(chunk_ok(P.rp, ch, L), P.rp.status)) return;
  const int64_t start = ch.start;
  const int cnt = ch.cnt;
  const int cnt8 = (cnt + 7) & ~7;  // whole k-steps: at most L rounded up to 8
  float* etab = reinterpret_cast<float*>(smem);
  ChunkSmem<float> s;
  {
    char* p = smem + align_up(sizeof(float) * ((size_t)(L + 7) & ~(size_t)7) * NS);
    s.tab = nullptr;
    s.rec = reinterpret_cast<Rec<float>*>(p); p += align_up(sizeof(Rec<float>) * (L + 1));
    s.zl = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * L);
    s.trig = reinterpret_cast<float2*>(p);
    s.slots = s.idle = nullptr;
  }
  load_chunk<float>(P, s, start, cnt);
  __syncthreads();
  // E table; rows cnt..cnt8-1 zero (their a, b are zero too)
  const float zend = s.zl[cnt - 1], zst = s.zl[0];
  for (int e = threadIdx.x; e < NP * cnt8; e += blockDim.x) {
    const int t = e / NP, p = e - t * NP;
    Cplx<float> ef = {0.0f, 0.0f}, eb = {0.0f, 0.0f};
    if (t < cnt) {
      const float ar = (float)pairs.a_re[p], ai = (float)pairs.a_im[p];
      ef = cexp_neg(ar, ai, zend - s.zl[t]);
      eb = cexp_neg(ar, ai, s.zl[t] - zst);
    }
    float* row = etab + (size_t)t * NS;
    row[2 * p] = ef.re;
    row[2 * p + 1] = ef.im;
    row[2 * NP + 2 * p] = eb.re;
    row[2 * NP + 2 * p + 1] = eb.im;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, q4 = lane & 3;
  const int Kr = P.rp.info[ch.r].K;
  const int S = pl.nstates;
  const size_t dirstride = (size_t)P.rp.nchunks * S * Kpad;
  Cplx<float>* af = P.agg + ((size_t)c * S) * Kpad;
  const size_t mrow = (size_t)ch.r * Kpad;
  for (int h = 0; h < kWarp / MB; ++h) {
    const int mb = blockIdx.y * pl.KR + w * kWarp + h * MB;   // first mode of the pass
    if (mb >= Kr) {
      // padding only: zero aggregates (the carries read every mode)
      for (int e = lane; e < 2 * S * MB; e += kWarp) {
        const int m = mb + e % MB, st = (e / MB) % S, dir = (e / MB) / S;
        af[dir * dirstride + (size_t)st * Kpad + m] = Cplx<float>{0.0f, 0.0f};
      }
      continue;
    }
    int32_t mx[MT], my[MT];
    float kk[MT];
#pragma unroll
    for (int i = 0; i < MT; ++i) {
      const size_t m = mrow + mb + 8 * i + g;
      mx[i] = P.modes.mx[m]; my[i] = P.modes.my[m]; kk[i] = P.modes.kk[m];
    }
    float run[MT][NT][4];
    Cplx<float> f0[MT], b0[MT];
#pragma unroll
    for (int i = 0; i < MT; ++i) {
      f0[i] = b0[i] = Cplx<float>{0.0f, 0.0f};
#pragma unroll
      for (int j = 0; j < NT; ++j) run[i][j][0] = run[i][j][1] = run[i][j][2] = run[i][j][3] = 0.0f;
    }
    for (int kb = 0; kb < cnt8; kb += 8 * KB) {
      float fr[MT][NT][4];
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j) fr[i][j][0] = fr[i][j][1] = fr[i][j][2] = fr[i][j][3] = 0.0f;
      const int kend = min(kb + 8 * KB, cnt8);
      for (int k0 = kb; k0 < kend; k0 += 8) {
        // B fragments: rows k0 + q4 and k0 + q4 + 4, column 8 j + g
        uint32_t bh[NT][2], bl[NT][2];
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
          for (int r = 0; r < 2; ++r)
            tf32_split(etab[(size_t)(k0 + q4 + 4 * r) * NS + 8 * j + g], bh[j][r], bl[j][r]);
#pragma unroll
        for (int i = 0; i < MT; ++i) {
          uint32_t ah[4], al[4];
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const int t = k0 + q4 + 4 * r;
            const int tc = t < cnt ? t : cnt - 1;
            const Rec<float> rr = s.rec[tc];
            float cs, sn;
            phase_cs(phase_turns(mx[i], my[i], rr.xh, rr.yh), s.trig, cs, sn);
            const float qv = t < cnt ? rr.q : 0.0f;
            const float a = qv * cs, b = qv * sn;   // u = a - i b
            const float zt = s.zl[tc];
            const float ef = exp_neg_term(kk[i] * (zend - zt));
            const float eb = exp_neg_term(kk[i] * (zt - zst));
            f0[i].re = fmaf(ef, a, f0[i].re); f0[i].im = fmaf(-ef, b, f0[i].im);
            b0[i].re = fmaf(eb, a, b0[i].re); b0[i].im = fmaf(-eb, b, b0[i].im);
            // A fragment: (row g, col q4) a(t0), (g + 8, q4) b(t0), (g, q4 + 4) a(t1), (g + 8, q4 + 4) b(t1)
            tf32_split(a, ah[2 * r], al[2 * r]);
            tf32_split(b, ah[2 * r + 1], al[2 * r + 1]);
          }
          // the three products (NT independent MMAs between dependent ones)
#pragma unroll
          for (int j = 0; j < NT; ++j) mma_tf32(fr[i][j], al, bh[j][0], bh[j][1]);
#pragma unroll
          for (int j = 0; j < NT; ++j) mma_tf32(fr[i][j], ah, bl[j][0], bl[j][1]);
#pragma unroll
          for (int j = 0; j < NT; ++j) mma_tf32(fr[i][j], ah, bh[j][0], bh[j][1]);
        }
      }
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
          for (int e = 0; e < 4; ++e) run[i][j][e] += fr[i][j][e];
    }
    // the beta = k sums over the mode's four lanes
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int o = 1; o < 4; o <<= 1) {
        f0[i].re += __shfl_xor_sync(0xffffffffu, f0[i].re, o);
        f0[i].im += __shfl_xor_sync(0xffffffffu, f0[i].im, o);
        b0[i].re += __shfl_xor_sync(0xffffffffu, b0[i].re, o);
        b0[i].im += __shfl_xor_sync(0xffffffffu, b0[i].im, o);
      }
#pragma unroll
    for (int i = 0; i < MT; ++i) {
      const int m = mb + 8 * i + g;
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int n = 8 * j + 2 * q4;              // columns n (re) and n + 1 (im)
        const int dir = n / (2 * NP), p = (n - dir * 2 * NP) >> 1;
        Cplx<float>* base = af + dir * dirstride + m;
        base[(size_t)(1 + 2 * p) * Kpad] = Cplx<float>{run[i][j][0], run[i][j][1]};   // sum a E
        base[(size_t)(2 + 2 * p) * Kpad] = Cplx<float>{run[i][j][2], run[i][j][3]};   // sum b E
      }
      if (q4 == 0) {
        af[m] = f0[i];
        af[dirstride + m] = b0[i];
      }
    }
  }
}

// ------------------------------------------------------------------ pass B
template <typename T, int NP>
__global__ void kspace_final_kernel(KParams<T> P, PairTab pairs) {
  extern __shared__ __align__(32) char smem[];
  const ScanPlan& pl = P.plan;
  const int c = blockIdx.x;
  const int W = pl.KR / kWarp;
  const int L = P.rp.L, Kpad = P.rp.Kpad;
  const CRange ch = kchunk(P.rp, c);
  if (!QS_DCHECK(chunk_ok(P.rp, ch, L), P.rp.status)) return;
  const int64_t start = ch.start;
  const int cnt = ch.cnt;
  ChunkSmem<T> s = carve<T>(smem, L, NP, W, true);
  load_chunk<T>(P, s, start, cnt);
  __syncthreads();
  // per-step decays [t][p] = e^{-a_p dz_t}, t = 0..cnt (t = cnt: next chunk)
  for (int e = threadIdx.x; e < NP * (cnt + 1); e += blockDim.x) {
    const int t = e / NP, p = e - t * NP;
    s.tab[t * NP + p] = cexp_neg((T)pairs.a_re[p], (T)pairs.a_im[p], s.rec[t].dz);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int m = blockIdx.y * pl.KR + threadIdx.x;
  ModeCoef<T, NP> mc;
  load_mode<T, NP>(P.modes, P.kstride, (size_t)ch.r * Kpad + m, mc);
  const int S = pl.nstates;
  const size_t dirstride = (size_t)P.rp.nchunks * S * Kpad;
  T* slot = s.slots + (size_t)w * L * 4;

  for (int dir = 0; dir < 2; ++dir) {
    const Cplx<T>* cin = P.carry + dir * dirstride + ((size_t)c * S) * Kpad + m;
    Cplx<T> g0 = cin[0];
    Cplx<T> ga[NP], gb[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      ga[p] = cin[(size_t)(1 + 2 * p) * Kpad];
      gb[p] = cin[(size_t)(2 + 2 * p) * Kpad];
    }
    const T zsign = dir == 0 ? (T)1 : (T)-1;
    for (int n0 = 0; n0 < cnt; n0 += 4) {
      T buf[16];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = n0 + j;
        if (n < cnt) {
          const int t = dir == 0 ? n : cnt - 1 - n;
          const int td = dir == 0 ? t : t + 1;      // index of the decay to apply
          const Rec<T> r = s.rec[t];
          const T dzd = dir == 0 ? r.dz : s.rec[td].dz;
          T cs, sn;
          phase_cs(phase_turns(mc.mx, mc.my, r.xh, r.yh), s.trig, cs, sn);
          const T a = r.q * cs, b = r.q * sn;
          // beta = k: real decay e^{-k dz}, complex input u = a - i b, as
          // G <- G + (u - e G) with e = 1 - e^{-k dz} (see one_minus_exp_neg)
          const T ek = one_minus_exp_neg(mc.kk * dzd);
          g0.re += fma(-ek, g0.re, a);
          g0.im += fma(-ek, g0.im, -b);
          T Yr = mc.ck * g0.re, Yi = mc.ck * g0.im;
          T Zr = mc.ckk * g0.re, Zi = mc.ckk * g0.im;
          const Cplx<T>* dt = s.tab + td * NP;
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            const Cplx<T> d = dt[p];
            const T ar = fma(d.re, ga[p].re, fma(-d.im, ga[p].im, a));
            const T ai = fma(d.re, ga[p].im, d.im * ga[p].re);
            const T br = fma(d.re, gb[p].re, fma(-d.im, gb[p].im, b));
            const T bi = fma(d.re, gb[p].im, d.im * gb[p].re);
            ga[p].re = ar; ga[p].im = ai; gb[p].re = br; gb[p].im = bi;
            Yr = fma(mc.cpr[p], ar, fma(-mc.cpi[p], ai, Yr));
            Yi = fma(-mc.cpr[p], br, fma(mc.cpi[p], bi, Yi));
            Zr = fma(mc.cbr[p], ar, fma(-mc.cbi[p], ai, Zr));
            Zi = fma(-mc.cbr[p], br, fma(mc.cbi[p], bi, Zi));
          }
          // the sums above include j = i; remove it (coefficients sY, sZ times u_i)
          Yr = fma(-mc.sY, a, Yr); Yi = fma(mc.sY, b, Yi);
          Zr = fma(-mc.sZ, a, Zr); Zi = fma(mc.sZ, b, Zi);
          const T W2 = cs * Yi + sn * Yr;         // Im e^{i k.rho} Y
          buf[4 * j + 0] = cs * Yr - sn * Yi;     // Re e^{i k.rho} Y
          buf[4 * j + 1] = mc.kx * W2;
          buf[4 * j + 2] = mc.ky * W2;
          buf[4 * j + 3] = zsign * (cs * Zr - sn * Zi);   // Re e^{i k.rho} Z
        } else {
          buf[4 * j + 0] = buf[4 * j + 1] = buf[4 * j + 2] = buf[4 * j + 3] = (T)0;
        }
      }
      const T v = warp_reduce16<T>(buf, lane);
      // every even lane now holds one (particle, quantity) total; all lanes
      // store (the others into an idle row) so that the warp does not diverge
      const int idx = lane >> 1, g = idx >> 2, qn = idx & 3;
      const bool own = !(lane & 1) && n0 + g < cnt;
      const int tt = dir == 0 ? n0 + g : cnt - 1 - (n0 + g);
      T* dst = own ? slot + tt * 4 + qn : s.idle + w * kWarp + lane;
      *dst = (dir == 0 ? (T)0 : *dst) + v;
    }
    __syncwarp();
  }
  __syncthreads();
  // sum the warps' slots and write this mode range's partial outputs
  T* out = P.part + (size_t)blockIdx.y * 4 * P.rp.N;
  for (int e = threadIdx.x; e < cnt * 4; e += blockDim.x) {
    const int t = e >> 2, qn = e & 3;
    T acc = 0;
    for (int ww = 0; ww < W; ++ww) acc += s.slots[((size_t)ww * L + t) * 4 + qn];
    out[(size_t)qn * P.rp.N + start + t] = acc;
  }
}

// ------------------------------------------------ pass B, packed FP32 form
// The same recurrences and gather on the FP32 path with two SOE pairs per
// 64-bit register: the sm_100-family packed FP32 instructions (__ffma2_rn,
// __fmul2_rn: two IEEE FMAs / products in one instruction) run the 16
// operations per pair and step as 8, which halves the issue slots of the
// arithmetic core. The pair (p, p+1) states sit in the two lanes of a float2;
// the decay table is stored re/im-split per particle so that the decays of
// two pairs load as one float2; the potential and force sums keep one
// partial sum per lane, added at the end of the step.
// Coefficients of the pairs one lane carries: NQ pair groups (two pairs per
// float2) of one mode, from group q0 on. A lane that carries the whole mode
// (NQ = NP/2) takes the mode table's j = i sums; a lane that carries part of
// it forms the partial sums of its own pairs the same way (FP64 sum of the
// FP32-rounded coefficients, one rounding), and only the mode's lead lane
// carries the beta = k coefficients ck, ckk.
template <int NQ>
struct ModeCoefF2 {
  int32_t mx, my;
  float kx, ky, kk, ck, ckk, sY, sZ;
  float2 cpr[NQ], ncpi[NQ], cbr[NQ], ncbi[NQ];   // ncpi = -cpi, ncbi = -cbi
};

template <int NP, int NQ>
__device__ __forceinline__ void load_mode_f2(const ModeTab<float>& mt, size_t kstride, size_t m,
                                             int q0, bool lead, ModeCoefF2<NQ>& c) {
  c.mx = mt.mx[m]; c.my = mt.my[m];
  c.kx = mt.kx[m]; c.ky = mt.ky[m]; c.kk = mt.kk[m];
  c.ck = lead ? mt.ck[m] : 0.0f;
  c.ckk = lead ? mt.ckk[m] : 0.0f;
  double sy = 0.0, sz = 0.0;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int p0 = 2 * (q0 + q), p1 = p0 + 1;
    c.cpr[q] = make_float2(mt.cp[(0 * NP + p0) * kstride + m], mt.cp[(0 * NP + p1) * kstride + m]);
    c.ncpi[q] = make_float2(-mt.cp[(1 * NP + p0) * kstride + m], -mt.cp[(1 * NP + p1) * kstride + m]);
    c.cbr[q] = make_float2(mt.cp[(2 * NP + p0) * kstride + m], mt.cp[(2 * NP + p1) * kstride + m]);
    c.ncbi[q] = make_float2(-mt.cp[(3 * NP + p0) * kstride + m], -mt.cp[(3 * NP + p1) * kstride + m]);
    sy += (double)c.cpr[q].x; sy += (double)c.cpr[q].y;
    sz += (double)c.cbr[q].x; sz += (double)c.cbr[q].y;
  }
  if (NQ == NP / 2) {
    c.sY = mt.sY[m]; c.sZ = mt.sZ[m];
  } else {
    c.sY = (float)((double)c.ck + sy);
    c.sZ = (float)((double)c.ckk + sz);
  }
}

// A lane's recurrence states: the beta = k state and, per pair group, the
// a- and b-states of two pairs (re and im parts split over two float2).
template <int NQ>
struct F2State {
  Cplx<float> g0;
  float2 Ra[NQ], Ia[NQ], Rb[NQ], Ib[NQ];
};

// the carried states of one direction (cin: the chunk's state 0 of this mode)
template <int NQ>
__device__ __forceinline__ void f2_load_state(const Cplx<float>* cin, int Kpad, int q0,
                                              F2State<NQ>& st) {
  st.g0 = cin[0];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int qq = q0 + q;
    const Cplx<float> a0 = cin[(size_t)(1 + 4 * qq) * Kpad], b0 = cin[(size_t)(2 + 4 * qq) * Kpad];
    const Cplx<float> a1 = cin[(size_t)(3 + 4 * qq) * Kpad], b1 = cin[(size_t)(4 + 4 * qq) * Kpad];
    st.Ra[q] = make_float2(a0.re, a1.re); st.Ia[q] = make_float2(a0.im, a1.im);
    st.Rb[q] = make_float2(b0.re, b1.re); st.Ib[q] = make_float2(b0.im, b1.im);
  }
}

// One step of a lane's recurrences at particle record r (dzd: the distance
// its decays span; dre, dim: their re and im rows from this lane's first
// pair group) and the lane's four output terms of that particle:
// Re e^{ik.rho} Y, kx and ky times Im e^{ik.rho} Y, zsign Re e^{ik.rho} Z.
template <int NQ>
__device__ __forceinline__ void f2_step(F2State<NQ>& st, const ModeCoefF2<NQ>& mc,
                                        const Rec<float>& r, float dzd, const float2* trig,
                                        const float2* dre, const float2* dim, float zsign,
                                        float* out) {
  const float2 minus1 = make_float2(-1.0f, -1.0f);
  float cs, sn;
  phase_cs(phase_turns(mc.mx, mc.my, r.xh, r.yh), trig, cs, sn);
  const float a = r.q * cs, b = r.q * sn;
  // beta = k: as in the scalar kernel
  const float ek = one_minus_exp_neg(mc.kk * dzd);
  st.g0.re += fmaf(-ek, st.g0.re, a);
  st.g0.im += fmaf(-ek, st.g0.im, -b);
  const float2 Ua = make_float2(a, a), Ub = make_float2(b, b);
  float2 Ya = make_float2(0.0f, 0.0f), Yb = Ya, Za = Ya, Zb = Ya;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const float2 Dr = dre[q], Di = dim[q];
    const float2 nDi = __fmul2_rn(Di, minus1);
    // a-state: (R + iI) <- D (R + iI) + a ; b-state likewise with b
    const float2 ra = __ffma2_rn(Dr, st.Ra[q], __ffma2_rn(nDi, st.Ia[q], Ua));
    const float2 ia = __ffma2_rn(Dr, st.Ia[q], __fmul2_rn(Di, st.Ra[q]));
    const float2 rb = __ffma2_rn(Dr, st.Rb[q], __ffma2_rn(nDi, st.Ib[q], Ub));
    const float2 ib = __ffma2_rn(Dr, st.Ib[q], __fmul2_rn(Di, st.Rb[q]));
    st.Ra[q] = ra; st.Ia[q] = ia; st.Rb[q] = rb; st.Ib[q] = ib;
    Ya = __ffma2_rn(mc.cpr[q], ra, __ffma2_rn(mc.ncpi[q], ia, Ya));
    Yb = __ffma2_rn(mc.cpr[q], rb, __ffma2_rn(mc.ncpi[q], ib, Yb));
    Za = __ffma2_rn(mc.cbr[q], ra, __ffma2_rn(mc.ncbi[q], ia, Za));
    Zb = __ffma2_rn(mc.cbr[q], rb, __ffma2_rn(mc.ncbi[q], ib, Zb));
  }
  // Y = ck G0 + sum_p Re(cp Ga) - i sum_p Re(cp Gb), Z likewise with cbp
  float Yr = fmaf(mc.ck, st.g0.re, Ya.x + Ya.y);
  float Yi = fmaf(mc.ck, st.g0.im, -(Yb.x + Yb.y));
  float Zr = fmaf(mc.ckk, st.g0.re, Za.x + Za.y);
  float Zi = fmaf(mc.ckk, st.g0.im, -(Zb.x + Zb.y));
  // the sums above include j = i; remove it (coefficients sY, sZ times u_i)
  Yr = fmaf(-mc.sY, a, Yr); Yi = fmaf(mc.sY, b, Yi);
  Zr = fmaf(-mc.sZ, a, Zr); Zi = fmaf(mc.sZ, b, Zi);
  const float W2 = cs * Yi + sn * Yr;         // Im e^{i k.rho} Y
  out[0] = cs * Yr - sn * Yi;                 // Re e^{i k.rho} Y
  out[1] = mc.kx * W2;
  out[2] = mc.ky * W2;
  out[3] = zsign * (cs * Zr - sn * Zi);       // Re e^{i k.rho} Z
}

// per-step decays of particle t: tabf[t][0][p] = Re, tabf[t][1][p] = Im of
// e^{-a_p dz_t}, t = 0..cnt (t = cnt: next chunk)
template <int NP>
__device__ __forceinline__ void step_decays_f2(float* tabf, const ChunkSmem<float>& s,
                                               const PairTab& pairs, int cnt) {
  for (int e = threadIdx.x; e < NP * (cnt + 1); e += blockDim.x) {
    const int t = e / NP, p = e - t * NP;
    const Cplx<float> d = cexp_neg((float)pairs.a_re[p], (float)pairs.a_im[p], s.rec[t].dz);
    tabf[t * 2 * NP + p] = d.re;
    tabf[t * 2 * NP + NP + p] = d.im;
  }
}

// The remainder modes. A warp whose 32 modes hold only r = 1..8 real ones
// (K mod 32 of its slab; the rest padding) would still cost a full warp's
// two passes over the chunk. Instead (NQR > 0) that warp runs the forward
// recurrences on lanes 0-15 and the backward ones on lanes 16-31 at the same
// time (each half at its own particle), each mode's pairs spread over two
// lanes of a half (NQR = NP/4 pair groups per lane): one pass over the chunk
// at about 45% of a full warp's instructions. The lanes' partial Y, Z enter
// the outputs linearly, so a half's sum over its 16 lanes is its sum over
// modes and pairs; only a mode's lead lane carries the beta = k
// coefficients. The halves write two slot rows (the warp's and one extra).
template <int NP, int NQR>
__device__ __forceinline__ void f2_remainder_warp(const KParams<float>& P, const ChunkSmem<float>& s,
                                                  const float* tabf, int c, int cnt, int k0,
                                                  int lane, float* slot_f, float* slot_b,
                                                  float* idle) {
  constexpr int NQ = NP / 2, SP = NQ / NQR;
  const CRange ch = kchunk(P.rp, c);
  const int Kpad = P.rp.Kpad;
  const int dir = lane >> 4, h = lane & 15;
  // modes k0 + h / SP; past K they are padding (zero coefficients, m < Kpad)
  const int m = k0 + h / SP, q0 = (h % SP) * NQR;
  ModeCoefF2<NQR> mc;
  load_mode_f2<NP, NQR>(P.modes, P.kstride, (size_t)ch.r * Kpad + m, q0, h % SP == 0, mc);
  const int S = P.plan.nstates;
  F2State<NQR> st;
  f2_load_state<NQR>(P.carry + (size_t)dir * P.rp.nchunks * S * Kpad + ((size_t)c * S) * Kpad + m,
                     Kpad, q0, st);
  const float zsign = dir == 0 ? 1.0f : -1.0f;
  float* myslot = dir == 0 ? slot_f : slot_b;
  for (int n0 = 0; n0 < cnt; n0 += 4) {
    float buf[16];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + j;
      if (n < cnt) {
        const int t = dir == 0 ? n : cnt - 1 - n;
        const int td = dir == 0 ? t : t + 1;
        const Rec<float> r = s.rec[t];
        const float dzd = dir == 0 ? r.dz : s.rec[td].dz;
        f2_step<NQR>(st, mc, r, dzd, s.trig,
                     reinterpret_cast<const float2*>(tabf + td * 2 * NP) + q0,
                     reinterpret_cast<const float2*>(tabf + td * 2 * NP + NP) + q0, zsign,
                     buf + 4 * j);
      } else {
        buf[4 * j + 0] = buf[4 * j + 1] = buf[4 * j + 2] = buf[4 * j + 3] = 0.0f;
      }
    }
    // every lane now holds one (particle, quantity) total of its half
    const float v = half_warp_reduce16<float>(buf, lane);
    const int g = h >> 2, qn = h & 3;
    const bool own = n0 + g < cnt;
    const int tt = dir == 0 ? n0 + g : cnt - 1 - (n0 + g);
    float* dst = own ? myslot + tt * 4 + qn : idle + lane;
    *dst = v;
  }
}

// NQR: pair groups per lane of a remainder warp (0: every warp runs as a full
// one). Which warps are remainder warps depends only on the slab's K and the
// mode range, so a slab gets the same arithmetic in a batch as on its own.
template <int NP, int NQR>
__global__ void kspace_final_f2_kernel(KParams<float> P, PairTab pairs) {
  extern __shared__ __align__(32) char smem[];
  const ScanPlan& pl = P.plan;
  const int c = blockIdx.x;
  const int W = pl.KR / kWarp;
  const int L = P.rp.L, Kpad = P.rp.Kpad;
  const CRange ch = kchunk(P.rp, c);
  if (!QS_DCHECK(chunk_ok(P.rp, ch, L), P.rp.status)) return;
  const int64_t start = ch.start;
  const int cnt = ch.cnt;
  // real modes of this CTA's range; with at most 8 in its last partial warp
  // that warp is a remainder warp and takes the extra slot row W
  const int kin = min(max(P.rp.info[ch.r].K - (int)blockIdx.y * pl.KR, 0), pl.KR);
  const bool rem_cta = NQR > 0 && (kin & (kWarp - 1)) >= 1 && (kin & (kWarp - 1)) <= 8;
  const int Wslots = W + (rem_cta ? 1 : 0);
  ChunkSmem<float> s = carve<float>(smem, L, NP, W + (NQR > 0 ? 1 : 0), true);
  load_chunk<float>(P, s, start, cnt);
  __syncthreads();
  float* tabf = reinterpret_cast<float*>(s.tab);
  step_decays_f2<NP>(tabf, s, pairs, cnt);
  __syncthreads();
  constexpr int NQ = NP / 2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nreal = min(max(kin - w * kWarp, 0), kWarp);   // this warp's real modes
  if (NQR > 0 && nreal == 0) {
    float* slot = s.slots + (size_t)w * L * 4;                 // padding only
    for (int e = lane; e < cnt * 4; e += kWarp) slot[e] = 0.0f;
  } else if (NQR > 0 && nreal <= 8) {
    if constexpr (NQR > 0)
      f2_remainder_warp<NP, NQR>(P, s, tabf, c, cnt, blockIdx.y * pl.KR + w * kWarp, lane,
                                 s.slots + (size_t)w * L * 4, s.slots + (size_t)W * L * 4,
                                 s.idle + w * kWarp);
  } else {
    const int m = blockIdx.y * pl.KR + threadIdx.x;
    ModeCoefF2<NQ> mc;
    load_mode_f2<NP, NQ>(P.modes, P.kstride, (size_t)ch.r * Kpad + m, 0, true, mc);
    const int S = pl.nstates;
    const size_t dirstride = (size_t)P.rp.nchunks * S * Kpad;
    float* slot = s.slots + (size_t)w * L * 4;

    // both directions unrolled: the direction-dependent indices and signs fold
    // into each copy of the loop (measured 3% faster)
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      F2State<NQ> st;
      f2_load_state<NQ>(P.carry + dir * dirstride + ((size_t)c * S) * Kpad + m, Kpad, 0, st);
      const float zsign = dir == 0 ? 1.0f : -1.0f;
      for (int n0 = 0; n0 < cnt; n0 += 4) {
        float buf[16];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int n = n0 + j;
          if (n < cnt) {
            const int t = dir == 0 ? n : cnt - 1 - n;
            const int td = dir == 0 ? t : t + 1;      // index of the decay to apply
            const Rec<float> r = s.rec[t];
            const float dzd = dir == 0 ? r.dz : s.rec[td].dz;
            f2_step<NQ>(st, mc, r, dzd, s.trig,
                        reinterpret_cast<const float2*>(tabf + td * 2 * NP),
                        reinterpret_cast<const float2*>(tabf + td * 2 * NP + NP), zsign,
                        buf + 4 * j);
          } else {
            buf[4 * j + 0] = buf[4 * j + 1] = buf[4 * j + 2] = buf[4 * j + 3] = 0.0f;
          }
        }
        const float v = warp_reduce16<float>(buf, lane);
        // every even lane now holds one (particle, quantity) total; all lanes
        // store (the others into an idle row) so that the warp does not diverge
        const int idx = lane >> 1, g = idx >> 2, qn = idx & 3;
        const bool own = !(lane & 1) && n0 + g < cnt;
        const int tt = dir == 0 ? n0 + g : cnt - 1 - (n0 + g);
        float* dst = own ? slot + tt * 4 + qn : s.idle + w * kWarp + lane;
        *dst = (dir == 0 ? 0.0f : *dst) + v;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // sum the warps' slots and write this mode range's partial outputs
  float* out = P.part + (size_t)blockIdx.y * 4 * P.rp.N;
  for (int e = threadIdx.x; e < cnt * 4; e += blockDim.x) {
    const int t = e >> 2, qn = e & 3;
    float acc = 0;
    for (int ww = 0; ww < Wslots; ++ww) acc += s.slots[((size_t)ww * L + t) * 4 + qn];
    out[(size_t)qn * P.rp.N + start + t] = acc;
  }
}

// pass B launcher: the packed kernel on the FP32 path, the scalar one on FP64
template <typename T, int NP>
struct FinalKernel {
  static void run(const KParams<T>& P, const PairTab& pairs, dim3 grid, int threads, size_t sm,
                  cudaStream_t st) {
    cudaFuncSetAttribute(kspace_final_kernel<T, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm);
    kspace_final_kernel<T, NP><<<grid, threads, sm, st>>>(P, pairs);
  }
};
template <int NP>
struct FinalKernel<float, NP> {
  template <int NQR>
  static void go(const KParams<float>& P, const PairTab& pairs, dim3 grid, int threads, size_t sm,
                 cudaStream_t st) {
    cudaFuncSetAttribute(kspace_final_f2_kernel<NP, NQR>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kspace_final_f2_kernel<NP, NQR><<<grid, threads, sm, st>>>(P, pairs);
  }
  static void run(const KParams<float>& P, const PairTab& pairs, dim3 grid, int threads, size_t sm,
                  cudaStream_t st) {
    if (P.plan.rem) go<NP / 4>(P, pairs, grid, threads, sm, st);
    else go<0>(P, pairs, grid, threads, sm, st);
  }
};

// pass A launcher: the tensor-core kernel on the FP32 path up to 12 pairs
// (at 12 with one m-tile per pass: confined slab 4.69 -> 4.40 ms; two m-tiles
// took 181 registers, one CTA per SM, and 4.85 ms), the scalar one otherwise
// (16 pairs: 218 registers)
template <typename T, int NP>
struct AggKernel {
  static void run(const KParams<T>& P, const PairTab& pairs, dim3 grid, int threads, size_t sm,
                  cudaStream_t st) {
    cudaFuncSetAttribute(kspace_aggregate_kernel<T, NP>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kspace_aggregate_kernel<T, NP><<<grid, threads, sm, st>>>(P, pairs);
  }
};
template <int NP>
struct AggKernel<float, NP> {
  static void run(const KParams<float>& P, const PairTab& pairs, dim3 grid, int threads,
                  size_t smA, cudaStream_t st) {
    if constexpr (NP <= 12) {
      const size_t sm = tc_agg_smem_bytes(P.rp.L, NP);
      cudaFuncSetAttribute(kspace_aggregate_tc_kernel<NP>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      kspace_aggregate_tc_kernel<NP><<<grid, threads, sm, st>>>(P, pairs);
    } else {
      cudaFuncSetAttribute(kspace_aggregate_kernel<float, NP>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smA);
      kspace_aggregate_kernel<float, NP><<<grid, threads, smA, st>>>(P, pairs);
    }
  }
};

// stage 0: pass A, carries and pass B; 1: pass A and carries only; 2: pass B
// only (from the carries a stage-1 launch left in place)
template <typename T, int NP>
static void kspace_run(const KParams<T>& P, const PairTab& pairs, void* dec,
                       cudaStream_t st, cudaEvent_t* ev, int stage) {
  const ScanPlan& pl = P.plan;
  const Reps& rp = P.rp;
  dim3 grid(rp.nchunks, pl.nkr);
  const size_t smA = chunk_smem_bytes<T>(rp.L, NP, 0, false);
  // pass B: with remainder warps (FP32), one more slot row
  const size_t smB = chunk_smem_bytes<T>(rp.L, NP, pl.KR / kWarp + (pl.rem ? 1 : 0), true);
  if (stage != 2) {
    AggKernel<T, NP>::run(P, pairs, grid, pl.KR, smA, st);
    if (ev) cudaEventRecord(ev[0], st);
    launch_kspace_carries<T>(pl, rp, pairs, P.zs, P.modes.kk, P.agg, P.carry, dec, st);
    if (ev) cudaEventRecord(ev[1], st);
  }
  if (stage != 1) {
    FinalKernel<T, NP>::run(P, pairs, grid, pl.KR, smB, st);
    if (ev) cudaEventRecord(ev[2], st);
  }
}

template <typename T>
void launch_kspace(const ScanPlan& plan, const Reps& rp, const ModeTab<T>& modes,
                   const PairTab& pairs, const T* zs, const T* dz, const T* qs,
                   const typename PhaseT<T>::type* xh,
                   const typename PhaseT<T>::type* yh, const float2* trig,
                   Cplx<T>* agg, Cplx<T>* carry, void* dec, T* part,
                   cudaStream_t st, cudaEvent_t* ev3, int stage) {
  KParams<T> P{plan, rp, modes, (size_t)rp.R * rp.Kpad, zs, dz, qs, xh, yh, trig, agg, carry,
               part};
  switch (plan.np) {
    case 4: kspace_run<T, 4>(P, pairs, dec, st, ev3, stage); break;
    case 8: kspace_run<T, 8>(P, pairs, dec, st, ev3, stage); break;
    case 12: kspace_run<T, 12>(P, pairs, dec, st, ev3, stage); break;
    default: kspace_run<T, 16>(P, pairs, dec, st, ev3, stage); break;
  }
}

// ============================================================ instantiations
template void launch_kspace<float>(const ScanPlan&, const Reps&, const ModeTab<float>&,
                                   const PairTab&, const float*, const float*, const float*,
                                   const uint32_t*, const uint32_t*, const float2*, Cplx<float>*,
                                   Cplx<float>*, void*, float*, cudaStream_t, cudaEvent_t*, int);
template void launch_kspace<double>(const ScanPlan&, const Reps&, const ModeTab<double>&,
                                    const PairTab&, const double*, const double*, const double*,
                                    const uint64_t*, const uint64_t*, const float2*,
                                    Cplx<double>*, Cplx<double>*, void*, double*, cudaStream_t,
                                    cudaEvent_t*, int);

}  // namespace qslab
