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
#include "qslab_internal.h"
#include "qslab_math.cuh"

namespace qslab {

// ================================================================= geometry

// Particle range of one chunk of a replica.
struct CRange {
  int64_t start;
  int cnt;
  int r;          // replica
  bool first;     // first chunk of the replica
  bool last;      // last chunk of the replica
};

// k-space chunk c (chunks of L)
__device__ __forceinline__ CRange kchunk(const Reps& rp, int c) {
  CRange x;
  x.r = rp.chunk_rep[c];
  const RepInfo& ri = rp.info[x.r];
  const int j = c - ri.c0;
  x.start = ri.off + (int64_t)j * rp.L;
  const int left = ri.n - j * rp.L;
  x.cnt = left < rp.L ? left : rp.L;
  x.first = j == 0;
  x.last = j == ri.nch - 1;
  return x;
}

// k = 0 chunk c (chunks of L0)
__device__ __forceinline__ CRange zchunk(const Reps& rp, int c) {
  CRange x;
  x.r = rp.zchunk_rep[c];
  const RepInfo& ri = rp.info[x.r];
  const int j = c - ri.z0;
  x.start = ri.off + (int64_t)j * rp.L0;
  const int left = ri.n - j * rp.L0;
  x.cnt = left < rp.L0 ? left : rp.L0;
  x.first = j == 0;
  x.last = j == ri.nz - 1;
  return x;
}

inline int chunk_threads(int L) {
  const int t = ((L + 31) / 32) * 32;
  return t < 256 ? t : 256;
}

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

// One CTA per k-space chunk (chunks are contiguous in the caller's order as
// well): finiteness and z-range checks, the z keys, the replica index and
// the replica's sums of q and |q|.
template <typename T>
__global__ void prepare_kernel(Reps rp, const T* __restrict__ pos, const T* __restrict__ q,
                               typename KeyOf<T>::type* keys, uint32_t* vals, int32_t* rid,
                               double* sums, unsigned* status) {
  __shared__ double red[2][32];
  const CRange ch = kchunk(rp, blockIdx.x);
  const double Lz = rp.info[ch.r].Lz;
  double sq = 0.0, sa = 0.0;
  unsigned flags = 0;
  for (int t = threadIdx.x; t < ch.cnt; t += blockDim.x) {
    const int64_t i = ch.start + t;
    const T x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2], qi = q[i];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(qi)) flags |= kStNonfinite;
    else if (!(z >= (T)0) || !((double)z <= Lz)) flags |= kStZRange;
    keys[i] = KeyOf<T>::key(z);
    vals[i] = (uint32_t)i;
    if (rid) rid[i] = ch.r;
    sq += (double)qi;
    sa += fabs((double)qi);
  }
  if (flags) atomicOr(status, flags);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o; o >>= 1) {
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
  }
  if (lane == 0) { red[0][w] = sq; red[1][w] = sa; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) { a += red[0][j]; b += red[1][j]; }
    atomicAdd(&sums[2 * ch.r], a);
    atomicAdd(&sums[2 * ch.r + 1], b);
  }
}

template <typename T>
void launch_prepare(const Reps& rp, const T* pos, const T* q, void* keys, uint32_t* vals,
                    int32_t* rid, double* sums, unsigned* status, cudaStream_t st) {
  prepare_kernel<T><<<rp.nchunks, chunk_threads(rp.L), 0, st>>>(
      rp, pos, q, static_cast<typename KeyOf<T>::type*>(keys), vals, rid, sums, status);
}

__global__ void check_neutral_kernel(int R, const double* sums, double tol, unsigned* status,
                                     uint64_t* ctr) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < R && tol >= 0.0 && fabs(sums[2 * r]) > tol * sums[2 * r + 1])
    atomicOr(status, kStNonneutral);
  if (ctr && r == 0) {
    const uint64_t c = ctr[0];
    ctr[1] = c;
    ctr[0] = c + 1;
  }
}

void launch_check_neutral(const Reps& rp, const double* sums, double tol, unsigned* status,
                          uint64_t* ctr, cudaStream_t st) {
  check_neutral_kernel<<<(rp.R + 255) / 256, 256, 0, st>>>(rp.R, sums, tol, status, ctr);
}

__global__ void rep_keys_kernel(int64_t N, const uint32_t* __restrict__ perm,
                                const int32_t* __restrict__ rid, uint32_t* keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    keys[i] = (uint32_t)rid[perm[i]];
}

void launch_rep_keys(int64_t N, const uint32_t* perm, const int32_t* rid, uint32_t* keys,
                     cudaStream_t st) {
  int blocks = (int)((N + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  rep_keys_kernel<<<blocks, 256, 0, st>>>(N, perm, rid, keys);
}

// ==================================================================== gather

__device__ __forceinline__ uint32_t to_fixed(float x, double L) {
  double f = (double)x / L;
  f -= floor(f);
  if (!(f < 1.0)) f = 0.0;
  return (uint32_t)(uint64_t)(f * 4294967296.0);
}
__device__ __forceinline__ uint64_t to_fixed(double x, double L) {
  double f = x / L;
  f -= floor(f);
  if (!(f < 1.0)) f = 0.0;
  return (uint64_t)(f * 18446744073709551616.0);
}

// One CTA per k-space chunk: the sorted SoA arrays, with dz = 0 at the first
// particle of every replica.
template <typename T>
__global__ void gather_kernel(Reps rp, const T* __restrict__ pos, const T* __restrict__ q,
                              const uint32_t* __restrict__ perm, T* zs, T* dz, T* qs,
                              typename PhaseT<T>::type* xh, typename PhaseT<T>::type* yh,
                              int32_t* perm_out) {
  const CRange ch = kchunk(rp, blockIdx.x);
  const double Lx = rp.info[ch.r].Lx, Ly = rp.info[ch.r].Ly;
  for (int t = threadIdx.x; t < ch.cnt; t += blockDim.x) {
    const int64_t i = ch.start + t;
    const uint32_t o = perm[i];
    const T z = pos[3 * (int64_t)o + 2];
    zs[i] = z;
    dz[i] = (t == 0 && ch.first) ? (T)0 : z - pos[3 * (int64_t)perm[i - 1] + 2];
    qs[i] = q[o];
    xh[i] = to_fixed(pos[3 * (int64_t)o], Lx);
    yh[i] = to_fixed(pos[3 * (int64_t)o + 1], Ly);
    perm_out[i] = (int32_t)o;
  }
}

template <typename T>
void launch_gather(const Reps& rp, const T* pos, const T* q, const uint32_t* perm, T* zs,
                   T* dz, T* qs, typename PhaseT<T>::type* xh,
                   typename PhaseT<T>::type* yh, int32_t* perm_out, cudaStream_t st) {
  gather_kernel<T><<<rp.nchunks, chunk_threads(rp.L), 0, st>>>(rp, pos, q, perm, zs, dz, qs,
                                                                xh, yh, perm_out);
}

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
  T* slots;       // pass B: [W][L][4]
};

__host__ __device__ inline size_t align_up(size_t x) { return (x + 31) & ~size_t(31); }

template <typename T>
__host__ __device__ inline size_t chunk_smem_bytes(int L, int NP, int W, bool passB) {
  size_t b = 0;
  b += align_up(sizeof(Cplx<T>) * (size_t)NP * (passB ? (L + 1) : 2 * L));
  b += align_up(sizeof(Rec<T>) * (L + 1));
  b += align_up(sizeof(T) * L);
  if (passB) b += align_up(sizeof(T) * (size_t)W * L * 4);
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
  s.slots = passB ? reinterpret_cast<T*>(p) : nullptr;
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
}

// ------------------------------------------------------------------ pass A
template <typename T, int NP>
__global__ void kspace_aggregate_kernel(KParams<T> P, PairTab pairs) {
  extern __shared__ __align__(32) char smem[];
  const ScanPlan& pl = P.plan;
  const int c = blockIdx.x;
  const CRange ch = kchunk(P.rp, c);
  const int64_t start = ch.start;
  const int cnt = ch.cnt;
  const int Kpad = P.rp.Kpad;
  ChunkSmem<T> s = carve<T>(smem, P.rp.L, NP, 0, false);
  load_chunk<T>(P, s, start, cnt);
  __syncthreads();
  // E tables: [t][0][p] = e^{-a_p (z_end - z_t)}, [t][1][p] = e^{-a_p (z_t - z_start)}
  const T zend = s.zl[cnt - 1], zst = s.zl[0];
  for (int e = threadIdx.x; e < NP * cnt; e += blockDim.x) {
    const int t = e / NP, p = e - t * NP;
    const T ar = (T)pairs.a_re[p], ai = (T)pairs.a_im[p];
    s.tab[(2 * t) * NP + p] = cexp_neg(ar, ai, zend - s.zl[t]);
    s.tab[(2 * t + 1) * NP + p] = cexp_neg(ar, ai, s.zl[t] - zst);
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
    sincos_turns(phase_turns(mc.mx, mc.my, r.xh, r.yh), cs, sn);
    const T a = r.q * cs, b = r.q * sn;   // u = a - i b
    const T zt = s.zl[t];
    const T ef = exp_neg(mc.kk * (zend - zt));
    const T eb = exp_neg(mc.kk * (zt - zst));
    f0.re = fma(ef, a, f0.re); f0.im = fma(-ef, b, f0.im);
    b0.re = fma(eb, a, b0.re); b0.im = fma(-eb, b, b0.im);
    const Cplx<T>* Et = s.tab + 2 * t * NP;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const Cplx<T> Ef = Et[p];
      const Cplx<T> Eb = Et[NP + p];
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

// --------------------------------------------------- chunk-to-chunk decays
// All decays between chunk reference points are computed in FP64 by these
// parallel kernels and stored in the carry type (FP64, or double-float on the
// FP32 path), so that the sequential chains below only multiply and add.
//   pair decays  pdec[dir][c][p]: forward e^{-a_p (z_end(c) - z_end(c-1))},
//                backward e^{-a_p (z_start(c+1) - z_start(c))}
//   mode decays  kdec[dir][c][m]: the same with beta = |k_m|
// Both are 1 (gap 0) where the chain of a replica starts, whose carry is 0.
template <typename T>
__device__ inline double chunk_gap(const T* zs, const CRange& ch, int dir, int L) {
  if (dir == 0) {
    if (ch.first) return 0.0;
    return (double)zs[ch.start + ch.cnt - 1] - (double)zs[ch.start - 1];
  }
  if (ch.last) return 0.0;
  return (double)zs[ch.start + L] - (double)zs[ch.start];   // chunk c is full
}

// zero_chunks = 0: k-space chunks (L), 1: k = 0 chunks (L0)
template <typename T>
__global__ void pair_decay_kernel(Reps rp, int zero_chunks, int np, const T* zs, PairTab pairs,
                                  Cplx<typename CarryNum<T>::type>* pdec,
                                  typename CarryNum<T>::type* gaps) {
  using CN = typename CarryNum<T>::type;
  const int nch = zero_chunks ? rp.nzchunks : rp.nchunks;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * nch * np) return;
  const int dir = e / (nch * np);
  const int r = e - dir * nch * np;
  const int c = r / np, p = r - c * np;
  const CRange ch = zero_chunks ? zchunk(rp, c) : kchunk(rp, c);
  const double gap = chunk_gap(zs, ch, dir, zero_chunks ? rp.L0 : rp.L);
  const Cplx<double> d = cexp_neg(pairs.a_re[p], pairs.a_im[p], gap);
  pdec[e] = Cplx<CN>{cn_from(d.re, (CN*)nullptr), cn_from(d.im, (CN*)nullptr)};
  if (gaps && p == 0) gaps[dir * nch + c] = cn_from(gap, (CN*)nullptr);
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

template <typename T>
__global__ void mode_decay_kernel(Reps rp, const T* zs, const T* kk,
                                  typename CarryNum<T>::type* kdec) {
  using CN = typename CarryNum<T>::type;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per_dir = (int64_t)rp.nchunks * rp.Kpad;
  if (e >= 2 * per_dir) return;
  const int dir = (int)(e / per_dir);
  const int64_t r = e - (int64_t)dir * per_dir;
  const int c = (int)(r / rp.Kpad), m = (int)(r - (int64_t)c * rp.Kpad);
  const CRange ch = kchunk(rp, c);
  const double x = (double)kk[(size_t)ch.r * rp.Kpad + m] * chunk_gap(zs, ch, dir, rp.L);
  kdec[e] = cn_from(exp_neg_small(x), (CN*)nullptr);
}

// ------------------------------------------------------------------ carries
// carry_in[c+1] = D_c carry_in[c] + A_c over the chunks of a replica
// (forward; mirrored backward), one chain per (replica, direction, state,
// mode), in the carry type. The chunks of a replica are cut into groups,
// and the chains run in three parallel phases: (1) every group composes its
// transfer (D_g = prod D_c, A_g = the group's output from a zero input);
// (2) a short chain over the replica's groups gives each group's input;
// (3) every group replays its chunks from that input and writes the
// carries. Depth 2g + G instead of G g for G groups of g chunks. The last
// group of a chain needs no transfer. Loads and stores are coalesced across
// modes.

template <typename T>
struct CarryCtx {
  Reps rp;
  int S, np;
  size_t cs;        // stride between chunks in agg/carry (S * Kpad)
  size_t dirstride; // nchunks * S * Kpad
};

template <typename T>
__device__ __forceinline__ void chunk_decay(const CarryCtx<T>& X, const Cplx<typename CarryNum<T>::type>* pdec,
                                            const typename CarryNum<T>::type* kdec, int dir, int st,
                                            int m, int c, typename CarryNum<T>::type& dr,
                                            typename CarryNum<T>::type& di) {
  using CN = typename CarryNum<T>::type;
  if (st == 0) {
    dr = kdec[((size_t)dir * X.rp.nchunks + c) * X.rp.Kpad + m];
    di = cn_zero((CN*)nullptr);
  } else {
    const Cplx<CN> d = pdec[((size_t)dir * X.rp.nchunks + c) * X.np + ((st - 1) >> 1)];
    dr = d.re; di = d.im;
  }
}

// phase 1 (replay = false) and phase 3 (replay = true); thread = (dir, state, group, mode)
template <typename T>
__global__ void carry_group_kernel(CarryCtx<T> X, const Cplx<T>* agg, Cplx<T>* carry,
                                   const Cplx<typename CarryNum<T>::type>* pdec,
                                   const typename CarryNum<T>::type* kdec,
                                   Cplx<typename CarryNum<T>::type>* gD,
                                   Cplx<typename CarryNum<T>::type>* gA, bool replay) {
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
  const CN zero = cn_zero((CN*)nullptr), one = cn_from(1.0, (CN*)nullptr);
  CN cr = zero, ci = zero, pr = one, pi = zero;
  if (replay) { cr = gA[gidx].re; ci = gA[gidx].im; }
  const Cplx<T>* A = agg + dir * X.dirstride + (size_t)st * Kpad + m;
  Cplx<T>* C = carry + dir * X.dirstride + (size_t)st * Kpad + m;
  const int ca = X.rp.gstart[grp], cb = X.rp.gstart[grp + 1];
  const int len = cb - ca;
  constexpr int B = 8;
  for (int jb = 0; jb < len; jb += B) {
    Cplx<T> a[B];
    CN dr[B], di[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int j = jb + u;
      dr[u] = zero; di[u] = zero; a[u] = Cplx<T>{0, 0};
      if (j < len) {
        const int c = dir == 0 ? ca + j : cb - 1 - j;
        a[u] = A[c * X.cs];
        chunk_decay<T>(X, pdec, kdec, dir, st, m, c, dr[u], di[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int j = jb + u;
      if (j < len) {
        const int c = dir == 0 ? ca + j : cb - 1 - j;
        if (replay) C[c * X.cs] = Cplx<T>{cn_to_t(cr), cn_to_t(ci)};
        const CN nr = dr[u] * cr - di[u] * ci + cn_from_t(a[u].re, (CN*)nullptr);
        const CN ni = dr[u] * ci + di[u] * cr + cn_from_t(a[u].im, (CN*)nullptr);
        cr = nr; ci = ni;
        if (!replay) {
          const CN npr = dr[u] * pr - di[u] * pi;
          const CN npi = dr[u] * pi + di[u] * pr;
          pr = npr; pi = npi;
        }
      }
    }
  }
  if (!replay) {
    gD[gidx] = Cplx<CN>{pr, pi};
    gA[gidx] = Cplx<CN>{cr, ci};
  }
}

// phase 2: thread = (dir, state, replica, mode); turns gA into each group's input
template <typename T>
__global__ void carry_chain_kernel(CarryCtx<T> X, const Cplx<typename CarryNum<T>::type>* gD,
                                   Cplx<typename CarryNum<T>::type>* gA) {
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
  const RepInfo& ri = X.rp.info[rep];
  const CN zero = cn_zero((CN*)nullptr);
  CN cr = zero, ci = zero;
  for (int j = 0; j < ri.ng; ++j) {
    const int grp = dir == 0 ? ri.g0 + j : ri.g0 + ri.ng - 1 - j;
    const size_t gidx = (((size_t)dir * X.S + st) * NG + grp) * Kpad + m;
    if (j == ri.ng - 1) {
      gA[gidx] = Cplx<CN>{cr, ci};
      break;
    }
    const Cplx<CN> d = gD[gidx], a = gA[gidx];
    gA[gidx] = Cplx<CN>{cr, ci};
    const CN nr = d.re * cr - d.im * ci + a.re;
    const CN ni = d.re * ci + d.im * cr + a.im;
    cr = nr; ci = ni;
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
          sincos_turns(phase_turns(mc.mx, mc.my, r.xh, r.yh), cs, sn);
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
      const int idx = lane >> 1, g = idx >> 2, qn = idx & 3;
      if (!(lane & 1) && n0 + g < cnt) {
        const int tt = dir == 0 ? n0 + g : cnt - 1 - (n0 + g);
        if (dir == 0) slot[tt * 4 + qn] = v;
        else slot[tt * 4 + qn] += v;
      }
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

template <typename T>
inline void decay_views(const ScanPlan& pl, const Reps& rp, void* dec,
                        Cplx<typename CarryNum<T>::type>*& pdec,
                        typename CarryNum<T>::type*& kdec,
                        Cplx<typename CarryNum<T>::type>*& gD,
                        Cplx<typename CarryNum<T>::type>*& gA) {
  using CN = typename CarryNum<T>::type;
  pdec = static_cast<Cplx<CN>*>(dec);
  kdec = reinterpret_cast<CN*>(pdec + (size_t)2 * rp.nchunks * pl.np);
  gD = reinterpret_cast<Cplx<CN>*>(kdec + (size_t)2 * rp.nchunks * rp.Kpad);
  gA = gD + (size_t)2 * pl.nstates * rp.ngroups * rp.Kpad;
}

template <typename T, int NP>
static void kspace_run(const KParams<T>& P, const PairTab& pairs, void* dec,
                       cudaStream_t st, cudaEvent_t* ev) {
  using CN = typename CarryNum<T>::type;
  const ScanPlan& pl = P.plan;
  const Reps& rp = P.rp;
  dim3 grid(rp.nchunks, pl.nkr);
  const size_t smA = chunk_smem_bytes<T>(rp.L, NP, 0, false);
  const size_t smB = chunk_smem_bytes<T>(rp.L, NP, pl.KR / kWarp, true);
  cudaFuncSetAttribute(kspace_aggregate_kernel<T, NP>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smA);
  cudaFuncSetAttribute(kspace_final_kernel<T, NP>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smB);
  kspace_aggregate_kernel<T, NP><<<grid, pl.KR, smA, st>>>(P, pairs);
  if (ev) cudaEventRecord(ev[0], st);
  Cplx<CN>* pdec; CN* kdec; Cplx<CN>* gD; Cplx<CN>* gA;
  decay_views<T>(pl, rp, dec, pdec, kdec, gD, gA);
  const int ne = 2 * rp.nchunks * pl.np;
  pair_decay_kernel<T><<<(ne + 255) / 256, 256, 0, st>>>(rp, 0, pl.np, P.zs, pairs, pdec, nullptr);
  const int64_t nk = (int64_t)2 * rp.nchunks * rp.Kpad;
  mode_decay_kernel<T><<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(rp, P.zs, P.modes.kk, kdec);
  CarryCtx<T> X;
  X.rp = rp;
  X.S = pl.nstates;
  X.np = pl.np;
  X.cs = (size_t)pl.nstates * rp.Kpad;
  X.dirstride = (size_t)rp.nchunks * pl.nstates * rp.Kpad;
  const int64_t ng = (int64_t)2 * X.S * rp.ngroups * rp.Kpad;
  carry_group_kernel<T><<<(unsigned)((ng + 127) / 128), 128, 0, st>>>(X, P.agg, P.carry, pdec, kdec,
                                                                      gD, gA, false);
  const int64_t nt = (int64_t)2 * X.S * rp.R * rp.Kpad;
  carry_chain_kernel<T><<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(X, gD, gA);
  carry_group_kernel<T><<<(unsigned)((ng + 127) / 128), 128, 0, st>>>(X, P.agg, P.carry, pdec, kdec,
                                                                      gD, gA, true);
  if (ev) cudaEventRecord(ev[1], st);
  kspace_final_kernel<T, NP><<<grid, pl.KR, smB, st>>>(P, pairs);
  if (ev) cudaEventRecord(ev[2], st);
}

size_t kspace_decay_bytes(const ScanPlan& pl, const Reps& rp, int fp64) {
  const size_t cn = fp64 ? sizeof(double) : sizeof(DF);
  // pair decays, mode decays, group transfers (D and A)
  return 2 * cn * (size_t)2 * rp.nchunks * pl.np + cn * (size_t)2 * rp.nchunks * rp.Kpad +
         2 * 2 * cn * (size_t)2 * pl.nstates * rp.ngroups * rp.Kpad + 1024;
}

template <typename T>
void launch_kspace(const ScanPlan& plan, const Reps& rp, const ModeTab<T>& modes,
                   const PairTab& pairs, const T* zs, const T* dz, const T* qs,
                   const typename PhaseT<T>::type* xh,
                   const typename PhaseT<T>::type* yh, Cplx<T>* agg,
                   Cplx<T>* carry, void* dec, T* part,
                   cudaStream_t st, cudaEvent_t* ev3) {
  KParams<T> P{plan, rp, modes, (size_t)rp.R * rp.Kpad, zs, dz, qs, xh, yh, agg, carry, part};
  switch (plan.np) {
    case 4: kspace_run<T, 4>(P, pairs, dec, st, ev3); break;
    case 8: kspace_run<T, 8>(P, pairs, dec, st, ev3); break;
    case 12: kspace_run<T, 12>(P, pairs, dec, st, ev3); break;
    default: kspace_run<T, 16>(P, pairs, dec, st, ev3); break;
  }
}

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

template <typename T>
__global__ void kzero_aggregate_kernel(K0Params Q, PairTab pr, const T* zs,
                                       const T* qs, Cplx<T>* agg,
                                       typename CarryNum<T>::type* csum) {
  using CN = typename CarryNum<T>::type;
  const int lanes = Q.npad;
  const int g = (blockIdx.x * blockDim.x + threadIdx.x);
  const int c = g / lanes, p = g - c * lanes;
  if (c >= Q.rp.nzchunks) return;
  const CRange ch = zchunk(Q.rp, c);
  const int64_t start = ch.start;
  const int cnt = ch.cnt;
  const T zst = zs[start], zen = zs[start + cnt - 1];
  const bool act = p < pr.np;
  const T ar = act ? (T)pr.a_re[p] : (T)0, ai = act ? (T)pr.a_im[p] : (T)0;
  Cplx<T> sf{0, 0}, hf{0, 0}, sb{0, 0}, hb{0, 0};
  CN q0 = cn_zero((CN*)nullptr), q1 = cn_zero((CN*)nullptr);
  for (int t = 0; t < cnt; ++t) {
    const T z = zs[start + t], qq = qs[start + t];
    if (p == 0) { q0 = cn_add(q0, qq); q1 = cn_add_prod(q1, qq, z); }
    if (!act) continue;
    const T xf = zen - z, xb = z - zst;
    const Cplx<T> ef = cexp_neg(ar, ai, xf);
    const Cplx<T> eb = cexp_neg(ar, ai, xb);
    sf.re = fma(qq, ef.re, sf.re); sf.im = fma(qq, ef.im, sf.im);
    hf.re = fma(qq * xf, ef.re, hf.re); hf.im = fma(qq * xf, ef.im, hf.im);
    sb.re = fma(qq, eb.re, sb.re); sb.im = fma(qq, eb.im, sb.im);
    hb.re = fma(qq * xb, eb.re, hb.re); hb.im = fma(qq * xb, eb.im, hb.im);
  }
  if (act) {
    Cplx<T>* a = agg + ((size_t)c * lanes + p) * 4;
    a[0] = sf; a[1] = hf; a[2] = sb; a[3] = hb;
  }
  if (p == 0) { csum[2 * c] = q0; csum[2 * c + 1] = q1; }
}

// One CTA per replica. One thread per (direction, pair) runs the chain over
// the replica's k = 0 chunks in the carry type; thread 32k (its own warp)
// scans the chunk sums of q and q z into per-chunk prefixes and the
// replica's totals.
template <typename T>
__global__ void kzero_carry_kernel(K0Params Q, PairTab pr, const typename CarryNum<T>::type* gaps,
                                   const Cplx<T>* agg,
                                   const Cplx<typename CarryNum<T>::type>* pdec,
                                   typename CarryNum<T>::type* carry,
                                   const typename CarryNum<T>::type* csum,
                                   typename CarryNum<T>::type* cpre,
                                   typename CarryNum<T>::type* rtot) {
  using CN = typename CarryNum<T>::type;
  const CN zero = cn_zero((CN*)nullptr);
  const int rep = blockIdx.x;
  const RepInfo& ri = Q.rp.info[rep];
  const int z0 = ri.z0, nz = ri.nz;
  const int nch = Q.rp.nzchunks;
  const int e = threadIdx.x;
  const int pre_thread = ((2 * Q.npad + 31) / 32) * 32;
  if (e == pre_thread) {
    CN a = zero, b = zero;
    constexpr int B = 16;
    for (int j0 = 0; j0 < nz; j0 += B) {
      CN va[B], vb[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        va[u] = zero; vb[u] = zero;
        if (j0 + u < nz) {
          const int c = z0 + j0 + u;
          va[u] = csum[2 * c]; vb[u] = csum[2 * c + 1];
        }
      }
#pragma unroll
      for (int u = 0; u < B; ++u) {
        if (j0 + u < nz) {
          const int c = z0 + j0 + u;
          cpre[2 * c] = a; cpre[2 * c + 1] = b;
          a = a + va[u]; b = b + vb[u];
        }
      }
    }
    rtot[2 * rep] = a; rtot[2 * rep + 1] = b;
    return;
  }
  if (e >= 2 * Q.npad) return;
  const int dir = e / Q.npad, p = e - dir * Q.npad;
  if (p >= pr.np) return;
  const int np = pr.np;
  CN sr = zero, si = zero, hr = zero, hi = zero;
  constexpr int B = 8;
  for (int j0 = 0; j0 < nz; j0 += B) {
    Cplx<T> as[B], ah[B];
    Cplx<CN> d[B];
    CN dzc[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int j = j0 + u;
      if (j < nz) {
        const int c = dir == 0 ? z0 + j : z0 + nz - 1 - j;
        const Cplx<T>* a = agg + ((size_t)c * Q.npad + p) * 4 + 2 * dir;
        as[u] = a[0];
        ah[u] = a[1];
        d[u] = pdec[((size_t)dir * nch + c) * np + p];
        dzc[u] = gaps[dir * nch + c];
      }
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int j = j0 + u;
      if (j < nz) {
        const int c = dir == 0 ? z0 + j : z0 + nz - 1 - j;
        CN* out = carry + (((size_t)dir * nch + c) * Q.npad + p) * 4;
        out[0] = sr; out[1] = si; out[2] = hr; out[3] = hi;
        // S' = d S + S_loc ; H' = d (H + dz S) + H_loc
        const CN tr = hr + dzc[u] * sr, ti = hi + dzc[u] * si;
        const CN nhr = d[u].re * tr - d[u].im * ti + cn_from_t(ah[u].re, (CN*)nullptr);
        const CN nhi = d[u].re * ti + d[u].im * tr + cn_from_t(ah[u].im, (CN*)nullptr);
        const CN nsr = d[u].re * sr - d[u].im * si + cn_from_t(as[u].re, (CN*)nullptr);
        const CN nsi = d[u].re * si + d[u].im * sr + cn_from_t(as[u].im, (CN*)nullptr);
        sr = nsr; si = nsi; hr = nhr; hi = nhi;
      }
    }
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
  extern __shared__ __align__(16) char ksm_raw[];   // [chunks per block][L0][2] of T
  T* ksm = reinterpret_cast<T*>(ksm_raw);
  const int lanes = Q.npad;
  const int L0 = Q.rp.L0;
  const int nch = Q.rp.nzchunks;
  const int64_t N = Q.rp.N;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = g / lanes, p = g - c * lanes;
  const int lc = threadIdx.x / lanes;
  T* acc = ksm + (size_t)lc * L0 * 2;
  const bool valid = c < nch;
  CRange ch{0, 0, 0, false, false};
  if (valid) ch = zchunk(Q.rp, c);
  const int64_t start = ch.start;
  const int cnt = ch.cnt;
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
  for (int t = threadIdx.x % lanes; t < L0; t += lanes) { acc[2 * t] = 0; acc[2 * t + 1] = 0; }
  __syncwarp();
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
      const int64_t i = start + t;
      T pot = 0, der = 0;
      if (act && live) {
        const T qq = qs[i];
        // the backward step applies the next particle's dz (0 past the
        // replica's end: its carry is 0 there)
        const int64_t id = dir == 0 ? i : i + 1;
        const T dzi = id < N ? dz[id] : (T)0;
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
  if (p == 0 && valid) {
    // sum_j q_j |z_i - z_j| = z_i (Q< - Q>) - P< + P>, from prefix sums in
    // the carry type (the terms cancel heavily); the result stays in the
    // carry type and the combine kernel widens it to FP64
    CN Ql = cpre[2 * c], Pl = cpre[2 * c + 1];
    const CN Qt = rtot[2 * ch.r], Pt = rtot[2 * ch.r + 1];
    const CN c1 = cn_from(Q.c1, (CN*)nullptr);
    const CN pre = cn_from(2.0 * 3.14159265358979323846 / Q.rp.info[ch.r].area, (CN*)nullptr);
    for (int t = 0; t < cnt; ++t) {
      const int64_t i = start + t;
      const T zt = zs[i], qt = qs[i];
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
  const int tot = nch * npad;
  constexpr int kK0Threads = 128;
  kzero_aggregate_kernel<T><<<(tot + kK0Threads - 1) / kK0Threads, kK0Threads, 0, st>>>(
      Q, pairs, zs, qs, agg, csum);
  const int ne = 2 * nch * pairs.np;
  pair_decay_kernel<T><<<(ne + 255) / 256, 256, 0, st>>>(rp, 1, pairs.np, zs, pairs, pdec, gaps);
  kzero_carry_kernel<T><<<rp.R, ((2 * npad + 31) / 32) * 32 + 32, 0, st>>>(
      Q, pairs, gaps, agg, pdec, carry, csum, cpre, rtot);
  // 8 chunks per CTA: npad * 8 threads is a whole number of warps for npad >= 4
  const int cpb = 8;
  const int thr = npad * cpb;
  const size_t sm = (size_t)cpb * rp.L0 * 2 * sizeof(T);
  cudaFuncSetAttribute(kzero_final_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  kzero_final_kernel<T><<<(tot + thr - 1) / thr, thr, sm, st>>>(
      Q, pairs, zs, dz, qs, carry, cpre, rtot, phi0, fz0);
}

size_t kzero_work_doubles(int nzchunks, int R, int np) {
  const int npad = kzero_lanes(np);
  // in 8-byte units (a double-float takes one), with room for the 256-byte
  // alignment of each of the 7 arrays
  return (size_t)nzchunks * npad * 4 * 2 + (size_t)nzchunks * 2 +
         (size_t)2 * nzchunks * kMaxPairs * 2 + (size_t)2 * nzchunks * npad * 4 +
         (size_t)nzchunks * 2 + (size_t)R * 2 + (size_t)2 * nzchunks + 7 * 32 + 64;
}

// ================================================================== combine

// One CTA per k-space chunk: sums the mode ranges' partial outputs, adds the
// k = 0 term and the j = i constant of the chunk's replica, scatters the
// potential and force to the caller's order and writes the chunk's energy
// 1/2 sum q_i phi_i.
template <typename T>
__global__ void combine_kernel(Reps rp, int nkr, const T* __restrict__ part,
                               const typename CarryNum<T>::type* __restrict__ phi0,
                               const typename CarryNum<T>::type* __restrict__ fz0,
                               const T* __restrict__ qs, const int32_t* __restrict__ perm,
                               double* echunk, T* phi_out, T* force_out) {
  __shared__ double red[32];
  const CRange ch = kchunk(rp, blockIdx.x);
  const double diagq = rp.info[ch.r].diagq;
  const int64_t N = rp.N;
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
    const int32_t o = perm[i];
    if (phi_out) phi_out[o] = (T)ph;
    if (force_out) {
      force_out[3 * (int64_t)o] = (T)fx;
      force_out[3 * (int64_t)o + 1] = (T)fy;
      force_out[3 * (int64_t)o + 2] = (T)fz;
    }
    e += 0.5 * qq * ph;
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
                    const void* fz0v, const T* qs, const int32_t* perm, double* echunk,
                    T* phi_out, T* force_out, double* energies, cudaStream_t st) {
  using CN = typename CarryNum<T>::type;
  const CN* phi0 = static_cast<const CN*>(phi0v);
  const CN* fz0 = static_cast<const CN*>(fz0v);
  combine_kernel<T><<<rp.nchunks, chunk_threads(rp.L), 0, st>>>(rp, nkr, part, phi0, fz0, qs, perm,
                                                                 echunk, phi_out, force_out);
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

// Fill the mode tables; thread = (mode, replica). Full k-sum: (mx, my) from
// the replica's half-plane list, weight 2 (k and -k), gam = (pi/A) C_k 2.
// Random batch: (mx, my) drawn here (Philox4x64-10 with counter
// (m, attempt, call, tag + replica * 2^32) and key (seed, 0); words 0,1 then
// 2,3 are inverted through the replica's per-axis cumulative tables; the
// origin is rejected), gam = (pi/A) (H/P) 2 alpha/(sqrt(pi) k) (Eq. 4.7 with
// 4.9: the Gaussian of C_k cancels against e^{k^2/(4 alpha^2)}).
template <typename T>
__global__ void mode_coef_kernel(Reps rp, int npc, const int32_t* list, int rbe, uint64_t seed,
                                 const uint64_t* ctr, const double* cdf, PairTab pr,
                                 double alpha, ModeTab<T> mt, int32_t* sampled) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int rep = blockIdx.y;
  const int Kpad = rp.Kpad;
  if (m >= Kpad) return;
  const RepInfo& ri = rp.info[rep];
  const int K = ri.K;
  const double Lx = ri.Lx, Ly = ri.Ly;
  const size_t mg = (size_t)rep * Kpad + m;
  const size_t ks = (size_t)rp.R * Kpad;
  const double pi = 3.14159265358979323846;
  const double sqpi = 1.7724538509055160;
  int mx = 0, my = 0;
  if (m < K) {
    if (!rbe) {
      mx = list[2 * ((size_t)ri.list0 + m)];
      my = list[2 * ((size_t)ri.list0 + m) + 1];
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
      if (sampled) {
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
  for (int p = 0; p < npc; ++p) {
    double cr = 0, ci = 0, br = 0, bi = 0;
    if (p < pr.np) {
      const double ar = pr.a_re[p], ai = pr.a_im[p];
      const double wr = pr.w_re[p], wi = pr.w_im[p];
      const double dr = ar * ar - ai * ai - k * k, di = 2 * ar * ai;   // a^2 - k^2
      const double dd = dr * dr + di * di;
      const double qr = (wr * dr + wi * di) / dd, qi = (wi * dr - wr * di) / dd;  // w/(a^2-k^2)
      ckk += pr.mult[p] * 2.0 * (ar * qr - ai * qi);     // sum over both nodes of 2 a w/(a^2-k^2)
      cr = -2.0 * k * qr * pr.mult[p] * gam;             // m_p gam c_{k,p}
      ci = -2.0 * k * qi * pr.mult[p] * gam;
      br = cr * ar - ci * ai;                            // times a_p
      bi = cr * ai + ci * ar;
      sY += cr;
      sZ += br;
    }
    mt.cp[((size_t)0 * npc + p) * ks + mg] = (T)cr;
    mt.cp[((size_t)1 * npc + p) * ks + mg] = (T)ci;
    mt.cp[((size_t)2 * npc + p) * ks + mg] = (T)br;
    mt.cp[((size_t)3 * npc + p) * ks + mg] = (T)bi;
  }
  const double ck = gam * ckk;
  mt.mx[mg] = mx;
  mt.my[mg] = my;
  mt.kx[mg] = (T)kx;
  mt.ky[mg] = (T)ky;
  mt.kk[mg] = (T)k;
  mt.ck[mg] = (T)ck;
  mt.ckk[mg] = (T)(ck * k);
  mt.sY[mg] = (T)(ck + sY);
  mt.sZ[mg] = (T)(ck * k + sZ);
}

template <typename T>
void launch_mode_coef(const Reps& rp, int npc, const int32_t* list, int rbe, uint64_t seed,
                      const uint64_t* ctr, const double* cdf, const PairTab& pairs,
                      double alpha, ModeTab<T> modes, int32_t* sampled, cudaStream_t st) {
  dim3 grid((rp.Kpad + 127) / 128, rp.R);
  mode_coef_kernel<T><<<grid, 128, 0, st>>>(rp, npc, list, rbe, seed, ctr, cdf, pairs, alpha,
                                            modes, sampled);
}

// ============================================================ instantiations
#define QSLAB_INST(T, PH)                                                                        \
  template void launch_prepare<T>(const Reps&, const T*, const T*, void*, uint32_t*, int32_t*,   \
                                  double*, unsigned*, cudaStream_t);                             \
  template void launch_gather<T>(const Reps&, const T*, const T*, const uint32_t*, T*, T*, T*,   \
                                 PH*, PH*, int32_t*, cudaStream_t);                              \
  template void launch_kspace<T>(const ScanPlan&, const Reps&, const ModeTab<T>&,                \
                                 const PairTab&, const T*, const T*, const T*, const PH*,        \
                                 const PH*, Cplx<T>*, Cplx<T>*, void*, T*, cudaStream_t,         \
                                 cudaEvent_t*);                                                  \
  template void launch_kzero<T>(const Reps&, const PairTab&, double, const T*, const T*,         \
                                const T*, double*, void*, void*, cudaStream_t);                  \
  template void launch_combine<T>(const Reps&, int, const T*, const void*, const void*,          \
                                  const T*, const int32_t*, double*, T*, T*, double*,            \
                                  cudaStream_t);                                                 \
  template void launch_mode_coef<T>(const Reps&, int, const int32_t*, int, uint64_t,             \
                                    const uint64_t*, const double*, const PairTab&, double,      \
                                    ModeTab<T>, int32_t*, cudaStream_t);
QSLAB_INST(float, uint32_t)
QSLAB_INST(double, uint64_t)
#undef QSLAB_INST

}  // namespace qslab
