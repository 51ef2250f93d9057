// The virial tensor of the long-range energy of a slab, W_ab = -dE/d eps_ab,
// for pressures in the NPT ensemble (Section 4.3 extends the random-batch
// dynamics to it through the virial; Thm 2.4's L_z-dependent constant is
// what the walls' part needs).
//
// Strain: r -> (I + eps) r for the particles, the lateral lattice vectors and
// the charged walls (which keep their charge per cell); eps_zx = eps_zy = 0
// so that the lattice stays in the plane z = 0.
//
// Lateral components (ab in xx, yy, xy). The phases k.rho_ij are invariant,
// every term of E but U_self carries 1/A, and |k| moves by -k_a eps_ab k_b/|k|:
//   W_ab = delta_ab (E + U_self) + sum_k (k_a k_b/|k|) D_k,
// with D_k the k-derivative of the mode's energy. For the SOE kernel of
// Eq. 3.21, (1/k)(xi+_M + xi-_M) = C_k sum_beta c_beta e^{-beta z}, only C_k,
// c_beta and the node beta = k depend on k, so per mode
//   D_k = gam_k [ (c_k g + c_k') S_k + sum_l Re((c_l g + c_l') S_l) - c_k S_z ],
//   g = C_k'/C_k = -k/(2 alpha^2) - 1/k,
//   S_beta = sum_i Re[conj(u_i) sum_{j<i} u_j e^{-beta (z_i - z_j)}],
//   S_z    = sum_i Re[conj(u_i) sum_{j<i} u_j (z_i - z_j) e^{-k (z_i - z_j)}],
// (pairs counted once: the pair sums over i != j are twice the sums over j < i),
// gam_k the mode's prefactor (pi/A) C_k times its weight (2 for a half-plane
// mode of the full k-sum; (H/P) e^{k^2/(4 alpha^2)} for a random-batch sample,
// Eq. 4.7). The j = i part of D_k is a host constant per replica times sum q^2.
//
// S_beta and S_z come from the forward recurrences (Eqs. 3.28-3.30) started
// from the carries of the long-range call; the z-weighted state for beta = k,
//   Gz_i = e^{-k dz_i} (Gz_{i-1} + dz_i G_{i-1}),
// needs its own carries: per chunk the aggregate Az = sum_j u_j (z_end - z_j)
// e^{-k (z_end - z_j)}, then one FP64 chain per (replica, mode) over the
// chunks, X_{c+1} = e^{-k gap_c} (X_c + gap_c G_c) + Az_c.
//
// Components zz, xz, yz move no lattice vector: W_ab = sum_i F_i,a z_i from
// the call's forces, plus the explicit terms of the top wall at z = L_z, which
// moves with the box (zz: -L_z dE/dL_z; xz, yz: its lateral shift).
#include <cstdint>
#include <cuda_runtime.h>

#include "qslab_geom.cuh"
#include "qslab_math.cuh"
#include "qslab_virial.h"

namespace qslab {
namespace {

constexpr double kPiV = 3.14159265358979323846;
constexpr double kSqrtPiV = 1.7724538509055160273;
constexpr int kZf = 5;      // per-chunk force sums: z Fx, z Fy, z Fz, q^2, q
constexpr int kWf = 6;      // per-chunk wall sums: lateral xx, yy, xy, dE/dLz, shift x, y
constexpr int kRedT = 256;  // threads of the per-replica reduction

struct CD { double re, im; };
__device__ __forceinline__ CD cmul(CD a, CD b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ CD cdiv(CD a, CD b) {
  const double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// ------------------------------------------------------------ coefficients
// vc[f][R * Kpad]: f = 0: gam (c_k g + c_k'), 1: -gam c_k, 2 + 2p / 3 + 2p:
// Re / Im of gam m_p (c_p g + c_p') for the SOE pair representative p
// (m_p = 2 for a conjugate pair, whose partner contributes the conjugate);
// then, at f = 2 + 2 npc + j, the lateral weights k_x^2/k, k_y^2/k, k_x k_y/k
// (0 for padding modes).
//   c_k = sum_l 2 a_l w_l/(a_l^2 - k^2),   c_k' = sum_l 4 k a_l w_l/(a_l^2 - k^2)^2
//   c_l = -2 k w_l/(a_l^2 - k^2),          c_l' = -2 w_l (a_l^2 + k^2)/(a_l^2 - k^2)^2
template <typename T>
__global__ void vir_coef_kernel(Reps rp, int npc, PairTab pr, double alpha, int rbe,
                                ModeTab<T> mt, double* vc) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int rep = blockIdx.y;
  const int Kpad = rp.Kpad;
  if (m >= Kpad) return;
  const RepInfo& ri = rp.info[rep];
  const size_t mg = (size_t)rep * Kpad + m;
  const size_t ks = (size_t)rp.R * Kpad;
  const int mx = mt.mx[mg], my = mt.my[mg];
  const bool live = m < ri.K && (mx != 0 || my != 0);
  const double kx = 2 * kPiV * mx / ri.Lx, ky = 2 * kPiV * my / ri.Ly;
  const double k = live ? sqrt(kx * kx + ky * ky) : 1.0;
  double gam = 0.0;
  if (live)
    gam = rbe ? kPiV / ri.area * (ri.H / ri.K) * 2.0 * alpha / (kSqrtPiV * k)
              : kPiV / ri.area * 2.0 * (2.0 * alpha * exp(-k * k / (4.0 * alpha * alpha)) / (kSqrtPiV * k));
  const double g = -k / (2.0 * alpha * alpha) - 1.0 / k;
  double ck = 0.0, dck = 0.0;
  for (int p = 0; p < npc; ++p) {
    CD v = {0.0, 0.0};
    if (p < pr.np) {
      const CD a = {pr.a_re[p], pr.a_im[p]};
      const CD w = {pr.w_re[p], pr.w_im[p]};
      const double mult = pr.mult[p];
      const CD a2 = cmul(a, a);
      const CD den = {a2.re - k * k, a2.im};
      const CD q1 = cdiv(w, den);                    // w/(a^2 - k^2)
      const CD aq = cmul(a, q1);
      ck += mult * 2.0 * aq.re;
      dck += mult * 4.0 * k * cdiv(aq, den).re;
      const CD cp = {-2.0 * k * q1.re, -2.0 * k * q1.im};
      const CD dcp = cdiv(cmul({-2.0 * (a2.re + k * k), -2.0 * a2.im}, q1), den);
      v = {gam * mult * (cp.re * g + dcp.re), gam * mult * (cp.im * g + dcp.im)};
    }
    vc[(2 + 2 * (size_t)p) * ks + mg] = v.re;
    vc[(3 + 2 * (size_t)p) * ks + mg] = v.im;
  }
  vc[mg] = gam * (ck * g + dck);
  vc[ks + mg] = -gam * ck;
  const size_t fw = 2 + 2 * (size_t)npc;
  vc[fw * ks + mg] = live ? kx * kx / k : 0.0;
  vc[(fw + 1) * ks + mg] = live ? ky * ky / k : 0.0;
  vc[(fw + 2) * ks + mg] = live ? kx * ky / k : 0.0;
}

// ------------------------------------------------ z-weighted chunk aggregates
template <typename T>
struct VRec {
  typename PhaseT<T>::type xh, yh;
  T q, zd;     // zd: z (aggregates) or dz (pass)
};

template <typename T>
__device__ inline void load_recs(const VirArgs<T>& a, VRec<T>* rec, float2* trig, int64_t start,
                                 int cnt, bool want_dz) {
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    const int64_t i = start + t;
    VRec<T> r;
    r.xh = a.xh[i];
    r.yh = a.yh[i];
    r.q = a.qs[i];
    r.zd = want_dz ? a.dz[i] : a.zs[i];
    rec[t] = r;
  }
  if (a.trig)
    for (int t = threadIdx.x; t < 256; t += blockDim.x) trig[t] = a.trig[t];
}

template <typename T>
__host__ __device__ inline size_t rec_bytes(int L) {
  return ((sizeof(VRec<T>) * (size_t)L + 31) & ~size_t(31)) + sizeof(float2) * 256;
}

// Az[c][m] = sum_{j in c} u_j (z_end - z_j) e^{-k (z_end - z_j)}
template <typename T>
__global__ void vir_zagg_kernel(VirArgs<T> a, Cplx<double>* az) {
  extern __shared__ __align__(32) char smem[];
  const int c = blockIdx.x;
  const CRange ch = kchunk(a.rp, c);
  const int L = a.rp.L, Kpad = a.rp.Kpad;
  VRec<T>* rec = reinterpret_cast<VRec<T>*>(smem);
  float2* trig = reinterpret_cast<float2*>(smem + ((sizeof(VRec<T>) * (size_t)L + 31) & ~size_t(31)));
  load_recs<T>(a, rec, trig, ch.start, ch.cnt, false);
  __syncthreads();
  const int m = blockIdx.y * a.plan.KR + threadIdx.x;
  const size_t mg = (size_t)ch.r * Kpad + m;
  const int32_t mx = a.modes.mx[mg], my = a.modes.my[mg];
  const T kk = a.modes.kk[mg];
  const T zend = rec[ch.cnt - 1].zd;
  T sr = 0, si = 0;
  for (int t = 0; t < ch.cnt; ++t) {
    const VRec<T> r = rec[t];
    T cs, sn;
    phase_cs(phase_turns(mx, my, r.xh, r.yh), trig, cs, sn);
    const T d = zend - r.zd;
    const T wgt = d * exp_neg_term(kk * d);
    sr = fma(wgt, r.q * cs, sr);
    si = fma(-wgt, r.q * sn, si);
  }
  az[(size_t)c * Kpad + m] = Cplx<double>{(double)sr, (double)si};
}

// gzc[c][m]: the z-weighted state entering chunk c (at z_end(c-1)). The
// chain X_{c+1} = e_c X_c + B_c, e_c = e^{-k gap_c}, B_c = e_c gap_c G_c + Az_c
// (G_c the forward beta = k carry of chunk c) is a linear recurrence with
// known coefficients, scanned in FP64 by one CTA per (mode, replica) in three
// phases: each thread composes the maps of its segment of chunks, an
// exclusive scan over the threads gives each segment its input, and each
// thread replays its segment. The maps compose as
// (e2, B2) o (e1, B1) = (e2 e1, e2 B1 + B2).
constexpr int kChainT = 128;

template <typename T>
__device__ __forceinline__ void chain_map(const VirArgs<T>& a, const Cplx<double>* az, int c,
                                          int m, double k, double& e, double& br, double& bi) {
  const CRange ch = kchunk(a.rp, c);
  const double gap = chunk_gap(a.zs, ch, 0, a.rp.L);
  const Cplx<T> G = a.carry[(size_t)c * a.plan.nstates * a.rp.Kpad + m];   // forward, beta = k
  const Cplx<double> A = az[(size_t)c * a.rp.Kpad + m];
  e = exp(-k * gap);
  const double eg = e * gap;
  br = fma(eg, (double)G.re, A.re);
  bi = fma(eg, (double)G.im, A.im);
}

template <typename T>
__global__ void __launch_bounds__(kChainT) vir_zchain_kernel(VirArgs<T> a, const Cplx<double>* az,
                                                            Cplx<T>* gzc) {
  __shared__ double se[kChainT], sr[kChainT], si[kChainT];
  const int m = blockIdx.x;
  const int rep = blockIdx.y;
  const int Kpad = a.rp.Kpad;
  const RepInfo& ri = a.rp.info[rep];
  const int nch = ri.nch;
  if (nch == 0) return;
  const double k = (double)a.modes.kk[(size_t)rep * Kpad + m];
  const int seg = (nch + kChainT - 1) / kChainT;
  const int j0 = threadIdx.x * seg;
  const int j1 = min(nch, j0 + seg);
  // phase 1: the segment's composed map
  double E = 1.0, Br = 0.0, Bi = 0.0;
  for (int j = j0; j < j1; ++j) {
    double e, br, bi;
    chain_map<T>(a, az, ri.c0 + j, m, k, e, br, bi);
    Br = fma(e, Br, br);
    Bi = fma(e, Bi, bi);
    E *= e;
  }
  // phase 2: inclusive scan of the maps over the threads (Hillis-Steele)
  se[threadIdx.x] = E; sr[threadIdx.x] = Br; si[threadIdx.x] = Bi;
  __syncthreads();
  for (int o = 1; o < kChainT; o <<= 1) {
    double pe = 1.0, pr = 0.0, pi = 0.0;
    const bool has = threadIdx.x >= o;
    if (has) { pe = se[threadIdx.x - o]; pr = sr[threadIdx.x - o]; pi = si[threadIdx.x - o]; }
    __syncthreads();
    if (has) {
      // (E, B) o (pe, p): the earlier map first
      sr[threadIdx.x] = fma(se[threadIdx.x], pr, sr[threadIdx.x]);
      si[threadIdx.x] = fma(se[threadIdx.x], pi, si[threadIdx.x]);
      se[threadIdx.x] *= pe;
    }
    __syncthreads();
  }
  // the input of this segment: the inclusive result of the previous thread
  // applied to X = 0 at the replica's first chunk
  double xr = threadIdx.x > 0 ? sr[threadIdx.x - 1] : 0.0;
  double xi = threadIdx.x > 0 ? si[threadIdx.x - 1] : 0.0;
  // phase 3: replay
  for (int j = j0; j < j1; ++j) {
    const int c = ri.c0 + j;
    gzc[(size_t)c * Kpad + m] = Cplx<T>{(T)xr, (T)xi};
    double e, br, bi;
    chain_map<T>(a, az, c, m, k, e, br, bi);
    xr = fma(e, xr, br);
    xi = fma(e, xi, bi);
  }
}

// ------------------------------------------------------------------ the pass
// Per (chunk, mode): the forward recurrences of beta = k, the SOE pairs and
// (WZ) the z-weighted state from the carries. Per particle the coefficients
// are applied first,
//   T_i = a_i Y_a + b_i Y_b,  Y_a = v_k Re x_k + v_z Re x_z + sum_p Re(v_p x_a,p),
//                            Y_b = -v_k Im x_k - v_z Im x_z + sum_p Re(v_p x_b,p),
// with the exclusive states x (the sums over j < i), so that the terms of
// the SOE combination cancel per particle, as in the potential of pass B,
// before anything is summed over particles; D(c, m) = sum over the chunk of
// T_i, compensated (Kahan). With the energy coefficients (ck, cp of the mode
// table) and no z-weighted state, D(c, m) is the chunk's share of the mode's
// pair energy gam Re sum_beta c_beta S_beta (the energy-only call); there the
// pairs are split: the pairs within the chunk come from recurrences started
// from zero (small states, small rounding), the pairs with earlier chunks
// from one product per state of the carry G_c and pass A's backward
// aggregate, sum_{i in c} u_i e^{-beta (z_i - z_start)}, times the decay
// e^{-beta dz_start} to the carry's reference point.
template <typename T>
__device__ __forceinline__ void kahan_add(T& s, T& c, T x) {
  const T y = x - c;
  const T t = s + y;
  c = (t - s) - y;
  s = t;
}

// The pairs of chunk c with all earlier particles of its slab, for the
// energy: sum_i Re[conj(u_i) e^{-beta (z_i - z_{s-1})} G_c] for beta = k and
// sum_i (a_i, b_i) e^{-beta (z_i - z_{s-1})} (G^a_c, G^b_c) for the pairs,
// with the coefficients: from the carry G_c (at z_{s-1}) and the backward
// aggregate A_c = sum_i u_i e^{-beta (z_i - z_s)}, joined by e^{-beta dz_s}.
// decay(p) gives e^{-a_p dz_s} of the chunk's first particle.
template <typename T, int NP, typename Decay>
__device__ inline double cross_energy(const VirArgs<T>& a, int c, int m, T kk, Decay decay,
                                      const double* vc, size_t mg, size_t ks) {
  const CRange ch = kchunk(a.rp, c);
  if (ch.first) return 0.0;           // no earlier particles: carry 0
  const int Kpad = a.rp.Kpad;
  const size_t cstride = (size_t)a.plan.nstates * Kpad;
  const size_t dirstride = (size_t)a.rp.nchunks * cstride;
  const Cplx<T>* G = a.carry + (size_t)c * cstride + m;
  const Cplx<T>* A = a.agg + dirstride + (size_t)c * cstride + m;
  const double dz0 = (double)a.dz[ch.start];
  // beta = k: Re[G e^{-k dz} conj(A)]
  const double ek = exp(-(double)kk * dz0);
  const Cplx<T> g = G[0], ab = A[0];
  double D = vc[mg] * ek * ((double)g.re * (double)ab.re + (double)g.im * (double)ab.im);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const Cplx<T> d = decay(p);
    const Cplx<T> gA = G[(size_t)(1 + 2 * p) * Kpad], gB = G[(size_t)(2 + 2 * p) * Kpad];
    const Cplx<T> aA = A[(size_t)(1 + 2 * p) * Kpad], aB = A[(size_t)(2 + 2 * p) * Kpad];
    // s = d (gA aA + gB aB), complex; add Re(v s)
    const double pr = (double)gA.re * aA.re - (double)gA.im * aA.im + (double)gB.re * aB.re -
                      (double)gB.im * aB.im;
    const double pi = (double)gA.re * aA.im + (double)gA.im * aA.re + (double)gB.re * aB.im +
                      (double)gB.im * aB.re;
    const double sr = (double)d.re * pr - (double)d.im * pi;
    const double si = (double)d.re * pi + (double)d.im * pr;
    D += vc[(2 + 2 * (size_t)p) * ks + mg] * sr - vc[(3 + 2 * (size_t)p) * ks + mg] * si;
  }
  return D;
}

template <typename T, int NP>
__device__ inline double cross_pairs(const VirArgs<T>& a, int c, int m, T kk, const Cplx<T>* tab,
                                     const double* vc, size_t mg, size_t ks) {
  return cross_energy<T, NP>(a, c, m, kk, [tab](int p) { return tab[p]; }, vc, mg, ks);
}

template <typename T, int NP, bool WZ>
__global__ void vir_pass_kernel(VirArgs<T> a, const double* vc, const Cplx<T>* gzc,
                                double* dpart) {
  extern __shared__ __align__(32) char smem[];
  const int c = blockIdx.x;
  const CRange ch = kchunk(a.rp, c);
  const int L = a.rp.L, Kpad = a.rp.Kpad;
  const int cnt = ch.cnt;
  VRec<T>* rec = reinterpret_cast<VRec<T>*>(smem);
  float2* trig = reinterpret_cast<float2*>(smem + ((sizeof(VRec<T>) * (size_t)L + 31) & ~size_t(31)));
  Cplx<T>* tab = reinterpret_cast<Cplx<T>*>(smem + rec_bytes<T>(L));
  load_recs<T>(a, rec, trig, ch.start, cnt, true);
  for (int e = threadIdx.x; e < NP * cnt; e += blockDim.x) {
    const int t = e / NP, p = e - t * NP;
    tab[e] = cexp_neg((T)a.pairs.a_re[p], (T)a.pairs.a_im[p], a.dz[ch.start + t]);
  }
  __syncthreads();
  const int m = blockIdx.y * a.plan.KR + threadIdx.x;
  const size_t mg = (size_t)ch.r * Kpad + m;
  const size_t ks = (size_t)a.rp.R * Kpad;
  const int32_t mx = a.modes.mx[mg], my = a.modes.my[mg];
  const T kk = a.modes.kk[mg];
  const T vk = (T)vc[mg];
  const T vz = WZ ? (T)vc[ks + mg] : (T)0;
  T vpr[NP], vpi[NP];
  const size_t cstride = (size_t)a.plan.nstates * Kpad;
  const Cplx<T>* cin = a.carry + (size_t)c * cstride + m;
  const Cplx<T> zc = {0, 0};
  Cplx<T> g0 = WZ ? cin[0] : zc;
  Cplx<T> ga[NP], gb[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    ga[p] = WZ ? cin[(size_t)(1 + 2 * p) * Kpad] : zc;
    gb[p] = WZ ? cin[(size_t)(2 + 2 * p) * Kpad] : zc;
    vpr[p] = (T)vc[(2 + 2 * (size_t)p) * ks + mg];
    vpi[p] = (T)vc[(3 + 2 * (size_t)p) * ks + mg];
  }
  Cplx<T> gz = WZ ? gzc[(size_t)c * Kpad + m] : Cplx<T>{0, 0};
  T acc = 0, cmp = 0;
  for (int t = 0; t < cnt; ++t) {
    const VRec<T> r = rec[t];
    T cs, sn;
    phase_cs(phase_turns(mx, my, r.xh, r.yh), trig, cs, sn);
    const T av = r.q * cs, bv = r.q * sn;     // u = av - i bv
    const T ek = one_minus_exp_neg(kk * r.zd);
    // beta = k: exclusive state, then add u
    const T xr = fma(-ek, g0.re, g0.re), xi = fma(-ek, g0.im, g0.im);
    T Ya = vk * xr, Yb = -vk * xi;
    if (WZ) {
      // z-weighted state from the state before this particle
      const T hr = fma(r.zd, g0.re, gz.re), hi = fma(r.zd, g0.im, gz.im);
      gz.re = fma(-ek, hr, hr);
      gz.im = fma(-ek, hi, hi);
      Ya = fma(vz, gz.re, Ya);
      Yb = fma(-vz, gz.im, Yb);
    }
    g0.re = xr + av;
    g0.im = xi - bv;
    const Cplx<T>* dt = tab + t * NP;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const Cplx<T> d = dt[p];
      const T ar = fma(d.re, ga[p].re, -d.im * ga[p].im);
      const T ai = fma(d.re, ga[p].im, d.im * ga[p].re);
      const T br = fma(d.re, gb[p].re, -d.im * gb[p].im);
      const T bi = fma(d.re, gb[p].im, d.im * gb[p].re);
      Ya = fma(vpr[p], ar, fma(-vpi[p], ai, Ya));
      Yb = fma(vpr[p], br, fma(-vpi[p], bi, Yb));
      ga[p].re = ar + av; ga[p].im = ai;
      gb[p].re = br + bv; gb[p].im = bi;
    }
    kahan_add(acc, cmp, fma(av, Ya, bv * Yb));
  }
  double D = (double)acc - (double)cmp;
  if (!WZ) D += cross_pairs<T, NP>(a, c, m, kk, tab, vc, mg, ks);
  dpart[(size_t)c * Kpad + m] = D;
}

// The same pass on the FP32 path with two SOE pairs per 64-bit register
// (packed FP32 FMAs, __ffma2_rn / __fmul2_rn): the decay table is stored
// re/im-split per particle so that two pairs' decays load as one float2.
template <int NP, bool WZ>
__global__ void vir_pass_f2_kernel(VirArgs<float> a, const double* vc, const Cplx<float>* gzc,
                                   double* dpart) {
  extern __shared__ __align__(32) char smem[];
  const int c = blockIdx.x;
  const CRange ch = kchunk(a.rp, c);
  const int L = a.rp.L, Kpad = a.rp.Kpad;
  const int cnt = ch.cnt;
  VRec<float>* rec = reinterpret_cast<VRec<float>*>(smem);
  float2* trig = reinterpret_cast<float2*>(smem + ((sizeof(VRec<float>) * (size_t)L + 31) & ~size_t(31)));
  float* tabf = reinterpret_cast<float*>(smem + rec_bytes<float>(L));
  load_recs<float>(a, rec, trig, ch.start, cnt, true);
  for (int e = threadIdx.x; e < NP * cnt; e += blockDim.x) {
    const int t = e / NP, p = e - t * NP;
    const Cplx<float> d = cexp_neg((float)a.pairs.a_re[p], (float)a.pairs.a_im[p], a.dz[ch.start + t]);
    tabf[t * 2 * NP + p] = d.re;
    tabf[t * 2 * NP + NP + p] = d.im;
  }
  __syncthreads();
  const int m = blockIdx.y * a.plan.KR + threadIdx.x;
  const size_t mg = (size_t)ch.r * Kpad + m;
  const size_t ks = (size_t)a.rp.R * Kpad;
  const int32_t mx = a.modes.mx[mg], my = a.modes.my[mg];
  const float kk = a.modes.kk[mg];
  const float vk = (float)vc[mg];
  const float vz = WZ ? (float)vc[ks + mg] : 0.0f;
  const size_t cstride = (size_t)a.plan.nstates * Kpad;
  const Cplx<float>* cin = a.carry + (size_t)c * cstride + m;
  const Cplx<float> zc = {0.0f, 0.0f};
  Cplx<float> g0 = WZ ? cin[0] : zc;
  float2 Ra[NP / 2], Ia[NP / 2], Rb[NP / 2], Ib[NP / 2], Vr[NP / 2], nVi[NP / 2];
#pragma unroll
  for (int q = 0; q < NP / 2; ++q) {
    const Cplx<float> a0 = WZ ? cin[(size_t)(1 + 4 * q) * Kpad] : zc;
    const Cplx<float> b0 = WZ ? cin[(size_t)(2 + 4 * q) * Kpad] : zc;
    const Cplx<float> a1 = WZ ? cin[(size_t)(3 + 4 * q) * Kpad] : zc;
    const Cplx<float> b1 = WZ ? cin[(size_t)(4 + 4 * q) * Kpad] : zc;
    Ra[q] = make_float2(a0.re, a1.re); Ia[q] = make_float2(a0.im, a1.im);
    Rb[q] = make_float2(b0.re, b1.re); Ib[q] = make_float2(b0.im, b1.im);
    const size_t p0 = 2 * q, p1 = 2 * q + 1;
    Vr[q] = make_float2((float)vc[(2 + 2 * p0) * ks + mg], (float)vc[(2 + 2 * p1) * ks + mg]);
    nVi[q] = make_float2(-(float)vc[(3 + 2 * p0) * ks + mg], -(float)vc[(3 + 2 * p1) * ks + mg]);
  }
  Cplx<float> gz = WZ ? gzc[(size_t)c * Kpad + m] : Cplx<float>{0.0f, 0.0f};
  float acc = 0.0f, cmp = 0.0f;
  for (int t = 0; t < cnt; ++t) {
    const VRec<float> r = rec[t];
    float cs, sn;
    phase_cs(phase_turns(mx, my, r.xh, r.yh), trig, cs, sn);
    const float av = r.q * cs, bv = r.q * sn;
    const float ek = one_minus_exp_neg(kk * r.zd);
    const float xr = fmaf(-ek, g0.re, g0.re), xi = fmaf(-ek, g0.im, g0.im);
    float ya = vk * xr, yb = -vk * xi;
    if (WZ) {
      const float hr = fmaf(r.zd, g0.re, gz.re), hi = fmaf(r.zd, g0.im, gz.im);
      gz.re = fmaf(-ek, hr, hr);
      gz.im = fmaf(-ek, hi, hi);
      ya = fmaf(vz, gz.re, ya);
      yb = fmaf(-vz, gz.im, yb);
    }
    g0.re = xr + av;
    g0.im = xi - bv;
    const float2 Ua = make_float2(av, av), Ub = make_float2(bv, bv);
    float2 Ya = make_float2(0.0f, 0.0f), Yb = Ya;
    const float2* dre = reinterpret_cast<const float2*>(tabf + t * 2 * NP);
    const float2* dim = reinterpret_cast<const float2*>(tabf + t * 2 * NP + NP);
#pragma unroll
    for (int q = 0; q < NP / 2; ++q) {
      const float2 Dr = dre[q], Di = dim[q];
      const float2 nDi = make_float2(-Di.x, -Di.y);
      // exclusive states D g (before this particle's input)
      const float2 ar = __ffma2_rn(Dr, Ra[q], __fmul2_rn(nDi, Ia[q]));
      const float2 ai = __ffma2_rn(Dr, Ia[q], __fmul2_rn(Di, Ra[q]));
      const float2 br = __ffma2_rn(Dr, Rb[q], __fmul2_rn(nDi, Ib[q]));
      const float2 bi = __ffma2_rn(Dr, Ib[q], __fmul2_rn(Di, Rb[q]));
      Ya = __ffma2_rn(Vr[q], ar, __ffma2_rn(nVi[q], ai, Ya));
      Yb = __ffma2_rn(Vr[q], br, __ffma2_rn(nVi[q], bi, Yb));
      Ra[q] = __fadd2_rn(ar, Ua); Ia[q] = ai;
      Rb[q] = __fadd2_rn(br, Ub); Ib[q] = bi;
    }
    ya += Ya.x + Ya.y;
    yb += Yb.x + Yb.y;
    kahan_add(acc, cmp, fmaf(av, ya, bv * yb));
  }
  double D = (double)acc - (double)cmp;
  if (!WZ)
    D += cross_energy<float, NP>(
        a, c, m, kk,
        [tabf](int p) { return Cplx<float>{tabf[p], tabf[NP + p]}; }, vc, mg, ks);
  dpart[(size_t)c * Kpad + m] = D;
}

// ------------------------------------------------------- fixed-order sums
// Sum of v over the block (blockDim.x a multiple of 32, <= 1024): warp
// shuffles, then warp 0 over the warps' totals; the result is valid in
// thread 0. Deterministic for a fixed assignment of terms to threads.
__device__ inline double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) s += sh[j];
  return s;
}

// zpart[c][5]: sum over the chunk's particles (caller's order; the index
// range of a replica is the same before and after sorting) of z Fx, z Fy,
// z Fz, q^2 and q.
template <typename T>
__global__ void vir_zf_kernel(VirArgs<T> a, double* zpart) {
  __shared__ double sh[32];
  const int c = blockIdx.x;
  const CRange ch = kchunk(a.rp, c);
  double acc[kZf] = {0, 0, 0, 0, 0};
  for (int t = threadIdx.x; t < ch.cnt; t += blockDim.x) {
    const int64_t i = ch.start + t;
    const double z = (double)a.pos[3 * i + 2];
    const double qi = (double)a.q[i];
    acc[0] += z * (double)a.force[3 * i];
    acc[1] += z * (double)a.force[3 * i + 1];
    acc[2] += z * (double)a.force[3 * i + 2];
    acc[3] += qi * qi;
    acc[4] += qi;
  }
  for (int j = 0; j < kZf; ++j) {
    const double s = block_sum(acc[j], sh);
    if (threadIdx.x == 0) zpart[(size_t)c * kZf + j] = s;
  }
}

// wpart[c][6]: the walls' Fourier modes (Thm 2.4), per chunk: the lateral
// sums (k_a k_b/k) q_i d phi_w/dk, q_i d phi_w/dL_z and q_i d phi_w/d shift of
// the top wall (x, y); each listed mode stands for k and -k (real sum: twice
// the real part). FP64.
template <typename T>
__global__ void vir_walls_kernel(VirArgs<T> a, double* wpart) {
  __shared__ double sh[32];
  const int c = blockIdx.x;
  const CRange ch = kchunk(a.rp, c);
  const RepInfo& ri = a.rp.info[ch.r];
  const WallTab& W = a.walls;
  double acc[kWf] = {0, 0, 0, 0, 0, 0};
  for (int t = threadIdx.x; t < ch.cnt; t += blockDim.x) {
    const int64_t i = ch.start + t;
    const double x = (double)a.pos[3 * i], y = (double)a.pos[3 * i + 1];
    const double zb = (double)a.pos[3 * i + 2], zt = ri.Lz - zb;
    const double qi = (double)a.q[i];
    for (int w = 0; w < W.nw; ++w) {
      const double kx = 2 * kPiV * W.m[w][0] / ri.Lx, ky = 2 * kPiV * W.m[w][1] / ri.Ly;
      const double k = sqrt(kx * kx + ky * ky);
      double sn, cs;
      sincos(kx * x + ky * y, &sn, &cs);
      const double eb = exp(-k * zb), et = exp(-k * zt);
      // 2 pi c e^{i k.rho} (bottom, top); the cell integral is A c, over A
      const CD hb = cmul({2 * kPiV * W.c[w][0], 2 * kPiV * W.c[w][1]}, {cs, sn});
      const CD ht = cmul({2 * kPiV * W.c[w][2], 2 * kPiV * W.c[w][3]}, {cs, sn});
      // d/dk of (1/k)(hb e^{-k zb} + ht e^{-k zt})
      const double dre = -(hb.re * eb + ht.re * et) / (k * k) - (hb.re * zb * eb + ht.re * zt * et) / k;
      const double D = 2.0 * qi * dre;
      acc[0] += kx * kx / k * D;
      acc[1] += ky * ky / k * D;
      acc[2] += kx * ky / k * D;
      // top-wall term (1/k) ht e^{-k zt}: d/dLz gives -k times it; a shift d
      // of the top wall multiplies it by e^{-i k.d}
      acc[3] += 2.0 * qi * (-ht.re * et);
      acc[4] += 2.0 * qi * kx * ht.im * et / k;
      acc[5] += 2.0 * qi * ky * ht.im * et / k;
    }
  }
  for (int j = 0; j < kWf; ++j) {
    const double s = block_sum(acc[j], sh);
    if (threadIdx.x == 0) wpart[(size_t)c * kWf + j] = s;
  }
}

// msum[mg] = sum over the replica's chunks of D(c, m). One CTA of 32 warps
// per (replica, 32 modes): lane = mode (coalesced), warp w sums the chunks
// w, w + 32, ..., then the warps' sums are added in a fixed order.
constexpr int kSumWarps = 32;
__global__ void __launch_bounds__(32 * kSumWarps) vir_modesum_kernel(Reps rp, const double* dpart,
                                                                    double* msum) {
  __shared__ double part[kSumWarps][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int m = blockIdx.x * 32 + lane;
  const int rep = blockIdx.y;
  const RepInfo& ri = rp.info[rep];
  double acc = 0.0;
  if (m < rp.Kpad)
    for (int j = w; j < ri.nch; j += kSumWarps) acc += dpart[((size_t)ri.c0 + j) * rp.Kpad + m];
  part[w][lane] = acc;
  __syncthreads();
  if (w == 0 && m < rp.Kpad) {
    double t = 0.0;
    for (int v = 0; v < kSumWarps; ++v) t += part[v][lane];
    msum[(size_t)rep * rp.Kpad + m] = t;
  }
}

// One CTA per replica: the lateral sums over modes (weights from the
// coefficient table), the force and wall sums over chunks, and the assembly
// of W (xx, yy, zz, xy, xz, yz).
template <typename T>
__global__ void vir_reduce_kernel(VirArgs<T> a, const double* msum, const double* vc,
                                  const double* zpart, const double* wpart) {
  __shared__ double sh[32];
  const int rep = blockIdx.x;
  const RepInfo& ri = a.rp.info[rep];
  const int Kpad = a.rp.Kpad;
  const size_t ks = (size_t)a.rp.R * Kpad;
  const size_t fw = 2 + 2 * (size_t)a.plan.np;
  double lat[3] = {0, 0, 0};
  for (int m = threadIdx.x; m < Kpad; m += blockDim.x) {
    const size_t mg = (size_t)rep * Kpad + m;
    const double D = msum[mg];
    lat[0] += vc[fw * ks + mg] * D;
    lat[1] += vc[(fw + 1) * ks + mg] * D;
    lat[2] += vc[(fw + 2) * ks + mg] * D;
  }
  double zs[kZf] = {0, 0, 0, 0, 0}, ws[kWf] = {0, 0, 0, 0, 0, 0};
  for (int j = threadIdx.x; j < ri.nch; j += blockDim.x) {
    const size_t c = (size_t)ri.c0 + j;
    for (int f = 0; f < kZf; ++f) zs[f] += zpart[c * kZf + f];
    if (wpart)
      for (int f = 0; f < kWf; ++f) ws[f] += wpart[c * kWf + f];
  }
  double tot[3 + kZf + kWf];
  for (int f = 0; f < 3; ++f) tot[f] = block_sum(lat[f], sh);
  for (int f = 0; f < kZf; ++f) tot[3 + f] = block_sum(zs[f], sh);
  for (int f = 0; f < kWf; ++f) tot[3 + kZf + f] = block_sum(ws[f], sh);
  if (threadIdx.x != 0) return;
  const double E = ri.n > 0 ? a.energies[rep] : 0.0;
  const double Q2 = tot[3 + 3], Q = tot[3 + 4];
  const double Uself = a.alpha / kSqrtPiV * Q2;
  const double* vd = a.vdiag + 3 * (size_t)rep;
  const double* wv = tot + 3 + kZf;
  double dEdLz = wv[3];
  if (a.walls.on) dEdLz += Q * (-2.0 * kPiV * a.walls.st0);
  double* out = a.virial + 6 * (size_t)rep;
  out[0] = E + Uself + tot[0] + Q2 * vd[0] + wv[0];             // xx
  out[1] = E + Uself + tot[1] + Q2 * vd[1] + wv[1];             // yy
  out[2] = tot[3 + 2] - ri.Lz * dEdLz;                          // zz
  out[3] = tot[2] + Q2 * vd[2] + wv[2];                         // xy
  out[4] = tot[3 + 0] - ri.Lz * wv[4];                          // xz
  out[5] = tot[3 + 1] - ri.Lz * wv[5];                          // yz
}

template <typename T, int NP, bool WZ>
struct VirPass {
  static void run(const VirArgs<T>& a, const double* vc, const Cplx<T>* gzc, double* dpart,
                  size_t sm, dim3 grid, cudaStream_t st) {
    cudaFuncSetAttribute(vir_pass_kernel<T, NP, WZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm);
    vir_pass_kernel<T, NP, WZ><<<grid, a.plan.KR, sm, st>>>(a, vc, gzc, dpart);
  }
};
template <int NP, bool WZ>
struct VirPass<float, NP, WZ> {
  static void run(const VirArgs<float>& a, const double* vc, const Cplx<float>* gzc,
                  double* dpart, size_t sm, dim3 grid, cudaStream_t st) {
    cudaFuncSetAttribute(vir_pass_f2_kernel<NP, WZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm);
    vir_pass_f2_kernel<NP, WZ><<<grid, a.plan.KR, sm, st>>>(a, vc, gzc, dpart);
  }
};

template <typename T, int NP, bool WZ>
int run_pass(const VirArgs<T>& a, const double* vc, const Cplx<T>* gzc, double* dpart,
             cudaStream_t st) {
  const int L = a.rp.L;
  const size_t sm = rec_bytes<T>(L) + sizeof(Cplx<T>) * (size_t)NP * L;
  VirPass<T, NP, WZ>::run(a, vc, gzc, dpart, sm, dim3(a.rp.nchunks, a.plan.nkr), st);
  return 1;
}

template <typename T, bool WZ>
int pass_np(const VirArgs<T>& a, const double* vc, const Cplx<T>* gzc, double* dpart,
            cudaStream_t st) {
  switch (a.plan.np) {
    case 4: return run_pass<T, 4, WZ>(a, vc, gzc, dpart, st);
    case 8: return run_pass<T, 8, WZ>(a, vc, gzc, dpart, st);
    case 12: return run_pass<T, 12, WZ>(a, vc, gzc, dpart, st);
    default: return run_pass<T, 16, WZ>(a, vc, gzc, dpart, st);
  }
}

// Energy coefficients in the layout of the virial table: f = 0: ck =
// gam c_kk, f = 1: 0, 2 + 2p / 3 + 2p: Re / Im of cp = m_p gam c_{k,p}
// (the mode table's own values, so that the energy-only call and the full
// call weight the pair sums identically).
template <typename T>
__global__ void energy_coef_kernel(Reps rp, int npc, ModeTab<T> mt, double* vc) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int rep = blockIdx.y;
  if (m >= rp.Kpad) return;
  const size_t mg = (size_t)rep * rp.Kpad + m;
  const size_t ks = (size_t)rp.R * rp.Kpad;
  vc[mg] = (double)mt.ck[mg];
  vc[ks + mg] = 0.0;
  for (int p = 0; p < npc; ++p) {
    vc[(2 + 2 * (size_t)p) * ks + mg] = (double)mt.cp[((size_t)0 * npc + p) * ks + mg];
    vc[(3 + 2 * (size_t)p) * ks + mg] = (double)mt.cp[((size_t)1 * npc + p) * ks + mg];
  }
}

// energies[r] += sum over the replica's modes of msum (fixed order): one
// warp per replica.
__global__ void energy_add_kernel(Reps rp, const double* msum, double* energies) {
  const int rep = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (rep >= rp.R) return;   // whole warps leave together
  double s = 0.0;
  for (int m = lane; m < rp.Kpad; m += 32) s += msum[(size_t)rep * rp.Kpad + m];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) energies[rep] += s;
}

struct VirLayout {
  size_t vc, az, gzc, dpart, msum, zpart, wpart, total;
};

VirLayout layout(const ScanPlan& pl, const Reps& rp) {
  VirLayout l{};
  size_t o = 0;
  auto take = [&o](size_t b) { size_t r = o; o += (b + 255) & ~size_t(255); return r; };
  const size_t cm = (size_t)rp.nchunks * rp.Kpad;
  l.vc = take(sizeof(double) * (5 + 2 * (size_t)pl.np) * rp.R * rp.Kpad);
  l.az = take(sizeof(Cplx<double>) * cm);
  l.gzc = take(sizeof(Cplx<double>) * cm);   // room for either precision
  l.dpart = take(sizeof(double) * cm);
  l.msum = take(sizeof(double) * rp.R * rp.Kpad);
  l.zpart = take(sizeof(double) * kZf * (size_t)rp.nchunks);
  l.wpart = take(sizeof(double) * kWf * (size_t)rp.nchunks);
  l.total = o;
  return l;
}

}  // namespace

size_t virial_workspace_bytes(const ScanPlan& plan, const Reps& rp) {
  return layout(plan, rp).total;
}

template <typename T>
int launch_virial(const VirArgs<T>& a, void* ws, cudaStream_t st) {
  const VirLayout l = layout(a.plan, a.rp);
  char* b = static_cast<char*>(ws);
  double* vc = reinterpret_cast<double*>(b + l.vc);
  Cplx<double>* az = reinterpret_cast<Cplx<double>*>(b + l.az);
  Cplx<T>* gzc = reinterpret_cast<Cplx<T>*>(b + l.gzc);
  double* dpart = reinterpret_cast<double*>(b + l.dpart);
  double* msum = reinterpret_cast<double*>(b + l.msum);
  double* zpart = reinterpret_cast<double*>(b + l.zpart);
  double* wpart = reinterpret_cast<double*>(b + l.wpart);
  const int Kpad = a.rp.Kpad;
  int nl = 0;
  vir_coef_kernel<T><<<dim3((Kpad + 127) / 128, a.rp.R), 128, 0, st>>>(
      a.rp, a.plan.np, a.pairs, a.alpha, a.rbe, a.modes, vc);
  ++nl;
  if (a.rp.nchunks > 0) {
    const size_t smz = rec_bytes<T>(a.rp.L);
    vir_zagg_kernel<T><<<dim3(a.rp.nchunks, a.plan.nkr), a.plan.KR, smz, st>>>(a, az);
    vir_zchain_kernel<T><<<dim3(Kpad, a.rp.R), kChainT, 0, st>>>(a, az, gzc);
    nl += 2;
    nl += pass_np<T, true>(a, vc, gzc, dpart, st);
    vir_modesum_kernel<<<dim3((Kpad + 31) / 32, a.rp.R), 32 * kSumWarps, 0, st>>>(a.rp, dpart, msum);
    vir_zf_kernel<T><<<a.rp.nchunks, 256, 0, st>>>(a, zpart);
    nl += 2;
    if (a.walls.on && a.walls.nw > 0) {
      vir_walls_kernel<T><<<a.rp.nchunks, 256, 0, st>>>(a, wpart);
      ++nl;
    }
  }
  vir_reduce_kernel<T><<<a.rp.R, kRedT, 0, st>>>(
      a, msum, vc, zpart, (a.walls.on && a.walls.nw > 0) ? wpart : nullptr);
  ++nl;
  return nl;
}

template <typename T>
int launch_energy_pass(const VirArgs<T>& a, void* ws, cudaStream_t st) {
  const VirLayout l = layout(a.plan, a.rp);
  char* b = static_cast<char*>(ws);
  double* vc = reinterpret_cast<double*>(b + l.vc);
  double* dpart = reinterpret_cast<double*>(b + l.dpart);
  double* msum = reinterpret_cast<double*>(b + l.msum);
  const int Kpad = a.rp.Kpad;
  energy_coef_kernel<T><<<dim3((Kpad + 127) / 128, a.rp.R), 128, 0, st>>>(a.rp, a.plan.np,
                                                                           a.modes, vc);
  pass_np<T, false>(a, vc, nullptr, dpart, st);
  vir_modesum_kernel<<<dim3((Kpad + 31) / 32, a.rp.R), 32 * kSumWarps, 0, st>>>(a.rp, dpart, msum);
  return 3;
}

int launch_energy_add(const ScanPlan& plan, const Reps& rp, const void* ws, double* energies,
                      cudaStream_t st) {
  const VirLayout l = layout(plan, rp);
  const double* msum = reinterpret_cast<const double*>(static_cast<const char*>(ws) + l.msum);
  const int64_t thr = (int64_t)rp.R * 32;
  energy_add_kernel<<<(unsigned)((thr + 255) / 256), 256, 0, st>>>(rp, msum, energies);
  return 1;
}

template int launch_virial<float>(const VirArgs<float>&, void*, cudaStream_t);
template int launch_virial<double>(const VirArgs<double>&, void*, cudaStream_t);
template int launch_energy_pass<float>(const VirArgs<float>&, void*, cudaStream_t);
template int launch_energy_pass<double>(const VirArgs<double>&, void*, cudaStream_t);

}  // namespace qslab
