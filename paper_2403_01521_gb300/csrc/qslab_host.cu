// qslab C ABI: context, configuration, host-side precompute (k-mode lists,
// SOE pair representatives, the normaliser H, the sampler's cumulative
// tables, the j = i constants), workspace management and the launch
// sequence of one compute call.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "qslab.h"
#include "qslab_internal.h"

using namespace qslab;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.7724538509055160273;

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct qslab_ctx {
  int device = 0;
  int prec = QSLAB_FP64;
  // configuration
  double Lx = 0, Ly = 0, Lz = 0, alpha = 0;
  bool has_box = false, has_alpha = false, has_soe = false;
  int mode = 0;                 // 1 full k-sum, 2 random batch
  double kc = 0;
  int P = 0;
  uint64_t seed = 0, counter = 0;
  std::vector<double> s_re, s_im, w_re, w_im;
  double neutral_tol = -2.0;    // < -1: default for the precision
  int tune_L = 0, tune_KR = 0;
  bool timing = false;
  // derived configuration
  bool dirty = true;
  PairTab pairs{};
  int npc = 4;                  // pair count the kernels are compiled for
  std::vector<int32_t> half_modes;
  int K = 0, Kpad = 0, KR = 32, nkr = 1;
  double diag_k = 0;            // sum over all summed k of (pi/A) erfc(k/2a)/k
  double H = 0;
  int cdf_nx = 0, cdf_ny = 0, mxmax = 0, mymax = 0;
  // persistent device data (per configuration)
  void* d_cfg = nullptr;
  size_t cfg_bytes = 0;
  int32_t* d_list = nullptr;
  double* d_cdfx = nullptr;
  double* d_cdfy = nullptr;
  int32_t* d_sampled = nullptr;
  void* d_modes = nullptr;      // mode table storage
  bool coef_ready = false;
  // small persistent buffers
  unsigned* d_status = nullptr;
  double* d_sums = nullptr;
  double* d_energy = nullptr;
  // per-N workspace
  void* d_ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t last_stream = nullptr;
  bool have_sample = false;
  cudaEvent_t ev[9] = {};
  int launches = 0;
  // the k = 0 term runs on a side stream, forked from and joined to the
  // caller's stream with these events (capturable in a CUDA graph)
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

namespace {

int cuda_fail(cudaError_t e) {
  if (e == cudaSuccess) return QSLAB_OK;
  if (e == cudaErrorMemoryAllocation) return QSLAB_ERR_ALLOC;
  return QSLAB_ERR_CUDA;
}

#define QS_CUDA(call)                          \
  do {                                         \
    cudaError_t e__ = (call);                  \
    if (e__ != cudaSuccess) return cuda_fail(e__); \
  } while (0)

bool finite_pos(double v) { return std::isfinite(v) && v > 0; }

// Representatives of conjugate pairs of SOE nodes (multiplicity 2) and real
// nodes (multiplicity 1); padded with zero-weight entries to a compiled size.
int build_pairs(qslab_ctx* c) {
  const int M = (int)c->s_re.size();
  PairTab t{};
  std::vector<bool> used(M, false);
  int np = 0;
  for (int l = 0; l < M; ++l) {
    if (used[l]) continue;
    const double sr = c->s_re[l], si = c->s_im[l];
    const double mag = std::hypot(sr, si);
    used[l] = true;
    double mult = 1.0;
    if (std::fabs(si) > 1e-12 * mag) {
      // find the conjugate partner
      int best = -1;
      double bd = 1e300;
      for (int j = 0; j < M; ++j) {
        if (used[j]) continue;
        const double d = std::hypot(c->s_re[j] - sr, c->s_im[j] + si);
        if (d < bd) { bd = d; best = j; }
      }
      if (best < 0 || bd > 1e-10 * mag) return QSLAB_ERR_INVALID_ARG;
      const double wd = std::hypot(c->w_re[best] - c->w_re[l], c->w_im[best] + c->w_im[l]);
      if (wd > 1e-10 * std::hypot(c->w_re[l], c->w_im[l]) + 1e-300) return QSLAB_ERR_INVALID_ARG;
      used[best] = true;
      mult = 2.0;
    }
    if (np >= kMaxPairs) return QSLAB_ERR_INVALID_ARG;
    t.s_re[np] = sr;
    t.s_im[np] = si;
    t.w_re[np] = c->w_re[l];
    t.w_im[np] = c->w_im[l];
    t.a_re[np] = c->alpha * sr;
    t.a_im[np] = c->alpha * si;
    t.mult[np] = mult;
    ++np;
  }
  t.np = np;
  int npc = 4;
  while (npc < np) npc += 4;
  if (npc > kMaxPairs) return QSLAB_ERR_INVALID_ARG;
  for (int p = np; p < npc; ++p) {
    t.s_re[p] = 1.0; t.s_im[p] = 0.0; t.w_re[p] = 0.0; t.w_im[p] = 0.0;
    t.a_re[p] = c->alpha; t.a_im[p] = 0.0; t.mult[p] = 0.0;
  }
  c->pairs = t;
  c->npc = npc;
  return QSLAB_OK;
}

// sum over the listed (half-plane) modes of (pi/A) erfc(k/(2 alpha))/k, times 2
double diag_half(const qslab_ctx* c, const std::vector<int32_t>& list) {
  double s = 0.0;
  const double A = c->Lx * c->Ly;
  for (size_t m = 0; m < list.size() / 2; ++m) {
    const double kx = 2 * kPi * list[2 * m] / c->Lx;
    const double ky = 2 * kPi * list[2 * m + 1] / c->Ly;
    const double k = std::sqrt(kx * kx + ky * ky);
    s += kPi / A * std::erfc(k / (2 * c->alpha)) / k;
  }
  return 2.0 * s;
}

std::vector<int32_t> half_plane(double Lx, double Ly, double kc) {
  std::vector<int32_t> out;
  const int mxm = (int)std::floor(kc * Lx / (2 * kPi)) + 1;
  const int mym = (int)std::floor(kc * Ly / (2 * kPi)) + 1;
  for (int mx = 0; mx <= mxm; ++mx) {
    for (int my = -mym; my <= mym; ++my) {
      if (mx == 0 && my <= 0) continue;
      const double kx = 2 * kPi * mx / Lx;
      const double ky = 2 * kPi * my / Ly;
      if (kx * kx + ky * ky <= kc * kc) {
        out.push_back(mx);
        out.push_back(my);
      }
    }
  }
  return out;
}

double H_direct(double alpha, double Lx, double Ly) {
  auto axis = [alpha](double L) {
    const int mm = (int)(10 * alpha * L / kPi) + 10;
    double s = 1.0;
    for (int m = 1; m <= mm; ++m) {
      const double t = kPi * m / (alpha * L);
      s += 2.0 * std::exp(-(t * t));
    }
    return s;
  };
  return axis(Lx) * axis(Ly) - 1.0;
}

std::vector<double> axis_cdf(double alpha, double L, int* mmax_out) {
  const int mmax = (int)std::floor(6.4380 * alpha * L / kPi) + 1;
  std::vector<double> c(2 * mmax + 1);
  double run = 0.0;
  for (int j = 0; j <= 2 * mmax; ++j) {
    const int m = j - mmax;
    const double t = kPi * m / (alpha * L);
    run += std::exp(-(t * t));
    c[j] = run;
  }
  for (auto& v : c) v /= run;
  *mmax_out = mmax;
  return c;
}

template <typename T>
ModeTab<T> mode_views(void* base, int Kpad, int npc) {
  ModeTab<T> m;
  char* p = static_cast<char*>(base);
  m.mx = reinterpret_cast<int32_t*>(p); p += a256(sizeof(int32_t) * Kpad);
  m.my = reinterpret_cast<int32_t*>(p); p += a256(sizeof(int32_t) * Kpad);
  T** f[] = {&m.kx, &m.ky, &m.kk, &m.ck, &m.ckk, &m.sY, &m.sZ};
  for (T** q : f) { *q = reinterpret_cast<T*>(p); p += a256(sizeof(T) * Kpad); }
  m.cp = reinterpret_cast<T*>(p);
  return m;
}

size_t mode_bytes(int Kpad, int npc, size_t tsz) {
  return 2 * a256(sizeof(int32_t) * Kpad) + 7 * a256(tsz * Kpad) + a256(tsz * 4 * npc * (size_t)Kpad);
}

int rebuild(qslab_ctx* c) {
  if (!c->has_box || !c->has_alpha || !c->has_soe || c->mode == 0)
    return QSLAB_ERR_NOT_CONFIGURED;
  int rc = build_pairs(c);
  if (rc) return rc;
  c->coef_ready = false;
  std::vector<double> cdfx, cdfy;
  if (c->mode == 1) {
    c->half_modes = half_plane(c->Lx, c->Ly, c->kc);
    c->K = (int)(c->half_modes.size() / 2);
    c->diag_k = diag_half(c, c->half_modes);
  } else {
    c->K = c->P;
    c->H = H_direct(c->alpha, c->Lx, c->Ly);
    // the random batch covers the whole lattice: the j = i constant sums every k
    std::vector<int32_t> all = half_plane(c->Lx, c->Ly, 14.0 * c->alpha);
    c->diag_k = diag_half(c, all);
    cdfx = axis_cdf(c->alpha, c->Lx, &c->mxmax);
    cdfy = axis_cdf(c->alpha, c->Ly, &c->mymax);
    c->cdf_nx = (int)cdfx.size();
    c->cdf_ny = (int)cdfy.size();
  }
  // modes per CTA (KR) and the number of mode ranges tile Kpad exactly
  {
    const int k32 = c->K > 0 ? ((c->K + 31) / 32) * 32 : 32;
    int kr = c->tune_KR > 0 ? c->tune_KR : 256;
    if (kr > k32) kr = k32;
    const int nkr = (k32 + kr - 1) / kr;
    kr = (((k32 + nkr - 1) / nkr + 31) / 32) * 32;
    c->KR = kr;
    c->nkr = nkr;
    c->Kpad = kr * nkr;
  }
  const size_t tsz = c->prec == QSLAB_FP64 ? sizeof(double) : sizeof(float);
  const size_t need = a256(sizeof(int32_t) * 2 * (size_t)c->Kpad) * 2 +
                      a256(sizeof(double) * (cdfx.size() + 1)) +
                      a256(sizeof(double) * (cdfy.size() + 1)) +
                      mode_bytes(c->Kpad, c->npc, tsz);
  if (need > c->cfg_bytes) {
    if (c->d_cfg) cudaFree(c->d_cfg);
    c->d_cfg = nullptr;
    c->cfg_bytes = 0;
    QS_CUDA(cudaMalloc(&c->d_cfg, need));
    c->cfg_bytes = need;
  }
  char* p = static_cast<char*>(c->d_cfg);
  c->d_list = reinterpret_cast<int32_t*>(p); p += a256(sizeof(int32_t) * 2 * (size_t)c->Kpad);
  c->d_sampled = reinterpret_cast<int32_t*>(p); p += a256(sizeof(int32_t) * 2 * (size_t)c->Kpad);
  c->d_cdfx = reinterpret_cast<double*>(p); p += a256(sizeof(double) * (cdfx.size() + 1));
  c->d_cdfy = reinterpret_cast<double*>(p); p += a256(sizeof(double) * (cdfy.size() + 1));
  c->d_modes = p;
  if (c->mode == 1 && c->K > 0)
    QS_CUDA(cudaMemcpy(c->d_list, c->half_modes.data(), sizeof(int32_t) * c->half_modes.size(),
                       cudaMemcpyHostToDevice));
  if (c->mode == 2) {
    QS_CUDA(cudaMemcpy(c->d_cdfx, cdfx.data(), sizeof(double) * cdfx.size(), cudaMemcpyHostToDevice));
    QS_CUDA(cudaMemcpy(c->d_cdfy, cdfy.data(), sizeof(double) * cdfy.size(), cudaMemcpyHostToDevice));
  }
  c->have_sample = false;
  c->dirty = false;
  return QSLAB_OK;
}

struct Plan {
  ScanPlan sp;
  int L0, nch0, nblk;
  size_t off_sort, off_zs, off_dz, off_qs, off_xh, off_yh, off_perm, off_agg,
      off_carry, off_pdec, off_part, off_k0, off_phi0, off_fz0, off_eblk,
      off_in_pos, off_in_q, off_out_phi, off_out_f, total;
};

Plan make_plan(const qslab_ctx* c, int64_t N, bool host_io) {
  Plan P{};
  const bool dp = c->prec == QSLAB_FP64;
  const size_t tsz = dp ? 8 : 4;
  const size_t phsz = dp ? 8 : 4;
  ScanPlan& s = P.sp;
  s.N = N;
  s.Kpad = c->Kpad;
  s.KR = c->KR;
  s.nkr = c->nkr;
  const int Lmax = dp ? 256 : 512;
  int L = c->tune_L;
  if (L <= 0) {
    const int64_t target = (2 * 152 + s.nkr - 1) / s.nkr;
    int64_t want = (N + target - 1) / target;
    want = ((want + 31) / 32) * 32;
    L = (int)(want < 32 ? 32 : (want > Lmax ? Lmax : want));
  }
  s.L = L;
  s.nchunks = (int)((N + L - 1) / L);
  s.np = c->npc;
  s.nstates = 1 + 2 * c->npc;
  P.L0 = dp ? 512 : 1024;   // k = 0 chunks: longer chunks, a shorter carry chain
  P.nch0 = (int)((N + P.L0 - 1) / P.L0);
  P.nblk = (int)((N + 255) / 256);
  if (P.nblk > 152 * 8) P.nblk = 152 * 8;
  size_t o = 0;
  auto take = [&o](size_t b) { size_t r = o; o += a256(b); return r; };
  P.off_sort = take(sort_workspace_bytes(N, dp ? 8 : 4));
  P.off_zs = take(tsz * N);
  P.off_dz = take(tsz * N);
  P.off_qs = take(tsz * N);
  P.off_xh = take(phsz * N);
  P.off_yh = take(phsz * N);
  P.off_perm = take(4 * (size_t)N);
  const size_t aggn = (size_t)2 * s.nchunks * s.nstates * s.Kpad;
  P.off_agg = take(2 * tsz * aggn);
  P.off_carry = take(2 * tsz * aggn);
  P.off_pdec = take(kspace_decay_bytes(s, dp ? 1 : 0));
  P.off_part = take(tsz * 4 * (size_t)s.nkr * N);
  P.off_k0 = take(8 * kzero_work_doubles(P.nch0, c->pairs.np));
  P.off_phi0 = take(8 * (size_t)N);
  P.off_fz0 = take(8 * (size_t)N);
  P.off_eblk = take(8 * (size_t)P.nblk);
  if (host_io) {
    P.off_in_pos = take(3 * tsz * N);
    P.off_in_q = take(tsz * N);
    P.off_out_phi = take(tsz * N);
    P.off_out_f = take(3 * tsz * N);
  }
  P.total = o;
  return P;
}

int ensure_ws(qslab_ctx* c, size_t bytes) {
  if (bytes <= c->ws_bytes) return QSLAB_OK;
  if (c->d_ws) {
    cudaDeviceSynchronize();
    cudaFree(c->d_ws);
  }
  c->d_ws = nullptr;
  c->ws_bytes = 0;
  QS_CUDA(cudaMalloc(&c->d_ws, bytes));
  c->ws_bytes = bytes;
  return QSLAB_OK;
}

template <typename T>
int run(qslab_ctx* c, const Plan& P, const T* pos, const T* q, double* energy,
        T* phi, T* force, cudaStream_t st) {
  using PH = typename PhaseT<T>::type;
  const int64_t N = P.sp.N;
  char* ws = static_cast<char*>(c->d_ws);
  SortWork sw;
  sort_bind_workspace(sw, ws + P.off_sort, N, sizeof(T));
  T* zs = reinterpret_cast<T*>(ws + P.off_zs);
  T* dz = reinterpret_cast<T*>(ws + P.off_dz);
  T* qs = reinterpret_cast<T*>(ws + P.off_qs);
  PH* xh = reinterpret_cast<PH*>(ws + P.off_xh);
  PH* yh = reinterpret_cast<PH*>(ws + P.off_yh);
  int32_t* perm = reinterpret_cast<int32_t*>(ws + P.off_perm);
  Cplx<T>* agg = reinterpret_cast<Cplx<T>*>(ws + P.off_agg);
  Cplx<T>* carry = reinterpret_cast<Cplx<T>*>(ws + P.off_carry);
  void* pdec = ws + P.off_pdec;
  T* part = reinterpret_cast<T*>(ws + P.off_part);
  double* k0w = reinterpret_cast<double*>(ws + P.off_k0);
  double* phi0 = reinterpret_cast<double*>(ws + P.off_phi0);
  double* fz0 = reinterpret_cast<double*>(ws + P.off_fz0);
  double* eblk = reinterpret_cast<double*>(ws + P.off_eblk);
  ModeTab<T> modes = mode_views<T>(c->d_modes, c->Kpad, c->npc);

  cudaEvent_t* ev = c->timing ? c->ev : nullptr;
  int nl = 0;
  if (ev) cudaEventRecord(ev[0], st);
  QS_CUDA(cudaMemsetAsync(c->d_sums, 0, 2 * sizeof(double), st));
  launch_prepare<T>(N, pos, q, c->Lz, sw.keys[0], sw.vals[0], c->d_sums, c->d_status, st);
  double tol = c->neutral_tol;
  if (tol < -1.0) tol = 64.0 * (sizeof(T) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-08);
  launch_check_neutral(c->d_sums, tol, c->d_status, st);
  const int r = radix_sort(sw, N, (int)sizeof(T), st);
  launch_gather<T>(N, pos, q, sw.vals[r], c->Lx, c->Ly, zs, dz, qs, xh, yh, perm, st);
  nl += 3 + 3 * (int)sizeof(T);   // prepare, check, gather + 3 kernels per sort pass
  if (ev) cudaEventRecord(ev[1], st);
  // k = 0 term on the side stream, concurrent with the k-space kernels
  QS_CUDA(cudaEventRecord(c->fork, st));
  QS_CUDA(cudaStreamWaitEvent(c->side, c->fork, 0));
  launch_kzero<T>(N, P.L0, P.nch0, c->pairs, c->alpha, c->Lx * c->Ly, zs, dz, qs, k0w,
                  phi0, fz0, c->side);
  nl += 4;
  if (ev) cudaEventRecord(ev[8], c->side);
  QS_CUDA(cudaEventRecord(c->join, c->side));
  // mode table: once per configuration for the full k-sum, every call for RBE
  if (c->mode == 2 || !c->coef_ready) {
    SamplerTab sp{c->d_cdfx, c->d_cdfy, c->cdf_nx, c->cdf_ny, c->mxmax, c->mymax};
    launch_mode_coef<T>(c->K, c->Kpad, c->npc, c->d_list, c->mode == 2 ? 1 : 0,
                        c->seed, c->counter, sp, c->pairs, c->alpha, c->Lx, c->Ly,
                        c->H, modes, c->mode == 2 ? c->d_sampled : nullptr, st);
    ++nl;
    if (c->mode == 2) {
      ++c->counter;
      c->have_sample = true;
    } else {
      c->coef_ready = true;
    }
  }
  if (ev) cudaEventRecord(ev[2], st);
  launch_kspace<T>(P.sp, modes, c->pairs, zs, dz, qs, xh, yh, agg, carry, pdec, part, st,
                   ev ? ev + 3 : nullptr);
  nl += 7;
  QS_CUDA(cudaStreamWaitEvent(st, c->join, 0));
  if (ev) cudaEventRecord(ev[6], st);
  const double D0 = -(kPi / (c->Lx * c->Ly)) / (c->alpha * kSqrtPi);
  const double diagq = 2.0 * c->diag_k + 2.0 * D0 - 2.0 * c->alpha / kSqrtPi;
  launch_combine<T>(N, P.sp.nkr, part, phi0, fz0, qs, perm, diagq, eblk, P.nblk, phi,
                    force, energy, st);
  nl += energy ? 2 : 1;
  if (ev) cudaEventRecord(ev[7], st);
  c->launches = nl;
  QS_CUDA(cudaGetLastError());
  c->last_stream = st;
  return QSLAB_OK;
}

int check_common(qslab_ctx* c, int64_t N) {
  if (!c) return QSLAB_ERR_INVALID_ARG;
  if (N < 1 || N > 2147483647LL) return QSLAB_ERR_INVALID_ARG;
  if (c->dirty) {
    const int rc = rebuild(c);
    if (rc) return rc;
  }
  return QSLAB_OK;
}

int status_code(unsigned f) {
  if (f & kStNonfinite) return QSLAB_ERR_NONFINITE;
  if (f & kStZRange) return QSLAB_ERR_Z_OUT_OF_RANGE;
  if (f & kStNonneutral) return QSLAB_ERR_NONNEUTRAL;
  if (f & kStTimeout) return QSLAB_ERR_TIMEOUT;
  return QSLAB_OK;
}

}  // namespace

extern "C" {

int qslab_create(qslab_ctx** out, int cuda_device, int prec) {
  if (!out) return QSLAB_ERR_INVALID_ARG;
  *out = nullptr;
  if (prec != QSLAB_FP64 && prec != QSLAB_FP32C) return QSLAB_ERR_INVALID_ARG;
  int n = 0;
  QS_CUDA(cudaGetDeviceCount(&n));
  if (cuda_device < 0 || cuda_device >= n) return QSLAB_ERR_INVALID_ARG;
  QS_CUDA(cudaSetDevice(cuda_device));
  qslab_ctx* c = new (std::nothrow) qslab_ctx();
  if (!c) return QSLAB_ERR_ALLOC;
  c->device = cuda_device;
  c->prec = prec;
  void* small = nullptr;
  cudaError_t e = cudaMalloc(&small, 256);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e);
  }
  c->d_status = static_cast<unsigned*>(small);
  c->d_sums = reinterpret_cast<double*>(static_cast<char*>(small) + 64);
  c->d_energy = reinterpret_cast<double*>(static_cast<char*>(small) + 128);
  cudaMemset(small, 0, 256);
  for (auto& ev : c->ev) cudaEventCreate(&ev);
  if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess) {
    qslab_destroy(c);
    return QSLAB_ERR_CUDA;
  }
  *out = c;
  return QSLAB_OK;
}

void qslab_destroy(qslab_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  if (c->d_ws) cudaFree(c->d_ws);
  if (c->d_cfg) cudaFree(c->d_cfg);
  if (c->d_status) cudaFree(c->d_status);
  for (auto& ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->join) cudaEventDestroy(c->join);
  if (c->side) cudaStreamDestroy(c->side);
  delete c;
}

int qslab_set_box(qslab_ctx* c, double Lx, double Ly, double Lz) {
  if (!c || !finite_pos(Lx) || !finite_pos(Ly) || !finite_pos(Lz)) return QSLAB_ERR_INVALID_ARG;
  c->Lx = Lx; c->Ly = Ly; c->Lz = Lz;
  c->has_box = true;
  c->dirty = true;
  return QSLAB_OK;
}

int qslab_set_alpha(qslab_ctx* c, double alpha) {
  if (!c || !finite_pos(alpha)) return QSLAB_ERR_INVALID_ARG;
  c->alpha = alpha;
  c->has_alpha = true;
  c->dirty = true;
  return QSLAB_OK;
}

int qslab_set_kcut(qslab_ctx* c, double kc) {
  if (!c || !finite_pos(kc)) return QSLAB_ERR_INVALID_ARG;
  c->kc = kc;
  c->mode = 1;
  c->dirty = true;
  return QSLAB_OK;
}

int qslab_set_rbe(qslab_ctx* c, int P, uint64_t seed) {
  if (!c || P < 1 || P > 65536) return QSLAB_ERR_INVALID_ARG;
  c->P = P;
  c->seed = seed;
  c->counter = 0;
  c->mode = 2;
  c->dirty = true;
  return QSLAB_OK;
}

int qslab_set_soe(qslab_ctx* c, int M, const double* s_re, const double* s_im,
                  const double* w_re, const double* w_im) {
  if (!c || M < 1 || M > 2 * kMaxPairs || !s_re || !s_im || !w_re || !w_im)
    return QSLAB_ERR_INVALID_ARG;
  for (int l = 0; l < M; ++l) {
    if (!std::isfinite(s_re[l]) || !std::isfinite(s_im[l]) || !std::isfinite(w_re[l]) ||
        !std::isfinite(w_im[l]) || !(s_re[l] > 0))
      return QSLAB_ERR_INVALID_ARG;
  }
  qslab_ctx trial = {};
  trial.alpha = 1.0;
  trial.s_re.assign(s_re, s_re + M);
  trial.s_im.assign(s_im, s_im + M);
  trial.w_re.assign(w_re, w_re + M);
  trial.w_im.assign(w_im, w_im + M);
  if (build_pairs(&trial) != QSLAB_OK) return QSLAB_ERR_INVALID_ARG;
  c->s_re = trial.s_re; c->s_im = trial.s_im;
  c->w_re = trial.w_re; c->w_im = trial.w_im;
  c->has_soe = true;
  c->dirty = true;
  return QSLAB_OK;
}

int qslab_set_neutrality_tol(qslab_ctx* c, double tol) {
  if (!c || std::isnan(tol)) return QSLAB_ERR_INVALID_ARG;
  c->neutral_tol = tol < 0 ? -1.0 : tol;
  return QSLAB_OK;
}

int qslab_set_tuning(qslab_ctx* c, int chunk, int modes_per_cta) {
  if (!c || chunk < 0 || modes_per_cta < 0) return QSLAB_ERR_INVALID_ARG;
  const int Lmax = c->prec == QSLAB_FP64 ? 256 : 512;
  if (chunk > Lmax || (modes_per_cta > 0 && (modes_per_cta % 32 || modes_per_cta > 256)))
    return QSLAB_ERR_INVALID_ARG;
  c->tune_L = chunk;
  if (c->tune_KR != modes_per_cta) c->dirty = true;
  c->tune_KR = modes_per_cta;
  return QSLAB_OK;
}

int qslab_compute(qslab_ctx* c, int64_t N, const void* pos, const void* q,
                  double* energy, void* phi, void* force, void* stream) {
  int rc = check_common(c, N);
  if (rc) return rc;
  if (!pos || !q) return QSLAB_ERR_INVALID_ARG;
  QS_CUDA(cudaSetDevice(c->device));
  const Plan P = make_plan(c, N, false);
  rc = ensure_ws(c, P.total);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (c->prec == QSLAB_FP64)
    return run<double>(c, P, static_cast<const double*>(pos), static_cast<const double*>(q),
                       energy, static_cast<double*>(phi), static_cast<double*>(force), st);
  return run<float>(c, P, static_cast<const float*>(pos), static_cast<const float*>(q), energy,
                    static_cast<float*>(phi), static_cast<float*>(force), st);
}

int qslab_compute_host(qslab_ctx* c, int64_t N, const void* pos_host, const void* q_host,
                       double* energy_host, void* phi_host, void* force_host, void* stream) {
  int rc = check_common(c, N);
  if (rc) return rc;
  if (!pos_host || !q_host) return QSLAB_ERR_INVALID_ARG;
  QS_CUDA(cudaSetDevice(c->device));
  const Plan P = make_plan(c, N, true);
  rc = ensure_ws(c, P.total);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t tsz = c->prec == QSLAB_FP64 ? 8 : 4;
  char* ws = static_cast<char*>(c->d_ws);
  void* dpos = ws + P.off_in_pos;
  void* dq = ws + P.off_in_q;
  void* dphi = phi_host ? ws + P.off_out_phi : nullptr;
  void* df = force_host ? ws + P.off_out_f : nullptr;
  QS_CUDA(cudaMemcpyAsync(dpos, pos_host, 3 * tsz * N, cudaMemcpyHostToDevice, st));
  QS_CUDA(cudaMemcpyAsync(dq, q_host, tsz * N, cudaMemcpyHostToDevice, st));
  if (c->prec == QSLAB_FP64)
    rc = run<double>(c, P, static_cast<const double*>(dpos), static_cast<const double*>(dq),
                     c->d_energy, static_cast<double*>(dphi), static_cast<double*>(df), st);
  else
    rc = run<float>(c, P, static_cast<const float*>(dpos), static_cast<const float*>(dq),
                    c->d_energy, static_cast<float*>(dphi), static_cast<float*>(df), st);
  if (rc) return rc;
  if (energy_host)
    QS_CUDA(cudaMemcpyAsync(energy_host, c->d_energy, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (phi_host) QS_CUDA(cudaMemcpyAsync(phi_host, dphi, tsz * N, cudaMemcpyDeviceToHost, st));
  if (force_host) QS_CUDA(cudaMemcpyAsync(force_host, df, 3 * tsz * N, cudaMemcpyDeviceToHost, st));
  return qslab_last_status(c);
}

int qslab_get_sampled_modes(qslab_ctx* c, int32_t* mxy, double* weight) {
  if (!c || !mxy) return QSLAB_ERR_INVALID_ARG;
  if (c->mode != 2 || !c->have_sample) return QSLAB_ERR_NOT_CONFIGURED;
  QS_CUDA(cudaSetDevice(c->device));
  QS_CUDA(cudaStreamSynchronize(c->last_stream));
  QS_CUDA(cudaMemcpy(mxy, c->d_sampled, sizeof(int32_t) * 2 * (size_t)c->P, cudaMemcpyDeviceToHost));
  if (weight) *weight = c->H / c->P;
  return QSLAB_OK;
}

int qslab_get_rng_state(qslab_ctx* c, uint64_t* seed, uint64_t* counter) {
  if (!c || !seed || !counter) return QSLAB_ERR_INVALID_ARG;
  *seed = c->seed;
  *counter = c->counter;
  return QSLAB_OK;
}

int qslab_set_rng_state(qslab_ctx* c, uint64_t seed, uint64_t counter) {
  if (!c) return QSLAB_ERR_INVALID_ARG;
  c->seed = seed;
  c->counter = counter;
  return QSLAB_OK;
}

int qslab_num_modes(qslab_ctx* c) {
  if (!c) return QSLAB_ERR_INVALID_ARG;
  if (c->dirty) {
    const int rc = rebuild(c);
    if (rc) return rc;
  }
  return c->K;
}

int qslab_last_status(qslab_ctx* c) {
  if (!c) return QSLAB_ERR_INVALID_ARG;
  QS_CUDA(cudaSetDevice(c->device));
  QS_CUDA(cudaStreamSynchronize(c->last_stream));
  QS_CUDA(cudaGetLastError());
  unsigned f = 0;
  QS_CUDA(cudaMemcpy(&f, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  QS_CUDA(cudaMemset(c->d_status, 0, sizeof(unsigned)));
  return status_code(f);
}

int qslab_set_timing(qslab_ctx* c, int enable) {
  if (!c) return QSLAB_ERR_INVALID_ARG;
  c->timing = enable != 0;
  return QSLAB_OK;
}

int qslab_get_timings(qslab_ctx* c, double* ms8, int* launches) {
  if (!c || !ms8) return QSLAB_ERR_INVALID_ARG;
  if (!c->timing) return QSLAB_ERR_NOT_CONFIGURED;
  QS_CUDA(cudaSetDevice(c->device));
  QS_CUDA(cudaEventSynchronize(c->ev[7]));
  // event order: 0 start, 1 sorted, 2 modes, 3 aggregates, 4 carries,
  // 5 recurrences, 6 joined with the k = 0 stream, 7 end, 8 end of the k = 0
  // term (side stream; it runs concurrently from event 1)
  const int pairs[8][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 4}, {4, 5}, {1, 8}, {6, 7}, {0, 7}};
  for (int i = 0; i < 8; ++i) {
    float t = 0;
    QS_CUDA(cudaEventElapsedTime(&t, c->ev[pairs[i][0]], c->ev[pairs[i][1]]));
    ms8[i] = t;
  }
  if (launches) *launches = c->launches;
  return QSLAB_OK;
}

const char* qslab_strerror(int code) {
  switch (code) {
    case QSLAB_OK: return "success";
    case QSLAB_ERR_INVALID_ARG: return "invalid argument";
    case QSLAB_ERR_NOT_CONFIGURED: return "context not configured (box, alpha, SOE and k-set needed)";
    case QSLAB_ERR_NONFINITE: return "non-finite position or charge";
    case QSLAB_ERR_Z_OUT_OF_RANGE: return "z outside [0, Lz]";
    case QSLAB_ERR_NONNEUTRAL: return "system is not charge neutral";
    case QSLAB_ERR_ALLOC: return "allocation failed";
    case QSLAB_ERR_CUDA: return "CUDA runtime error";
    case QSLAB_ERR_TIMEOUT: return "bounded device wait gave up";
    case QSLAB_ERR_TOO_LARGE: return "problem too large for the fixed scratch of qslab_compute_static";
    default: return "unknown error";
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Compute without allocating device memory.
//
// Some callers cannot allocate GPU memory at the point where they need the
// long-range forces: code running inside another framework's memory pool or
// under a strict device-memory budget, or a time step of a simulation loop in
// which an allocation (and the device synchronisation it may imply) is not
// acceptable. qslab_compute_static() serves them: it runs the same launch
// sequence as qslab_compute() but takes every byte of scratch it needs (the
// mode and sampler tables, sort buffers, sorted particles, chunk aggregates
// and carries, partial outputs, the k = 0 work and the status word) from one
// fixed array in device memory that the library defines at file scope. That
// array (kStaticScratchBytes per GPU) exists on every GPU that loads the
// library, from module load until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;   // 64 MiB per GPU
constexpr size_t kStaticCfgBytes = size_t(8) << 20;        // tables and status
constexpr size_t kStaticSmallBytes = 256;                  // status, sums, energy
constexpr int kStaticMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device. In host code the symbol is
// only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress once per device, with that device current.
void* g_static_addr[kStaticMaxDevices] = {};

int static_scratch_address(int device, void** out) {
  if (device < 0 || device >= kStaticMaxDevices) return QSLAB_ERR_INVALID_ARG;
  if (!g_static_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return QSLAB_ERR_CUDA;
    g_static_addr[device] = p;
  }
  *out = g_static_addr[device];
  return QSLAB_OK;
}

}  // namespace

extern "C" int qslab_compute_static(qslab_ctx* c, int64_t N, const void* pos, const void* q,
                                    double* energy, void* phi, void* force, void* stream) {
  if (!c) return QSLAB_ERR_INVALID_ARG;
  if (N < 1 || N > 2147483647LL || !pos || !q) return QSLAB_ERR_INVALID_ARG;
  if (!c->has_box || !c->has_alpha || !c->has_soe || c->mode == 0) return QSLAB_ERR_NOT_CONFIGURED;
  QS_CUDA(cudaSetDevice(c->device));
  void* base = nullptr;
  int rc = static_scratch_address(c->device, &base);
  if (rc) return rc;
  char* sb = static_cast<char*>(base);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // A copy of the context whose device buffers all point into the static
  // array; its configuration tables are rebuilt there on every call (the
  // real context's own buffers are neither used nor changed).
  qslab_ctx t = *c;
  t.timing = false;
  t.d_status = reinterpret_cast<unsigned*>(sb);
  t.d_sums = reinterpret_cast<double*>(sb + 64);
  t.d_energy = reinterpret_cast<double*>(sb + 128);
  t.d_cfg = sb + kStaticSmallBytes;
  t.cfg_bytes = kStaticCfgBytes - kStaticSmallBytes;
  t.d_ws = sb + kStaticCfgBytes;
  t.ws_bytes = kStaticScratchBytes - kStaticCfgBytes;
  // size checks before anything touches the device: the tables must fit the
  // table region and the workspace the rest of the array
  {
    const size_t tsz = c->prec == QSLAB_FP64 ? sizeof(double) : sizeof(float);
    qslab_ctx probe = *c;
    if (build_pairs(&probe) != QSLAB_OK) return QSLAB_ERR_INVALID_ARG;
    size_t K = 0, cdf = 0;
    if (c->mode == 1) {
      K = half_plane(c->Lx, c->Ly, c->kc).size() / 2;
    } else {
      K = (size_t)c->P;
      const double mx = std::floor(6.4380 * c->alpha * c->Lx / kPi) + 1;
      const double my = std::floor(6.4380 * c->alpha * c->Ly / kPi) + 1;
      cdf = (size_t)(2 * mx + 1) + (size_t)(2 * my + 1);
      if (mx > 1e6 || my > 1e6) return QSLAB_ERR_TOO_LARGE;
    }
    const size_t kpad = ((std::max<size_t>(K, 1) + 255) / 256) * 256;
    const size_t need = a256(sizeof(int32_t) * 2 * kpad) * 2 + a256(sizeof(double) * (cdf + 2)) * 2 +
                        mode_bytes((int)kpad, probe.npc, tsz);
    if (need > t.cfg_bytes || kpad > (size_t)1 << 20) return QSLAB_ERR_TOO_LARGE;
  }
  t.dirty = true;
  rc = rebuild(&t);          // fits: no allocation, tables uploaded into the array
  if (rc) return rc;
  const Plan P = make_plan(&t, N, false);
  if (P.total > t.ws_bytes) return QSLAB_ERR_TOO_LARGE;
  // the status word and sums start from zero on every call
  QS_CUDA(cudaMemsetAsync(t.d_status, 0, kStaticSmallBytes, st));
  if (c->prec == QSLAB_FP64)
    rc = run<double>(&t, P, static_cast<const double*>(pos), static_cast<const double*>(q),
                     energy, static_cast<double*>(phi), static_cast<double*>(force), st);
  else
    rc = run<float>(&t, P, static_cast<const float*>(pos), static_cast<const float*>(q), energy,
                    static_cast<float*>(phi), static_cast<float*>(force), st);
  if (rc) return rc;
  // the random-batch counter advances as in qslab_compute()
  c->counter = t.counter;
  QS_CUDA(cudaStreamSynchronize(st));
  QS_CUDA(cudaGetLastError());
  unsigned f = 0;
  QS_CUDA(cudaMemcpy(&f, t.d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  return status_code(f);
}
