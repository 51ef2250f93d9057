// qslab C ABI: context, configuration, host-side precompute (k-mode lists,
// SOE pair representatives, the normaliser H, the sampler's cumulative
// tables, the j = i constants), workspace management and the launch
// sequence of one compute call.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "qslab.h"
#include "qslab_internal.h"
#include "qslab_real.h"
#include "qslab_virial.h"
#include "qslab_md.h"

using namespace qslab;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.7724538509055160273;

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Host-side description of a call's replicas and the tables derived from
// it. Cached in the context: rebuilt only when the configuration, the
// replica offsets, the boxes or the tuning change.
struct Tables {
  bool valid = false;
  uint64_t cfg_version = 0;
  // key
  int R = 0;
  std::vector<int64_t> off;     // R + 1
  std::vector<double> box;      // 3 R
  int tune_L = 0, tune_KR = 0;
  // derived
  std::vector<RepInfo> info;
  std::vector<int32_t> chunk_rep, zchunk_rep, gstart, group_rep, zgstart, zgroup_rep, list;
  std::vector<double> cdf;
  std::vector<double> vdiag;    // 3 R: j = i lateral virial per unit sum q^2 (xx, yy, xy)
  int Kpad = 32, KR = 32, nkr = 1, L = 32, L0 = 128;
  int nchunks = 0, nz = 0, ngroups = 0, nzgroups = 0;
  int kflat = 1, zflat = 1;     // every replica's carry chains are one group
  int64_t N = 0;
  // device layout of the table buffer
  size_t o_info = 0, o_crep = 0, o_zrep = 0, o_gstart = 0, o_grep = 0, o_zgstart = 0, o_zgrep = 0,
         o_list = 0, o_cdf = 0, o_trig = 0, o_vdiag = 0,
         o_sampled = 0, o_modes = 0, bytes = 0;
};

struct qslab_ctx {
  int device = 0;
  int sm_count = 152;           // multiprocessors of the device (queried at creation)
  int prec = QSLAB_FP64;
  // configuration
  double Lx = 0, Ly = 0, Lz = 0, alpha = 0;
  bool has_box = false, has_alpha = false, has_soe = false;
  int mode = 0;                 // 1 full k-sum, 2 random batch
  double kc = 0;
  int P = 0;
  uint64_t seed = 0;
  std::vector<double> s_re, s_im, w_re, w_im;
  double neutral_tol = -2.0;    // < -1: default for the precision
  int tune_L = 0, tune_KR = 0;
  bool timing = false;
  double rc = 0;                // real-space cut-off (0: not set)
  WallTab walls{};              // charged walls (walls.on = 0: none)
  int sampler = QSLAB_SAMPLER_IID;   // random-batch k-sampler
  int mh_thin = 1;              // Metropolis downsampling rate
  // Langevin dynamics driver
  bool md_on = false;
  MDDev md{};
  double lj_eps = 0, lj_sigma = 0;
  void* d_md = nullptr;         // F_lr, F_rs (3N each), partial sums, e_lr, e_rs
  size_t md_bytes = 0;
  uint64_t* d_md_ctr = nullptr; // step counter of the noise (device)
  // derived configuration
  bool cfg_dirty = true;
  uint64_t cfg_version = 0;
  PairTab pairs{};
  int npc = 4;                  // pair count the kernels are compiled for
  Tables tab;
  // device tables (per configuration and replica geometry)
  void* d_tab = nullptr;
  size_t tab_bytes = 0;
  bool coef_ready = false;      // full-k mode tables filled for tab
  // small persistent buffers: status word, energy, random-batch counter
  // (ctr[0] = counter of the next call, ctr[1] = counter of the last one)
  unsigned* d_status = nullptr;
  double* d_energy = nullptr;
  uint64_t* d_ctr = nullptr;
  // per-call workspace
  void* d_ws = nullptr;
  size_t ws_bytes = 0;
  void* d_rs_ws = nullptr;      // real-space workspace
  size_t rs_ws_bytes = 0;
  cudaStream_t last_stream = nullptr;
  bool primed = false;          // an energy-only call left its workspace for the adjoint
  bool have_sample = false;
  int last_R = 1;
  cudaEvent_t ev[9] = {};
  int launches = 0;
  // the k = 0 term runs on a side stream, forked from and joined to the
  // caller's stream with these events (capturable in a CUDA graph)
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  // an MD force pass runs the real-space call on its own side stream,
  // concurrently with the long-range call (their outputs are disjoint)
  cudaStream_t rs_side = nullptr;
  cudaEvent_t rs_fork = nullptr, rs_join = nullptr;
  // the mode tables (sampling, Metropolis chain, coefficients) need only
  // the call counter and the configuration's tables: they are built on a
  // third side stream, concurrently with the sort and the gather
  cudaStream_t tab_side = nullptr;
  cudaEvent_t tab_fork = nullptr, tab_join = nullptr;
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

// Every device allocation of the library goes through lib_malloc: it counts
// them (qslab_debug_alloc_count) and, for failure-injection tests, makes the
// next g_fail_allocs of them fail as an out-of-memory cudaMalloc would, on
// the host, without calling the runtime.
std::atomic<long long> g_alloc_count{0};
std::atomic<int> g_fail_allocs{0};

cudaError_t lib_malloc(void** p, size_t bytes) {
  int left = g_fail_allocs.load();
  while (left > 0) {
    if (g_fail_allocs.compare_exchange_weak(left, left - 1)) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) ++g_alloc_count;
  return e;
}

// Grow a device buffer to at least `need` bytes. The new buffer is allocated
// before the old one is released, so that a failed allocation leaves the old
// buffer and its contents in place; only when that fails is the old buffer
// released (*released = true) and the allocation tried once more.
int grow_buffer(void** buf, size_t* have, size_t need, bool* released) {
  if (need <= *have && *buf) return QSLAB_OK;
  void* nb = nullptr;
  cudaError_t e = lib_malloc(&nb, need);
  if (e != cudaSuccess && *buf) {
    cudaDeviceSynchronize();
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    if (released) *released = true;
    e = lib_malloc(&nb, need);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  if (*buf) {
    cudaDeviceSynchronize();
    cudaFree(*buf);
  }
  *buf = nb;
  *have = need;
  return QSLAB_OK;
}

constexpr int kMaxReplicas = 1 << 20;
constexpr int kFlatChunks = 32;   // carry chains shorter than this are one group

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

int ensure_config(qslab_ctx* c) {
  if (!c->has_alpha || !c->has_soe || c->mode == 0) return QSLAB_ERR_NOT_CONFIGURED;
  if (!c->cfg_dirty) return QSLAB_OK;
  const int rc = build_pairs(c);
  if (rc) return rc;
  ++c->cfg_version;
  c->cfg_dirty = false;
  return QSLAB_OK;
}

// The k-derivative of the j = i term of a mode, (pi/(2A)) d/dk [2 erfc(k/(2 alpha))/k],
// weighted by k_a k_b/k, added to vd[3] (xx, yy, xy) with multiplicity w: the
// j = i part of the lateral virial per unit sum q^2.
void add_vdiag(double alpha, double A, double kx, double ky, double w, double* vd) {
  const double k = std::sqrt(kx * kx + ky * ky);
  const double dG = -2.0 * std::erfc(k / (2 * alpha)) / (k * k) -
                    2.0 * std::exp(-k * k / (4 * alpha * alpha)) / (alpha * kSqrtPi * k);
  const double t = w * kPi / (2 * A) * dG / k;
  vd[0] += t * kx * kx;
  vd[1] += t * ky * ky;
  vd[2] += t * kx * ky;
}

// (pi/A) erfc(k/(2 alpha))/k summed over the listed (half-plane) modes, times 2
// (k and -k); vd (may be NULL) receives the lateral virial constants
double diag_half(double alpha, double Lx, double Ly, const int32_t* list, size_t K,
                 double* vd = nullptr) {
  double s = 0.0;
  const double A = Lx * Ly;
  for (size_t m = 0; m < K; ++m) {
    const double kx = 2 * kPi * list[2 * m] / Lx;
    const double ky = 2 * kPi * list[2 * m + 1] / Ly;
    const double k = std::sqrt(kx * kx + ky * ky);
    s += kPi / A * std::erfc(k / (2 * alpha)) / k;
    if (vd) add_vdiag(alpha, A, kx, ky, 2.0, vd);
  }
  return 2.0 * s;
}

// The same over every k != 0 (the random batch samples the whole lattice);
// erfc(k/(2 alpha)) < 1e-21 beyond |k| = 14 alpha. The terms of (mx, my) and
// (mx, -my) are equal and are summed once.
double diag_all(double alpha, double Lx, double Ly, double* vd = nullptr) {
  const double kc = 14.0 * alpha;
  const int mxm = (int)std::floor(kc * Lx / (2 * kPi)) + 1;
  const int mym = (int)std::floor(kc * Ly / (2 * kPi)) + 1;
  const double A = Lx * Ly;
  double s = 0.0;
  for (int mx = 0; mx <= mxm; ++mx) {
    for (int my = (mx == 0 ? 1 : 0); my <= mym; ++my) {
      const double kx = 2 * kPi * mx / Lx;
      const double ky = 2 * kPi * my / Ly;
      const double k2 = kx * kx + ky * ky;
      if (k2 > kc * kc) break;
      const double k = std::sqrt(k2);
      const double t = kPi / A * std::erfc(k / (2 * alpha)) / k;
      const double mult = (mx > 0 && my > 0) ? 2.0 : 1.0;
      s += mult * t;
      // xx, yy are even in mx and in my; xy cancels over the lattice
      if (vd) add_vdiag(alpha, A, kx, ky, 2.0 * mult, vd);
    }
  }
  if (vd) vd[2] = 0.0;
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

int axis_mmax(double alpha, double L) { return (int)std::floor(6.4380 * alpha * L / kPi) + 1; }

std::vector<double> axis_cdf(double alpha, double L, int* mmax_out) {
  const int mmax = axis_mmax(alpha, L);
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

// Metropolis log-weights of one axis (App. G): -(pi m/(alpha L))^2 - log q(m)
// for m = -mmax..mmax, with q(m) the probability that the proposal normal of
// variance (alpha L)^2/(2 pi^2) rounds to m (the erf difference of App. G,
// written with erfc so that the tail keeps its relative accuracy).
std::vector<double> axis_mh_logw(double alpha, double L, int mmax) {
  std::vector<double> v(2 * mmax + 1);
  const double a = kPi / (2.0 * alpha * L);
  for (int j = 0; j <= 2 * mmax; ++j) {
    const int m = j - mmax;
    const double am = std::fabs((double)m);
    const double q = m == 0 ? std::erf(a)
                            : 0.5 * (std::erfc(a * (2.0 * am - 1.0)) - std::erfc(a * (2.0 * am + 1.0)));
    const double t = kPi * m / (alpha * L);
    v[j] = -(t * t) - std::log(q);
  }
  return v;
}

template <typename T>
ModeTab<T> mode_views(void* base, size_t n, int npc) {
  ModeTab<T> m;
  char* p = static_cast<char*>(base);
  m.mx = reinterpret_cast<int32_t*>(p); p += a256(sizeof(int32_t) * n);
  m.my = reinterpret_cast<int32_t*>(p); p += a256(sizeof(int32_t) * n);
  T** f[] = {&m.kx, &m.ky, &m.kk, &m.ck, &m.ckk, &m.sY, &m.sZ};
  for (T** q : f) { *q = reinterpret_cast<T*>(p); p += a256(sizeof(T) * n); }
  m.cp = reinterpret_cast<T*>(p);
  (void)npc;
  return m;
}

size_t mode_bytes(size_t n, int npc, size_t tsz) {
  return 2 * a256(sizeof(int32_t) * n) + 7 * a256(tsz * n) + a256(tsz * 4 * npc * n);
}

bool same_key(const Tables& t, const qslab_ctx* c, int R, const int64_t* off, const double* box) {
  if (!t.valid || t.cfg_version != c->cfg_version || t.R != R || t.tune_L != c->tune_L ||
      t.tune_KR != c->tune_KR)
    return false;
  return std::memcmp(t.off.data(), off, sizeof(int64_t) * (R + 1)) == 0 &&
         std::memcmp(t.box.data(), box, sizeof(double) * 3 * R) == 0;
}

// Automatic chunk length of the k-space passes. The passes run two CTAs per
// SM, one per (chunk, mode range), all of about the same duration, so the
// grid runs in waves of 2 x SMs CTAs:
//   - small problems: about one wave, chunks of 16 below about 5000
//     particles (shorter serial loops beat the extra carry work there), else
//     a multiple of 32;
//   - large ones: the longest chunks, except that among the multiples of 32
//     in [3/4 Lmax, Lmax] the one whose last wave is fullest is taken (a last
//     wave of 0.4 leaves most SMs idle for one CTA time);
//   - FP32 with four or more mode ranges (full k-sums of thousands of modes,
//     whose parallelism comes from the modes): at most 256 particles, which
//     halves the FP32 steps between two double-float carries and costs no
//     time there.
int auto_chunk(const qslab_ctx* c, const Tables& t, int R, const int64_t* off, int64_t N) {
  const bool dp = c->prec == QSLAB_FP64;
  int Lmax = dp ? 256 : 512;
  if (!dp && t.nkr >= 4) Lmax = 256;
  const int64_t slots = 2 * (int64_t)c->sm_count;
  const int64_t target = (slots + t.nkr - 1) / t.nkr;
  int64_t want = (N + target - 1) / target;
  want = want <= 16 ? 16 : ((want + 31) / 32) * 32;
  if (want < Lmax) return (int)want;
  int best = Lmax;
  double best_eff = -1.0;
  for (int L = Lmax; L >= (3 * Lmax) / 4; L -= 32) {
    int64_t ctas = 0;
    for (int r = 0; r < R; ++r) ctas += (off[r + 1] - off[r] + L - 1) / L;
    ctas *= t.nkr;
    const int64_t waves = (ctas + slots - 1) / slots;
    const double eff = (double)ctas / (double)(waves * slots);
    if (eff > best_eff + 0.02) { best_eff = eff; best = L; }
  }
  return best;
}

// Host part of the tables of a call (no device work). Validates the replica
// offsets and boxes.
int build_tables(const qslab_ctx* c, int R, const int64_t* off, const double* box, Tables& t,
                 const Tables* prev = nullptr) {
  if (R < 1 || R > kMaxReplicas || !off || !box) return QSLAB_ERR_INVALID_ARG;
  if (off[0] != 0) return QSLAB_ERR_INVALID_ARG;
  for (int r = 0; r < R; ++r) {
    const int64_t n = off[r + 1] - off[r];
    if (n < 0 || n > 2147483647LL) return QSLAB_ERR_INVALID_ARG;
    if (!finite_pos(box[3 * r]) || !finite_pos(box[3 * r + 1]) || !finite_pos(box[3 * r + 2]))
      return QSLAB_ERR_INVALID_ARG;
  }
  const int64_t N = off[R];
  if (N < 1 || N > 2147483647LL) return QSLAB_ERR_INVALID_ARG;
  const bool dp = c->prec == QSLAB_FP64;
  t = Tables();
  t.cfg_version = c->cfg_version;
  t.R = R;
  t.off.assign(off, off + R + 1);
  t.box.assign(box, box + 3 * R);
  t.tune_L = c->tune_L;
  t.tune_KR = c->tune_KR;
  t.N = N;
  t.info.assign(R, RepInfo{});
  t.vdiag.assign(3 * (size_t)R, 0.0);
  const double alpha = c->alpha;
  // the per-box data of the previous tables still hold when only the
  // offsets or the launch shape changed
  const bool reuse = prev && prev->valid && prev->cfg_version == c->cfg_version &&
                     prev->R == R &&
                     std::memcmp(prev->box.data(), box, sizeof(double) * 3 * R) == 0;
  if (reuse) {
    t.list = prev->list;
    t.cdf = prev->cdf;
  }
  // modes, sampler tables and j = i constants per replica (memoised by box)
  std::map<std::pair<double, double>, int> seen;
  int Kmax = 1;
  for (int r = 0; r < R; ++r) {
    RepInfo& ri = t.info[r];
    ri.off = off[r];
    ri.n = (int32_t)(off[r + 1] - off[r]);
    ri.Lx = box[3 * r]; ri.Ly = box[3 * r + 1]; ri.Lz = box[3 * r + 2];
    ri.area = ri.Lx * ri.Ly;
    ri.k0pre = 2.0 * kPi / ri.area;
    auto it = seen.find({ri.Lx, ri.Ly});
    if (reuse) {
      const RepInfo& o = prev->info[r];
      ri.K = o.K; ri.list0 = o.list0; ri.cdfx0 = o.cdfx0; ri.nx = o.nx;
      ri.cdfy0 = o.cdfy0; ri.ny = o.ny; ri.mxmax = o.mxmax; ri.mymax = o.mymax;
      ri.H = o.H; ri.diagq = o.diagq;
      std::copy(prev->vdiag.begin() + 3 * r, prev->vdiag.begin() + 3 * r + 3, t.vdiag.begin() + 3 * r);
    } else if (it != seen.end()) {
      const RepInfo& o = t.info[it->second];
      ri.K = o.K; ri.list0 = o.list0; ri.cdfx0 = o.cdfx0; ri.nx = o.nx;
      ri.cdfy0 = o.cdfy0; ri.ny = o.ny; ri.mxmax = o.mxmax; ri.mymax = o.mymax;
      ri.H = o.H; ri.diagq = o.diagq;
      std::copy(t.vdiag.begin() + 3 * it->second, t.vdiag.begin() + 3 * it->second + 3,
                t.vdiag.begin() + 3 * r);
    } else {
      seen[{ri.Lx, ri.Ly}] = r;
      double dk = 0.0;
      if (c->mode == 1) {
        const std::vector<int32_t> l = half_plane(ri.Lx, ri.Ly, c->kc);
        ri.K = (int32_t)(l.size() / 2);
        ri.list0 = (int32_t)(t.list.size() / 2);
        dk = diag_half(alpha, ri.Lx, ri.Ly, l.data(), l.size() / 2, &t.vdiag[3 * (size_t)r]);
        t.list.insert(t.list.end(), l.begin(), l.end());
        if (t.list.size() > (size_t)1 << 30) return QSLAB_ERR_INVALID_ARG;
      } else {
        ri.K = c->P;
        ri.H = H_direct(alpha, ri.Lx, ri.Ly);
        dk = diag_all(alpha, ri.Lx, ri.Ly, &t.vdiag[3 * (size_t)r]);
        int mx = 0, my = 0;
        const std::vector<double> cx = axis_cdf(alpha, ri.Lx, &mx);
        const std::vector<double> cy = axis_cdf(alpha, ri.Ly, &my);
        ri.cdfx0 = (int32_t)t.cdf.size(); ri.nx = (int32_t)cx.size(); ri.mxmax = mx;
        t.cdf.insert(t.cdf.end(), cx.begin(), cx.end());
        ri.cdfy0 = (int32_t)t.cdf.size(); ri.ny = (int32_t)cy.size(); ri.mymax = my;
        t.cdf.insert(t.cdf.end(), cy.begin(), cy.end());
        const std::vector<double> lx = axis_mh_logw(alpha, ri.Lx, mx);
        const std::vector<double> ly = axis_mh_logw(alpha, ri.Ly, my);
        t.cdf.insert(t.cdf.end(), lx.begin(), lx.end());
        t.cdf.insert(t.cdf.end(), ly.begin(), ly.end());
        if (t.cdf.size() > (size_t)1 << 28) return QSLAB_ERR_INVALID_ARG;
      }
      // j = i constant per unit q_i^2 of the potential: k != 0 (Eq. 3.20),
      // k = 0 (-2 sqrt(pi)/(alpha A), the j = i term of Eq. 2.16) and the
      // self term -2 alpha/sqrt(pi) (Eq. 2.12)
      const double D0 = -(kPi / ri.area) / (alpha * kSqrtPi);
      ri.diagq = 2.0 * dk + 2.0 * D0 - 2.0 * alpha / kSqrtPi;
    }
    Kmax = std::max(Kmax, (int)ri.K);
  }
  // modes per CTA (KR) and the number of mode ranges tile Kpad exactly
  {
    const int k32 = ((Kmax + 31) / 32) * 32;
    int kr = c->tune_KR > 0 ? c->tune_KR : 256;
    if (kr > k32) kr = k32;
    const int nkr = (k32 + kr - 1) / kr;
    kr = (((k32 + nkr - 1) / nkr + 31) / 32) * 32;
    t.KR = kr;
    t.nkr = nkr;
    t.Kpad = kr * nkr;
  }
  if ((size_t)R * t.Kpad > ((size_t)1 << 31) / 64) return QSLAB_ERR_INVALID_ARG;
  // chunk length: about two CTAs per SM over all replicas and mode ranges
  int L = c->tune_L;
  if (L <= 0) L = auto_chunk(c, t, R, off, N);
  t.L = L;
  // k = 0 chunks: short sequential loops, many threads (no longer than the
  // k-space chunks, so that small slabs get more, shorter chains)
  t.L0 = std::min(128, L);
  // carry chains shorter than kFlatChunks chunks are one group (a single
  // serial replay); the rule looks at each replica alone, so that a replica
  // gets the same arithmetic in a batch as in a call of its own. When every
  // chain is one group, the group and chain phases are not launched.
  // chunks, k = 0 chunks and carry groups per replica
  for (int r = 0; r < R; ++r) {
    RepInfo& ri = t.info[r];
    ri.c0 = (int32_t)t.chunk_rep.size();
    ri.nch = (int32_t)((ri.n + (int64_t)L - 1) / L);
    t.chunk_rep.insert(t.chunk_rep.end(), ri.nch, r);
    ri.z0 = (int32_t)t.zchunk_rep.size();
    ri.nz = (int32_t)((ri.n + (int64_t)t.L0 - 1) / t.L0);
    t.zchunk_rep.insert(t.zchunk_rep.end(), ri.nz, r);
    // k = 0 carry groups: about sqrt(nz) groups of about sqrt(nz) chunks
    ri.zg0 = (int32_t)t.zgroup_rep.size();
    ri.nzg = 0;
    if (ri.nz > 0) {
      const int G =
          ri.nz < kFlatChunks ? 1 : std::max(1, (int)std::lround(std::sqrt((double)ri.nz)));
      const int g = (ri.nz + G - 1) / G;
      for (int a = 0; a < ri.nz; a += g) {
        t.zgstart.push_back(ri.z0 + a);
        t.zgroup_rep.push_back(r);
        ++ri.nzg;
      }
    }
    // groups: about sqrt(nch) groups of about sqrt(nch) chunks (serial depth
    // of the three carry phases about 3 sqrt(nch))
    ri.g0 = (int32_t)t.group_rep.size();
    ri.ng = 0;
    if (ri.nch > 0) {
      const int G = ri.nch < kFlatChunks
                        ? 1
                        : std::max(2, (int)std::lround(std::sqrt((double)ri.nch)));
      const int g = (ri.nch + G - 1) / G;
      for (int a = 0; a < ri.nch; a += g) {
        t.gstart.push_back(ri.c0 + a);
        t.group_rep.push_back(r);
        ++ri.ng;
      }
    }
  }
  t.kflat = 1;
  t.zflat = 1;
  for (int r = 0; r < R; ++r) {
    if (t.info[r].ng > 1) t.kflat = 0;
    if (t.info[r].nzg > 1) t.zflat = 0;
  }
  t.nchunks = (int)t.chunk_rep.size();
  t.nz = (int)t.zchunk_rep.size();
  t.ngroups = (int)t.group_rep.size();
  t.gstart.push_back(t.nchunks);
  t.nzgroups = (int)t.zgroup_rep.size();
  t.zgstart.push_back(t.nz);
  // device layout
  const size_t tsz = dp ? sizeof(double) : sizeof(float);
  size_t o = 0;
  auto take = [&o](size_t b) { size_t r = o; o += a256(b); return r; };
  t.o_info = take(sizeof(RepInfo) * R);
  t.o_crep = take(sizeof(int32_t) * t.nchunks);
  t.o_zrep = take(sizeof(int32_t) * t.nz);
  t.o_gstart = take(sizeof(int32_t) * t.gstart.size());
  t.o_grep = take(sizeof(int32_t) * std::max(t.ngroups, 1));
  t.o_zgstart = take(sizeof(int32_t) * t.zgstart.size());
  t.o_zgrep = take(sizeof(int32_t) * std::max(t.nzgroups, 1));
  t.o_list = take(sizeof(int32_t) * std::max<size_t>(t.list.size(), 2));
  t.o_cdf = take(sizeof(double) * std::max<size_t>(t.cdf.size(), 1));
  t.o_trig = take(sizeof(float) * 2 * 256);
  t.o_vdiag = take(sizeof(double) * 3 * (size_t)R);
  t.o_sampled = take(sizeof(int32_t) * 2 * (size_t)R * t.Kpad);
  t.o_modes = take(mode_bytes((size_t)R * t.Kpad, c->npc, tsz));
  t.bytes = o;
  t.valid = true;
  return QSLAB_OK;
}

// Upload the host tables into a device buffer of at least t.bytes, ordered
// on the call's stream (after the work of earlier calls on it that may still
// read the buffer, before this call's kernels; the pageable source is staged
// by the runtime before cudaMemcpyAsync returns).
int upload_tables(const Tables& t, void* dst, cudaStream_t st) {
  std::vector<char> stage(t.o_sampled, 0);
  auto put = [&stage](size_t o, const void* src, size_t b) {
    if (b) std::memcpy(stage.data() + o, src, b);
  };
  put(t.o_info, t.info.data(), sizeof(RepInfo) * t.R);
  put(t.o_crep, t.chunk_rep.data(), sizeof(int32_t) * t.chunk_rep.size());
  put(t.o_zrep, t.zchunk_rep.data(), sizeof(int32_t) * t.zchunk_rep.size());
  put(t.o_gstart, t.gstart.data(), sizeof(int32_t) * t.gstart.size());
  put(t.o_grep, t.group_rep.data(), sizeof(int32_t) * t.group_rep.size());
  put(t.o_zgstart, t.zgstart.data(), sizeof(int32_t) * t.zgstart.size());
  put(t.o_zgrep, t.zgroup_rep.data(), sizeof(int32_t) * t.zgroup_rep.size());
  put(t.o_list, t.list.data(), sizeof(int32_t) * t.list.size());
  put(t.o_cdf, t.cdf.data(), sizeof(double) * t.cdf.size());
  // (cos, sin) of the turns j/256 for the FP32 phases, rounded from FP64
  float trig[512];
  for (int j = 0; j < 256; ++j) {
    trig[2 * j] = (float)std::cos(2.0 * kPi * j / 256.0);
    trig[2 * j + 1] = (float)std::sin(2.0 * kPi * j / 256.0);
  }
  put(t.o_trig, trig, sizeof(trig));
  put(t.o_vdiag, t.vdiag.data(), sizeof(double) * t.vdiag.size());
  QS_CUDA(cudaMemcpyAsync(dst, stage.data(), stage.size(), cudaMemcpyHostToDevice, st));
  return QSLAB_OK;
}

// Make c->tab describe (R, off, box), rebuilding and uploading if needed.
// New tables end what an energy-only call left for its adjoint.
int select_tables(qslab_ctx* c, int R, const int64_t* off, const double* box, cudaStream_t st) {
  int rc = ensure_config(c);
  if (rc) return rc;
  if (same_key(c->tab, c, R, off, box)) return QSLAB_OK;
  Tables t;
  rc = build_tables(c, R, off, box, t, &c->tab);
  if (rc) return rc;
  bool released = false;
  rc = grow_buffer(&c->d_tab, &c->tab_bytes, t.bytes, &released);
  if (released) {
    c->tab.valid = false;
    c->primed = false;
  }
  if (rc) return rc;
  c->tab.valid = false;
  c->primed = false;
  rc = upload_tables(t, c->d_tab, st);
  if (rc) return rc;
  c->tab = std::move(t);
  c->coef_ready = false;
  c->have_sample = false;
  return QSLAB_OK;
}

Reps reps_view(const qslab_ctx* c) {
  const Tables& t = c->tab;
  const char* b = static_cast<const char*>(c->d_tab);
  Reps rp;
  rp.R = t.R;
  rp.L = t.L;
  rp.L0 = t.L0;
  rp.nchunks = t.nchunks;
  rp.nzchunks = t.nz;
  rp.ngroups = t.ngroups;
  rp.Kpad = t.Kpad;
  rp.N = t.N;
  rp.info = reinterpret_cast<const RepInfo*>(b + t.o_info);
  rp.chunk_rep = reinterpret_cast<const int32_t*>(b + t.o_crep);
  rp.zchunk_rep = reinterpret_cast<const int32_t*>(b + t.o_zrep);
  rp.gstart = reinterpret_cast<const int32_t*>(b + t.o_gstart);
  rp.group_rep = reinterpret_cast<const int32_t*>(b + t.o_grep);
  rp.zgstart = reinterpret_cast<const int32_t*>(b + t.o_zgstart);
  rp.zgroup_rep = reinterpret_cast<const int32_t*>(b + t.o_zgrep);
  rp.nzgroups = t.nzgroups;
  rp.kflat = t.kflat;
  rp.zflat = t.zflat;
  rp.status = c->d_status;
  return rp;
}

struct Plan {
  ScanPlan sp;
  size_t off_sort, off_rid, off_sums, off_zs, off_dz, off_qs, off_xh, off_yh, off_perm,
      off_agg, off_carry, off_dec, off_part, off_k0, off_phi0, off_fz0, off_echunk, off_in_pos,
      off_in_q, off_out_phi, off_out_f, off_vir, total;
};

Plan make_plan(const qslab_ctx* c, bool host_io, bool virial = false) {
  Plan P{};
  const Tables& t = c->tab;
  const bool dp = c->prec == QSLAB_FP64;
  const size_t tsz = dp ? 8 : 4;
  const int64_t N = t.N;
  ScanPlan& s = P.sp;
  s.KR = t.KR;
  s.nkr = t.nkr;
  s.np = c->npc;
  s.nstates = 1 + 2 * c->npc;
  s.rem = 0;
  if (!dp)
    for (const RepInfo& ri : t.info)
      if ((ri.K % kWarp >= 1 && ri.K % kWarp <= 8) || t.Kpad - ri.K >= kWarp) s.rem = 1;
  const Reps rp = reps_view(c);
  size_t o = 0;
  auto take = [&o](size_t b) { size_t r = o; o += a256(b); return r; };
  P.off_sort = take(sort_workspace_bytes(N, dp ? 8 : 4));
  P.off_rid = take(t.R > 1 ? 4 * (size_t)N : 0);
  P.off_sums = take(16 * (size_t)t.nchunks);
  P.off_zs = take(tsz * N);
  P.off_dz = take(tsz * N);
  P.off_qs = take(tsz * N);
  P.off_xh = take(tsz * N);
  P.off_yh = take(tsz * N);
  P.off_perm = take(4 * (size_t)N);
  const size_t aggn = (size_t)2 * t.nchunks * s.nstates * t.Kpad;
  P.off_agg = take(2 * tsz * aggn);
  P.off_carry = take(2 * tsz * aggn);
  P.off_dec = take(kspace_decay_bytes(s, rp, dp ? 1 : 0));
  P.off_part = take(tsz * 4 * (size_t)s.nkr * N);
  P.off_k0 = take(8 * kzero_work_doubles(t.nz, t.nzgroups, t.R, c->pairs.np));
  P.off_phi0 = take(8 * (size_t)N);
  P.off_fz0 = take(8 * (size_t)N);
  P.off_echunk = take(8 * (size_t)t.nchunks);
  if (host_io) {
    P.off_in_pos = take(3 * tsz * N);
    P.off_in_q = take(tsz * N);
    P.off_out_phi = take(tsz * N);
    P.off_out_f = take(3 * tsz * N);
  }
  if (virial) P.off_vir = take(virial_workspace_bytes(s, rp));
  P.total = o;
  return P;
}

int ensure_ws(qslab_ctx* c, size_t bytes) {
  bool released = false;
  const int rc = grow_buffer(&c->d_ws, &c->ws_bytes, bytes, &released);
  if (released) c->primed = false;   // the adjoint's stored state is gone
  return rc;
}

template <typename T>
// what = 0: energy, potentials, forces (and the virial if requested);
// what = 1: the energy only, from forward sums, leaving the sorted data,
// carries, mode tables and the k = 0 term in the workspace for the adjoint
// (run_adjoint).
int run(qslab_ctx* c, const Plan& P, const T* pos, const T* q, double* energies, T* phi,
        T* force, cudaStream_t st, double* virial = nullptr, int what = 0) {
  using PH = typename PhaseT<T>::type;
  const Tables& tb = c->tab;
  const int64_t N = tb.N;
  const int R = tb.R;
  const Reps rp = reps_view(c);
  char* ws = static_cast<char*>(c->d_ws);
  char* tab = static_cast<char*>(c->d_tab);
  SortWork sw;
  sort_bind_workspace(sw, ws + P.off_sort, N, sizeof(T));
  sw.status = c->d_status;
  int32_t* rid = reinterpret_cast<int32_t*>(ws + P.off_rid);
  double* sums = reinterpret_cast<double*>(ws + P.off_sums);
  T* zs = reinterpret_cast<T*>(ws + P.off_zs);
  T* dz = reinterpret_cast<T*>(ws + P.off_dz);
  T* qs = reinterpret_cast<T*>(ws + P.off_qs);
  PH* xh = reinterpret_cast<PH*>(ws + P.off_xh);
  PH* yh = reinterpret_cast<PH*>(ws + P.off_yh);
  int32_t* perm = reinterpret_cast<int32_t*>(ws + P.off_perm);
  Cplx<T>* agg = reinterpret_cast<Cplx<T>*>(ws + P.off_agg);
  Cplx<T>* carry = reinterpret_cast<Cplx<T>*>(ws + P.off_carry);
  void* dec = ws + P.off_dec;
  T* part = reinterpret_cast<T*>(ws + P.off_part);
  double* k0w = reinterpret_cast<double*>(ws + P.off_k0);
  double* phi0 = reinterpret_cast<double*>(ws + P.off_phi0);
  double* fz0 = reinterpret_cast<double*>(ws + P.off_fz0);
  double* echunk = reinterpret_cast<double*>(ws + P.off_echunk);
  ModeTab<T> modes = mode_views<T>(tab + tb.o_modes, (size_t)R * tb.Kpad, c->npc);
  const bool rbe = c->mode == 2;

  cudaEvent_t* ev = c->timing ? c->ev : nullptr;
  int nl = 0;
  c->primed = false;
  if (ev) cudaEventRecord(ev[0], st);
  launch_prepare<T>(rp, pos, q, sw.keys[0], sw.vals[0], R > 1 ? rid : nullptr, sums,
                    c->d_status, st);
  double tol = c->neutral_tol;
  if (tol < -1.0) tol = 64.0 * (sizeof(T) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-08);
  launch_check_neutral(rp, sums, tol, c->walls.on ? c->walls.sb0 : 0.0,
                       c->walls.on ? c->walls.st0 : 0.0, c->d_status, rbe ? c->d_ctr : nullptr, st);
  // mode tables: once per configuration for the full k-sum, every call for
  // RBE (after the counter's advance above), on the table stream
  const bool want_modes = rbe || !c->coef_ready;
  if (want_modes) {
    const double* cdf = reinterpret_cast<const double*>(tab + tb.o_cdf);
    int32_t* sampled = rbe ? reinterpret_cast<int32_t*>(tab + tb.o_sampled) : nullptr;
    const bool mh = rbe && c->sampler == QSLAB_SAMPLER_METROPOLIS;
    QS_CUDA(cudaEventRecord(c->tab_fork, st));
    QS_CUDA(cudaStreamWaitEvent(c->tab_side, c->tab_fork, 0));
    if (mh) {
      launch_mh_chain(rp, c->P, c->mh_thin, c->seed, c->d_ctr, cdf, c->alpha, sampled,
                      c->tab_side);
      ++nl;
    }
    launch_mode_coef<T>(rp, c->npc, reinterpret_cast<const int32_t*>(tab + tb.o_list),
                        rbe ? (mh ? 2 : 1) : 0, c->seed, c->d_ctr, cdf, c->pairs, c->alpha, modes,
                        sampled, c->tab_side);
    ++nl;
    QS_CUDA(cudaEventRecord(c->tab_join, c->tab_side));
    if (rbe) c->have_sample = true;
    else c->coef_ready = true;
  }
  int r = radix_sort(sw, N, (int)sizeof(T), (int)sizeof(T), 0, st, true);
  nl += 2 + sort_launches(N, (int)sizeof(T), true);   // prepare, check, the sort
  if (R > 1) {
    // stable second sort on the replica index: replicas contiguous, z-ordered within
    launch_rep_keys(N, sw.vals[r], rid, static_cast<uint32_t*>(sw.keys[r]), st);
    const int passes = R <= 256 ? 1 : (R <= 65536 ? 2 : 3);
    r = radix_sort(sw, N, 4, passes, r, st, true);
    nl += 1 + sort_launches(N, passes, true);
  }
  launch_gather<T>(rp, pos, q, sw.vals[r], R == 1 ? sw.keys[r] : nullptr, zs, dz, qs, xh, yh,
                   perm, st);
  ++nl;
  if (ev) cudaEventRecord(ev[1], st);
  // k = 0 term on the side stream, concurrent with the k-space kernels
  QS_CUDA(cudaEventRecord(c->fork, st));
  QS_CUDA(cudaStreamWaitEvent(c->side, c->fork, 0));
  launch_kzero<T>(rp, c->pairs, c->alpha, zs, dz, qs, k0w, phi0, fz0, c->side);
  nl += rp.zflat ? 4 : 6;
  if (ev) cudaEventRecord(ev[8], c->side);
  QS_CUDA(cudaEventRecord(c->join, c->side));
  if (want_modes) QS_CUDA(cudaStreamWaitEvent(st, c->tab_join, 0));
  if (ev) cudaEventRecord(ev[2], st);
  const float2* trig = sizeof(T) == 4 ? reinterpret_cast<const float2*>(tab + tb.o_trig) : nullptr;
  if (what == 1) {
    // energy only: pass A and the carries, then the forward pair sums per
    // mode (no bidirectional gather); the k = 0 term, the j = i constants and
    // the walls come from the combine kernel with no k-space planes
    launch_kspace<T>(P.sp, rp, modes, c->pairs, zs, dz, qs, xh, yh, trig, agg, carry, dec, part,
                     st, ev ? ev + 3 : nullptr, 1);
    VirArgs<T> va{P.sp, rp, modes, c->pairs, c->alpha, rbe ? 1 : 0, zs, dz, qs, xh, yh, trig,
                  carry, agg, pos, q, nullptr, energies, nullptr, c->walls, nullptr};
    // pass A, decays, 1 or 3 carry kernels
    nl += (rp.kflat ? 3 : 5) + launch_energy_pass<T>(va, ws + P.off_vir, st);
    if (ev) cudaEventRecord(ev[5], st);
    QS_CUDA(cudaStreamWaitEvent(st, c->join, 0));
    if (ev) cudaEventRecord(ev[6], st);
    launch_combine<T>(rp, 0, part, phi0, fz0, qs, zs, xh, yh, c->walls, perm, echunk, nullptr,
                      nullptr, energies, st);
    nl += 2 + launch_energy_add(P.sp, rp, ws + P.off_vir, energies, st);
    if (ev) cudaEventRecord(ev[7], st);
    c->launches = nl;
    c->last_R = R;
    QS_CUDA(cudaGetLastError());
    c->last_stream = st;
    c->primed = true;
    return QSLAB_OK;
  }
  launch_kspace<T>(P.sp, rp, modes, c->pairs, zs, dz, qs, xh, yh, trig, agg, carry, dec, part, st,
                   ev ? ev + 3 : nullptr);
  nl += rp.kflat ? 4 : 6;   // pass A, decays, 1 or 3 carry kernels, pass B
  QS_CUDA(cudaStreamWaitEvent(st, c->join, 0));
  if (ev) cudaEventRecord(ev[6], st);
  launch_combine<T>(rp, P.sp.nkr, part, phi0, fz0, qs, zs, xh, yh, c->walls, perm, echunk, phi,
                    force, energies, st);
  nl += energies ? 2 : 1;
  if (virial) {
    // the virial of the same energy, from this call's sorted data, mode
    // tables, forward carries, forces and energies
    VirArgs<T> va{P.sp, rp, modes, c->pairs, c->alpha, rbe ? 1 : 0, zs, dz, qs, xh, yh,
                  sizeof(T) == 4 ? reinterpret_cast<const float2*>(tab + tb.o_trig) : nullptr,
                  carry, agg, pos, q, force, energies,
                  reinterpret_cast<const double*>(tab + tb.o_vdiag), c->walls, virial};
    nl += launch_virial<T>(va, ws + P.off_vir, st);
  }
  if (ev) cudaEventRecord(ev[7], st);
  c->launches = nl;
  c->last_R = R;
  QS_CUDA(cudaGetLastError());
  c->last_stream = st;
  return QSLAB_OK;
}

// The adjoint of an energy-only call (what = 1 above): pass B over the
// sorted order, carries and mode tables that call left in the workspace
// (phases recomputed), then the combine kernel with the stored k = 0 term:
// phi = dE/dq and F = -dE/dr in the caller's order.
template <typename T>
int run_adjoint(qslab_ctx* c, const Plan& P, T* phi, T* force, cudaStream_t st) {
  using PH = typename PhaseT<T>::type;
  const Tables& tb = c->tab;
  const int R = tb.R;
  const Reps rp = reps_view(c);
  char* ws = static_cast<char*>(c->d_ws);
  char* tab = static_cast<char*>(c->d_tab);
  T* zs = reinterpret_cast<T*>(ws + P.off_zs);
  T* dz = reinterpret_cast<T*>(ws + P.off_dz);
  T* qs = reinterpret_cast<T*>(ws + P.off_qs);
  PH* xh = reinterpret_cast<PH*>(ws + P.off_xh);
  PH* yh = reinterpret_cast<PH*>(ws + P.off_yh);
  int32_t* perm = reinterpret_cast<int32_t*>(ws + P.off_perm);
  Cplx<T>* agg = reinterpret_cast<Cplx<T>*>(ws + P.off_agg);
  Cplx<T>* carry = reinterpret_cast<Cplx<T>*>(ws + P.off_carry);
  void* dec = ws + P.off_dec;
  T* part = reinterpret_cast<T*>(ws + P.off_part);
  double* phi0 = reinterpret_cast<double*>(ws + P.off_phi0);
  double* fz0 = reinterpret_cast<double*>(ws + P.off_fz0);
  double* echunk = reinterpret_cast<double*>(ws + P.off_echunk);
  ModeTab<T> modes = mode_views<T>(tab + tb.o_modes, (size_t)R * tb.Kpad, c->npc);
  const float2* trig = sizeof(T) == 4 ? reinterpret_cast<const float2*>(tab + tb.o_trig) : nullptr;
  launch_kspace<T>(P.sp, rp, modes, c->pairs, zs, dz, qs, xh, yh, trig, agg, carry, dec, part, st,
                   nullptr, 2);
  launch_combine<T>(rp, P.sp.nkr, part, phi0, fz0, qs, zs, xh, yh, c->walls, perm, echunk, phi,
                    force, nullptr, st);
  c->launches = 2;
  QS_CUDA(cudaGetLastError());
  c->last_stream = st;
  return QSLAB_OK;
}

int status_code(unsigned f) {
  if (f & kStNonfinite) return QSLAB_ERR_NONFINITE;
  if (f & kStZRange) return QSLAB_ERR_Z_OUT_OF_RANGE;
  if (f & kStNonneutral) return QSLAB_ERR_NONNEUTRAL;
  if (f & kStTimeout) return QSLAB_ERR_TIMEOUT;
  if (f & kStDebug) return QSLAB_ERR_INTERNAL;
  return QSLAB_OK;
}

// Tables and workspace for one call; on success P describes the workspace.
int setup_call(qslab_ctx* c, int R, const int64_t* off, const double* box, bool host_io,
               Plan& P, cudaStream_t st, bool virial = false) {
  QS_CUDA(cudaSetDevice(c->device));
  int rc = select_tables(c, R, off, box, st);
  if (rc) return rc;
  P = make_plan(c, host_io, virial);
  return ensure_ws(c, P.total);
}

int dispatch(qslab_ctx* c, const Plan& P, const void* pos, const void* q, double* energies,
             void* phi, void* force, cudaStream_t st, double* virial = nullptr, int what = 0) {
  if (c->prec == QSLAB_FP64)
    return run<double>(c, P, static_cast<const double*>(pos), static_cast<const double*>(q),
                       energies, static_cast<double*>(phi), static_cast<double*>(force), st,
                       virial, what);
  return run<float>(c, P, static_cast<const float*>(pos), static_cast<const float*>(q), energies,
                    static_cast<float*>(phi), static_cast<float*>(force), st, virial, what);
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
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cuda_device) == cudaSuccess &&
      sms > 0)
    c->sm_count = sms;
  void* small = nullptr;
  cudaError_t e = lib_malloc(&small, 256);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e);
  }
  c->d_status = static_cast<unsigned*>(small);
  c->d_energy = reinterpret_cast<double*>(static_cast<char*>(small) + 128);
  c->d_ctr = reinterpret_cast<uint64_t*>(static_cast<char*>(small) + 192);
  c->d_md_ctr = reinterpret_cast<uint64_t*>(static_cast<char*>(small) + 224);
  if (cudaMemset(small, 0, 256) != cudaSuccess) {
    cudaFree(small);
    delete c;
    return QSLAB_ERR_CUDA;
  }
  for (auto& ev : c->ev) cudaEventCreate(&ev);
  if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->rs_side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->rs_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->rs_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->tab_side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->tab_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->tab_join, cudaEventDisableTiming) != cudaSuccess) {
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
  if (c->d_rs_ws) cudaFree(c->d_rs_ws);
  if (c->d_md) cudaFree(c->d_md);
  if (c->d_tab) cudaFree(c->d_tab);
  if (c->d_status) cudaFree(c->d_status);
  for (auto& ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->join) cudaEventDestroy(c->join);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->rs_fork) cudaEventDestroy(c->rs_fork);
  if (c->rs_join) cudaEventDestroy(c->rs_join);
  if (c->rs_side) cudaStreamDestroy(c->rs_side);
  if (c->tab_fork) cudaEventDestroy(c->tab_fork);
  if (c->tab_join) cudaEventDestroy(c->tab_join);
  if (c->tab_side) cudaStreamDestroy(c->tab_side);
  delete c;
}

int qslab_set_box(qslab_ctx* c, double Lx, double Ly, double Lz) {
  if (!c || !finite_pos(Lx) || !finite_pos(Ly) || !finite_pos(Lz)) return QSLAB_ERR_INVALID_ARG;
  c->Lx = Lx; c->Ly = Ly; c->Lz = Lz;
  c->has_box = true;
  return QSLAB_OK;
}

int qslab_set_alpha(qslab_ctx* c, double alpha) {
  if (!c || !finite_pos(alpha)) return QSLAB_ERR_INVALID_ARG;
  c->alpha = alpha;
  c->has_alpha = true;
  c->cfg_dirty = true;
  c->primed = false;
  return QSLAB_OK;
}

int qslab_set_kcut(qslab_ctx* c, double kc) {
  if (!c || !finite_pos(kc)) return QSLAB_ERR_INVALID_ARG;
  c->kc = kc;
  c->mode = 1;
  c->cfg_dirty = true;
  c->primed = false;
  return QSLAB_OK;
}

int qslab_set_rbe(qslab_ctx* c, int P, uint64_t seed) {
  if (!c || P < 1 || P > 65536) return QSLAB_ERR_INVALID_ARG;
  QS_CUDA(cudaSetDevice(c->device));
  const uint64_t zero[2] = {0, 0};
  QS_CUDA(cudaMemcpy(c->d_ctr, zero, sizeof(zero), cudaMemcpyHostToDevice));
  c->P = P;
  c->seed = seed;
  c->mode = 2;
  c->cfg_dirty = true;
  c->primed = false;
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
  c->cfg_dirty = true;
  c->primed = false;
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
  c->tune_KR = modes_per_cta;
  c->primed = false;
  return QSLAB_OK;
}

int qslab_compute(qslab_ctx* c, int64_t N, const void* pos, const void* q,
                  double* energy, void* phi, void* force, void* stream) {
  if (!c || !pos || !q || N < 1 || N > 2147483647LL) return QSLAB_ERR_INVALID_ARG;
  if (!c->has_box) return QSLAB_ERR_NOT_CONFIGURED;
  const int64_t off[2] = {0, N};
  const double box[3] = {c->Lx, c->Ly, c->Lz};
  Plan P;
  const int rc = setup_call(c, 1, off, box, false, P, static_cast<cudaStream_t>(stream));
  if (rc) return rc;
  return dispatch(c, P, pos, q, energy, phi, force, static_cast<cudaStream_t>(stream));
}

int qslab_compute_batched(qslab_ctx* c, int R, const int64_t* offsets, const double* boxes,
                          const void* pos, const void* q, double* energies, void* phi,
                          void* force, void* stream) {
  if (!c || !pos || !q || !offsets || !boxes || R < 1 || R > kMaxReplicas)
    return QSLAB_ERR_INVALID_ARG;
  Plan P;
  const int rc = setup_call(c, R, offsets, boxes, false, P, static_cast<cudaStream_t>(stream));
  if (rc) return rc;
  return dispatch(c, P, pos, q, energies, phi, force, static_cast<cudaStream_t>(stream));
}

int qslab_compute_virial(qslab_ctx* c, int64_t N, const void* pos, const void* q,
                         double* energy, void* phi, void* force, double* virial, void* stream) {
  if (!c || !pos || !q || !energy || !force || !virial || N < 1 || N > 2147483647LL)
    return QSLAB_ERR_INVALID_ARG;
  if (!c->has_box) return QSLAB_ERR_NOT_CONFIGURED;
  const int64_t off[2] = {0, N};
  const double box[3] = {c->Lx, c->Ly, c->Lz};
  Plan P;
  const int rc = setup_call(c, 1, off, box, false, P, static_cast<cudaStream_t>(stream), true);
  if (rc) return rc;
  return dispatch(c, P, pos, q, energy, phi, force, static_cast<cudaStream_t>(stream), virial);
}

int qslab_compute_batched_virial(qslab_ctx* c, int R, const int64_t* offsets,
                                 const double* boxes, const void* pos, const void* q,
                                 double* energies, void* phi, void* force, double* virial,
                                 void* stream) {
  if (!c || !pos || !q || !offsets || !boxes || !energies || !force || !virial || R < 1 ||
      R > kMaxReplicas)
    return QSLAB_ERR_INVALID_ARG;
  Plan P;
  const int rc = setup_call(c, R, offsets, boxes, false, P, static_cast<cudaStream_t>(stream), true);
  if (rc) return rc;
  return dispatch(c, P, pos, q, energies, phi, force, static_cast<cudaStream_t>(stream), virial);
}

int qslab_compute_energy(qslab_ctx* c, int64_t N, const void* pos, const void* q,
                         double* energy, void* stream) {
  if (!c || !pos || !q || !energy || N < 1 || N > 2147483647LL) return QSLAB_ERR_INVALID_ARG;
  if (!c->has_box) return QSLAB_ERR_NOT_CONFIGURED;
  const int64_t off[2] = {0, N};
  const double box[3] = {c->Lx, c->Ly, c->Lz};
  Plan P;
  c->primed = false;
  const int rc = setup_call(c, 1, off, box, false, P, static_cast<cudaStream_t>(stream), true);
  if (rc) return rc;
  return dispatch(c, P, pos, q, energy, nullptr, nullptr, static_cast<cudaStream_t>(stream),
                  nullptr, 1);
}

int qslab_compute_batched_energy(qslab_ctx* c, int R, const int64_t* offsets,
                                 const double* boxes, const void* pos, const void* q,
                                 double* energies, void* stream) {
  if (!c || !pos || !q || !offsets || !boxes || !energies || R < 1 || R > kMaxReplicas)
    return QSLAB_ERR_INVALID_ARG;
  Plan P;
  c->primed = false;
  const int rc = setup_call(c, R, offsets, boxes, false, P, static_cast<cudaStream_t>(stream), true);
  if (rc) return rc;
  return dispatch(c, P, pos, q, energies, nullptr, nullptr, static_cast<cudaStream_t>(stream),
                  nullptr, 1);
}

int qslab_compute_adjoint(qslab_ctx* c, void* phi, void* force, void* stream) {
  if (!c || (!phi && !force)) return QSLAB_ERR_INVALID_ARG;
  if (!c->primed || c->cfg_dirty || !c->tab.valid || c->tab.cfg_version != c->cfg_version)
    return QSLAB_ERR_NOT_CONFIGURED;
  QS_CUDA(cudaSetDevice(c->device));
  const Plan P = make_plan(c, false, true);
  if (P.total > c->ws_bytes) return QSLAB_ERR_NOT_CONFIGURED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (c->prec == QSLAB_FP64)
    return run_adjoint<double>(c, P, static_cast<double*>(phi), static_cast<double*>(force), st);
  return run_adjoint<float>(c, P, static_cast<float*>(phi), static_cast<float*>(force), st);
}

int qslab_compute_host(qslab_ctx* c, int64_t N, const void* pos_host, const void* q_host,
                       double* energy_host, void* phi_host, void* force_host, void* stream) {
  if (!c || !pos_host || !q_host || N < 1 || N > 2147483647LL) return QSLAB_ERR_INVALID_ARG;
  if (!c->has_box) return QSLAB_ERR_NOT_CONFIGURED;
  const int64_t off[2] = {0, N};
  const double box[3] = {c->Lx, c->Ly, c->Lz};
  Plan P;
  int rc = setup_call(c, 1, off, box, true, P, static_cast<cudaStream_t>(stream));
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
  rc = dispatch(c, P, dpos, dq, c->d_energy, dphi, df, st);
  if (rc) return rc;
  if (energy_host)
    QS_CUDA(cudaMemcpyAsync(energy_host, c->d_energy, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (phi_host) QS_CUDA(cudaMemcpyAsync(phi_host, dphi, tsz * N, cudaMemcpyDeviceToHost, st));
  if (force_host) QS_CUDA(cudaMemcpyAsync(force_host, df, 3 * tsz * N, cudaMemcpyDeviceToHost, st));
  return qslab_last_status(c);
}

int qslab_set_walls(qslab_ctx* c, double sigma_bot, double sigma_top, int nw,
                    const int32_t* mxy, const double* bot, const double* top) {
  if (!c || !std::isfinite(sigma_bot) || !std::isfinite(sigma_top) || nw < 0 ||
      nw > kMaxWallModes || (nw > 0 && (!mxy || !bot || !top)))
    return QSLAB_ERR_INVALID_ARG;
  WallTab w{};
  w.on = 1;
  w.nw = nw;
  w.sb0 = sigma_bot;
  w.st0 = sigma_top;
  for (int i = 0; i < nw; ++i) {
    const int32_t mx = mxy[2 * i], my = mxy[2 * i + 1];
    if (mx == 0 && my == 0) return QSLAB_ERR_INVALID_ARG;
    if (mx < -(1 << 20) || mx > (1 << 20) || my < -(1 << 20) || my > (1 << 20))
      return QSLAB_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j) {   // each pair (m, -m) at most once
      const int32_t ax = mxy[2 * j], ay = mxy[2 * j + 1];
      if ((ax == mx && ay == my) || (ax == -mx && ay == -my)) return QSLAB_ERR_INVALID_ARG;
    }
    for (int k = 0; k < 2; ++k)
      if (!std::isfinite(bot[2 * i + k]) || !std::isfinite(top[2 * i + k]))
        return QSLAB_ERR_INVALID_ARG;
    w.m[i][0] = mx;
    w.m[i][1] = my;
    w.c[i][0] = bot[2 * i];
    w.c[i][1] = bot[2 * i + 1];
    w.c[i][2] = top[2 * i];
    w.c[i][3] = top[2 * i + 1];
  }
  c->walls = w;
  c->primed = false;
  return QSLAB_OK;
}

int qslab_set_rbe_sampler(qslab_ctx* c, int kind, int thin) {
  if (!c || (kind != QSLAB_SAMPLER_IID && kind != QSLAB_SAMPLER_METROPOLIS) || thin < 1 ||
      thin > 4096)
    return QSLAB_ERR_INVALID_ARG;
  c->sampler = kind;
  c->mh_thin = kind == QSLAB_SAMPLER_METROPOLIS ? thin : 1;
  c->have_sample = false;
  c->primed = false;
  return QSLAB_OK;
}

int qslab_clear_walls(qslab_ctx* c) {
  if (!c) return QSLAB_ERR_INVALID_ARG;
  c->walls = WallTab{};
  c->primed = false;
  return QSLAB_OK;
}

int qslab_set_rcut(qslab_ctx* c, double rc) {
  if (!c || !finite_pos(rc)) return QSLAB_ERR_INVALID_ARG;
  c->rc = rc;
  return QSLAB_OK;
}

}  // extern "C"

namespace {

// The real-space sum (with the LJ pairs when lj_eps > 0) on stream st.
int realspace_call(qslab_ctx* c, int64_t N, const void* pos, const void* q, double* energy,
                   void* phi, void* force, cudaStream_t st, double lj_eps, double lj_sigma,
                   double* virial = nullptr) {
  if (!c || !pos || !q || N < 1 || N > 2147483647LL) return QSLAB_ERR_INVALID_ARG;
  if (!c->has_box || !c->has_alpha || c->rc <= 0) return QSLAB_ERR_NOT_CONFIGURED;
  RsGrid g;
  g.N = N;
  g.Lx = c->Lx; g.Ly = c->Ly; g.Lz = c->Lz;
  g.alpha = c->alpha;
  g.rc = c->rc;
  g.lj_eps = lj_eps;
  g.lj_sigma = lj_sigma;
  if (lj_eps > 0.0 && 1.122462048309373 * lj_sigma > c->rc) return QSLAB_ERR_INVALID_ARG;
  if (std::floor(c->Lx / c->rc) < 3 || std::floor(c->Ly / c->rc) < 3)
    return QSLAB_ERR_INVALID_ARG;   // needs rc <= min(Lx, Ly)/3
  // cells of edge >= rc/2: a 5 x 5 x 5 stencil covers rc with less volume
  // than 3 x 3 x 3 cells of edge rc (15.6 rc^3 instead of 27 rc^3)
  g.s = 2;
  const double fx = std::floor(c->Lx * g.s / c->rc), fy = std::floor(c->Ly * g.s / c->rc);
  const double fz = std::max(1.0, std::floor(c->Lz * g.s / c->rc));
  if (fx * fy * fz > 1.0e8) return QSLAB_ERR_INVALID_ARG;
  g.ncx = (int)fx; g.ncy = (int)fy; g.ncz = (int)fz;
  g.hz = c->Lz / g.ncz;
  QS_CUDA(cudaSetDevice(c->device));
  const size_t need = rs_workspace_bytes(g);
  const int grc = grow_buffer(&c->d_rs_ws, &c->rs_ws_bytes, need, nullptr);
  if (grc) return grc;
  if (c->prec == QSLAB_FP64)
    launch_realspace<double>(g, static_cast<const double*>(pos), static_cast<const double*>(q),
                             c->d_rs_ws, c->d_status, energy, static_cast<double*>(phi),
                             static_cast<double*>(force), st, virial);
  else
    launch_realspace<float>(g, static_cast<const float*>(pos), static_cast<const float*>(q),
                            c->d_rs_ws, c->d_status, energy, static_cast<float*>(phi),
                            static_cast<float*>(force), st, virial);
  QS_CUDA(cudaGetLastError());
  c->last_stream = st;
  return QSLAB_OK;
}

}  // namespace

extern "C" {

int qslab_compute_realspace(qslab_ctx* c, int64_t N, const void* pos, const void* q,
                            double* energy, void* phi, void* force, void* stream) {
  return realspace_call(c, N, pos, q, energy, phi, force, static_cast<cudaStream_t>(stream), 0.0,
                        0.0);
}

int qslab_compute_realspace_virial(qslab_ctx* c, int64_t N, const void* pos, const void* q,
                                   double* energy, void* phi, void* force, double* virial,
                                   void* stream) {
  if (!virial) return QSLAB_ERR_INVALID_ARG;
  return realspace_call(c, N, pos, q, energy, phi, force, static_cast<cudaStream_t>(stream), 0.0,
                        0.0, virial);
}

int qslab_md_configure(qslab_ctx* c, double dt, double mass, double gamma, double kT,
                       double lj_eps, double lj_sigma, double wall_eps, double wall_sigma,
                       uint64_t seed) {
  if (!c || !finite_pos(dt) || !finite_pos(mass) || !std::isfinite(gamma) || gamma < 0 ||
      !std::isfinite(kT) || kT < 0 || !std::isfinite(lj_eps) || lj_eps < 0 ||
      !std::isfinite(wall_eps) || wall_eps < 0 || (lj_eps > 0 && !finite_pos(lj_sigma)) ||
      (wall_eps > 0 && !finite_pos(wall_sigma)))
    return QSLAB_ERR_INVALID_ARG;
  MDDev m{};
  m.dt = dt;
  m.mass = mass;
  m.c1 = std::exp(-gamma * dt / mass);
  m.c2 = std::sqrt((1.0 - m.c1 * m.c1) * kT / mass);
  m.wall_eps = wall_eps;
  m.wall_sigma = wall_eps > 0 ? wall_sigma : 1.0;
  m.seed = seed;
  c->md = m;
  c->lj_eps = lj_eps;
  c->lj_sigma = lj_eps > 0 ? lj_sigma : 0.0;
  c->md_on = true;
  return QSLAB_OK;
}

int qslab_md_set_step(qslab_ctx* c, uint64_t step) {
  if (!c) return QSLAB_ERR_INVALID_ARG;
  QS_CUDA(cudaSetDevice(c->device));
  QS_CUDA(cudaStreamSynchronize(c->last_stream));
  QS_CUDA(cudaMemcpy(c->d_md_ctr, &step, sizeof(uint64_t), cudaMemcpyHostToDevice));
  return QSLAB_OK;
}

int qslab_md_get_step(qslab_ctx* c, uint64_t* step) {
  if (!c || !step) return QSLAB_ERR_INVALID_ARG;
  QS_CUDA(cudaSetDevice(c->device));
  QS_CUDA(cudaStreamSynchronize(c->last_stream));
  QS_CUDA(cudaMemcpy(step, c->d_md_ctr, sizeof(uint64_t), cudaMemcpyDeviceToHost));
  return QSLAB_OK;
}

}  // extern "C"

namespace {

struct MDBufs {
  void* flr;
  void* frs;
  double* part;
  double* e_lr;
  double* e_rs;
};

int md_buffers(qslab_ctx* c, int64_t N, MDBufs& b) {
  const size_t tsz = c->prec == QSLAB_FP64 ? 8 : 4;
  const size_t f = a256(3 * tsz * (size_t)N);
  const size_t need = 2 * f + a256(16 * (size_t)md_blocks(N)) + 256;
  const int grc = grow_buffer(&c->d_md, &c->md_bytes, need, nullptr);
  if (grc) return grc;
  char* p = static_cast<char*>(c->d_md);
  b.flr = p;
  b.frs = p + f;
  b.part = reinterpret_cast<double*>(p + 2 * f);
  b.e_lr = reinterpret_cast<double*>(p + 2 * f + a256(16 * (size_t)md_blocks(N)));
  b.e_rs = b.e_lr + 1;
  return QSLAB_OK;
}

// Forces at pos (long range, real space with LJ pairs, LJ walls) into
// `force`; with kick, the closing half kick of a step. The real-space call
// runs on the context's second side stream, forked from `st` and joined
// back before the closing kernel, so that it overlaps the long-range call.
template <typename T>
int md_force_pass(qslab_ctx* c, const Plan& P, int64_t N, const MDBufs& b, const void* pos,
                  const void* q, void* vel, void* force, bool kick, cudaStream_t st) {
  QS_CUDA(cudaEventRecord(c->rs_fork, st));
  QS_CUDA(cudaStreamWaitEvent(c->rs_side, c->rs_fork, 0));
  int rc = realspace_call(c, N, pos, q, b.e_rs, nullptr, b.frs, c->rs_side, c->lj_eps,
                          c->lj_sigma);
  // joined on every path, so that a captured stream never ends with the fork open
  QS_CUDA(cudaEventRecord(c->rs_join, c->rs_side));
  if (!rc) rc = dispatch(c, P, pos, q, b.e_lr, nullptr, b.flr, st);
  QS_CUDA(cudaStreamWaitEvent(st, c->rs_join, 0));
  if (rc) return rc;
  launch_md_end<T>(N, c->md, static_cast<const T*>(pos), static_cast<T*>(vel),
                   static_cast<const T*>(b.flr), static_cast<const T*>(b.frs),
                   static_cast<T*>(force), b.part, c->d_md_ctr, kick, st);
  return QSLAB_OK;
}

template <typename T>
int md_run(qslab_ctx* c, int64_t N, void* pos, void* vel, const void* q, void* force, int nsteps,
           double* energies, cudaStream_t st) {
  const int64_t off[2] = {0, N};
  const double box[3] = {c->Lx, c->Ly, c->Lz};
  Plan P;
  int rc = setup_call(c, 1, off, box, false, P, st);
  if (rc) return rc;
  MDBufs b;
  rc = md_buffers(c, N, b);
  if (rc) return rc;
  c->md.Lx = c->Lx; c->md.Ly = c->Ly; c->md.Lz = c->Lz;
  if (nsteps == 0) {
    rc = md_force_pass<T>(c, P, N, b, pos, q, vel, force, false, st);
    if (rc) return rc;
  }
  for (int n = 0; n < nsteps; ++n) {
    launch_md_begin<T>(N, c->md, static_cast<T*>(pos), static_cast<T*>(vel),
                       static_cast<const T*>(force), c->d_md_ctr, st);
    rc = md_force_pass<T>(c, P, N, b, pos, q, vel, force, true, st);
    if (rc) return rc;
  }
  if (energies) launch_md_energies(N, b.part, b.e_lr, b.e_rs, energies, st);
  QS_CUDA(cudaGetLastError());
  c->last_stream = st;
  return QSLAB_OK;
}

}  // namespace

extern "C" {

int qslab_md_forces(qslab_ctx* c, int64_t N, const void* pos, const void* q, void* vel,
                    void* force, double* energies, void* stream) {
  if (!c || !pos || !q || !force || N < 1 || N > 2147483647LL) return QSLAB_ERR_INVALID_ARG;
  if (!c->md_on || !c->has_box || c->rc <= 0) return QSLAB_ERR_NOT_CONFIGURED;
  QS_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (c->prec == QSLAB_FP64)
    return md_run<double>(c, N, const_cast<void*>(pos), vel, q, force, 0, energies, st);
  return md_run<float>(c, N, const_cast<void*>(pos), vel, q, force, 0, energies, st);
}

int qslab_md_step(qslab_ctx* c, int64_t N, void* pos, void* vel, const void* q, void* force,
                  int nsteps, double* energies, void* stream) {
  if (!c || !pos || !vel || !q || !force || N < 1 || N > 2147483647LL || nsteps < 1)
    return QSLAB_ERR_INVALID_ARG;
  if (!c->md_on || !c->has_box || c->rc <= 0) return QSLAB_ERR_NOT_CONFIGURED;
  QS_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (c->prec == QSLAB_FP64)
    return md_run<double>(c, N, pos, vel, q, force, nsteps, energies, st);
  return md_run<float>(c, N, pos, vel, q, force, nsteps, energies, st);
}

int qslab_get_sampled_modes(qslab_ctx* c, int32_t* mxy, double* weight) {
  if (!c || !mxy) return QSLAB_ERR_INVALID_ARG;
  if (c->mode != 2 || !c->have_sample || !c->tab.valid) return QSLAB_ERR_NOT_CONFIGURED;
  QS_CUDA(cudaSetDevice(c->device));
  QS_CUDA(cudaStreamSynchronize(c->last_stream));
  const Tables& t = c->tab;
  QS_CUDA(cudaMemcpy(mxy, static_cast<char*>(c->d_tab) + t.o_sampled,
                     sizeof(int32_t) * 2 * (size_t)t.R * c->P, cudaMemcpyDeviceToHost));
  if (weight)
    for (int r = 0; r < t.R; ++r) weight[r] = t.info[r].H / c->P;
  return QSLAB_OK;
}

int qslab_get_rng_state(qslab_ctx* c, uint64_t* seed, uint64_t* counter) {
  if (!c || !seed || !counter) return QSLAB_ERR_INVALID_ARG;
  QS_CUDA(cudaSetDevice(c->device));
  QS_CUDA(cudaStreamSynchronize(c->last_stream));
  QS_CUDA(cudaMemcpy(counter, c->d_ctr, sizeof(uint64_t), cudaMemcpyDeviceToHost));
  *seed = c->seed;
  return QSLAB_OK;
}

int qslab_set_rng_state(qslab_ctx* c, uint64_t seed, uint64_t counter) {
  if (!c) return QSLAB_ERR_INVALID_ARG;
  QS_CUDA(cudaSetDevice(c->device));
  QS_CUDA(cudaStreamSynchronize(c->last_stream));
  QS_CUDA(cudaMemcpy(c->d_ctr, &counter, sizeof(uint64_t), cudaMemcpyHostToDevice));
  c->seed = seed;
  return QSLAB_OK;
}

int qslab_num_modes(qslab_ctx* c) {
  if (!c) return QSLAB_ERR_INVALID_ARG;
  if (!c->has_box || !c->has_alpha || !c->has_soe || c->mode == 0) return QSLAB_ERR_NOT_CONFIGURED;
  if (c->mode == 2) return c->P;
  return (int)(half_plane(c->Lx, c->Ly, c->kc).size() / 2);
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

int qslab_autotune(qslab_ctx* c, int R, const int64_t* offsets, const double* boxes,
                   const void* pos, const void* q, void* stream, int reps, int* chunk,
                   int* modes_per_cta) {
  if (!c || !offsets || !boxes || !pos || !q || R < 1 || R > kMaxReplicas || reps < 1 ||
      reps > 100)
    return QSLAB_ERR_INVALID_ARG;
  QS_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = ensure_config(c);
  if (rc) return rc;
  // the tuning calls must not consume random-batch samples: keep the counter
  uint64_t ctr_saved = 0;
  QS_CUDA(cudaStreamSynchronize(st));
  QS_CUDA(cudaMemcpy(&ctr_saved, c->d_ctr, sizeof(uint64_t), cudaMemcpyDeviceToHost));
  const int old_L = c->tune_L, old_KR = c->tune_KR;
  const bool old_timing = c->timing;
  c->timing = false;
  // candidates: chunk lengths (particles per CTA along the scan) and mode
  // ranges (threads per CTA); the largest K decides which mode widths apply
  std::vector<int> Ls = c->prec == QSLAB_FP64 ? std::vector<int>{64, 128, 256}
                                              : std::vector<int>{64, 128, 256, 512};
  int Kmax = c->mode == 2 ? c->P : 1;
  if (c->mode == 1) {
    std::map<std::pair<double, double>, int> seen;
    for (int r = 0; r < R; ++r) {
      const std::pair<double, double> key(boxes[3 * r], boxes[3 * r + 1]);
      if (seen.count(key)) continue;
      seen[key] = 1;
      Kmax = std::max(Kmax, (int)(half_plane(key.first, key.second, c->kc).size() / 2));
    }
  }
  const int k32 = ((Kmax + 31) / 32) * 32;
  std::vector<int> KRs;
  for (int kr : {64, 128, 192, 256})
    if (kr < k32) KRs.push_back(kr);
  KRs.push_back(0);   // automatic: one range when K <= 256
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  QS_CUDA(cudaEventCreate(&e0));
  QS_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bestL = 0, bestKR = 0;
  rc = QSLAB_OK;
  for (int L : Ls) {
    for (int kr : KRs) {
      c->tune_L = L;
      c->tune_KR = kr;
      Plan P;
      rc = setup_call(c, R, offsets, boxes, false, P, st);
      if (rc == QSLAB_ERR_ALLOC) { rc = QSLAB_OK; cudaGetLastError(); continue; }
      if (rc) break;
      rc = dispatch(c, P, pos, q, nullptr, nullptr, nullptr, st);   // warm-up
      if (rc) break;
      if (cudaEventRecord(e0, st) != cudaSuccess) { rc = QSLAB_ERR_CUDA; break; }
      for (int i = 0; i < reps && !rc; ++i) rc = dispatch(c, P, pos, q, nullptr, nullptr, nullptr, st);
      if (rc) break;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        rc = QSLAB_ERR_CUDA;
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; bestL = L; bestKR = kr; }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->timing = old_timing;
  c->have_sample = false;   // the tuning calls' samples are not the user's
  if (cudaMemcpy(c->d_ctr, &ctr_saved, sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess &&
      !rc)
    rc = QSLAB_ERR_CUDA;
  const int st_rc = qslab_last_status(c);
  if (!rc) rc = st_rc;
  if (rc || best >= 1e30f) {
    c->tune_L = old_L;
    c->tune_KR = old_KR;
    return rc ? rc : QSLAB_ERR_ALLOC;
  }
  c->tune_L = bestL;
  c->tune_KR = bestKR;
  if (chunk) *chunk = bestL;
  if (modes_per_cta) *modes_per_cta = bestKR;
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
    case QSLAB_ERR_INTERNAL: return "internal index check failed (debug build)";
    default: return "unknown error";
  }
}

long long qslab_debug_alloc_count(void) { return g_alloc_count.load(); }

int qslab_debug_stall_sort(int tile) {
  if (tile < 0) return QSLAB_ERR_INVALID_ARG;
  sort_debug_stall(tile);
  return QSLAB_OK;
}

int qslab_debug_fail_alloc(int n) {
  if (n < 0) return QSLAB_ERR_INVALID_ARG;
  g_fail_allocs.store(n);
  return QSLAB_OK;
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
constexpr size_t kStaticSmallBytes = 256;                  // status word
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
  if (!c->has_box) return QSLAB_ERR_NOT_CONFIGURED;
  int rc = ensure_config(c);
  if (rc) return rc;
  QS_CUDA(cudaSetDevice(c->device));
  void* base = nullptr;
  rc = static_scratch_address(c->device, &base);
  if (rc) return rc;
  char* sb = static_cast<char*>(base);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // A copy of the context whose device buffers all point into the static
  // array (the random-batch counter word excepted: it stays the context's);
  // its tables are rebuilt there on every call (the real context's own
  // buffers are neither used nor changed).
  qslab_ctx t = *c;
  t.timing = false;
  t.d_status = reinterpret_cast<unsigned*>(sb);
  t.d_tab = sb + kStaticSmallBytes;
  t.tab_bytes = kStaticCfgBytes - kStaticSmallBytes;
  t.d_ws = sb + kStaticCfgBytes;
  t.ws_bytes = kStaticScratchBytes - kStaticCfgBytes;
  // size checks before anything touches the device: the tables must fit the
  // table region and the workspace the rest of the array
  const int64_t off[2] = {0, N};
  const double box[3] = {c->Lx, c->Ly, c->Lz};
  if (c->mode == 2 && (axis_mmax(c->alpha, c->Lx) > 1000000 || axis_mmax(c->alpha, c->Ly) > 1000000))
    return QSLAB_ERR_TOO_LARGE;
  Tables tb;
  rc = build_tables(&t, 1, off, box, tb, c->tab.valid ? &c->tab : nullptr);
  if (rc) return rc;
  t.tab = std::move(tb);
  if (t.tab.bytes > t.tab_bytes) return QSLAB_ERR_TOO_LARGE;
  const Plan P = make_plan(&t, false);
  if (P.total > t.ws_bytes) return QSLAB_ERR_TOO_LARGE;
  rc = upload_tables(t.tab, t.d_tab, st);   // fits: no allocation
  if (rc) return rc;
  t.coef_ready = false;
  // the status word starts from zero on every call
  QS_CUDA(cudaMemsetAsync(t.d_status, 0, kStaticSmallBytes, st));
  rc = dispatch(&t, P, pos, q, energy, phi, force, st);
  if (rc) return rc;
  QS_CUDA(cudaStreamSynchronize(st));
  QS_CUDA(cudaGetLastError());
  unsigned f = 0;
  QS_CUDA(cudaMemcpy(&f, t.d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  return status_code(f);
}
