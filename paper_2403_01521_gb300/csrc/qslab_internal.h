// Internal declarations shared by the qslab CUDA translation units.
//
// A call processes R independent slabs ("replicas"; R = 1 for
// qslab_compute). Replica r owns the particles [off_r, off_r + n_r) of the
// caller's arrays; after sorting it owns the same index range, ordered by z.
//
// Data layout in HBM (all arrays indexed by the sorted particle index i):
//   zs[i], qs[i]
//   dz[i] = zs[i] - zs[i-1] within a replica, 0 at a replica's first
//           particle                                            type T
//   xh[i], yh[i]  fixed-point fractions x/Lx, y/Ly of the replica's box
//                 (2^32 or 2^64 units of a turn)                uint32 (FP32C)
//                                                               uint64 (FP64)
//   perm[i]       original index of sorted particle i           int32
// Each replica is cut into k-space chunks of L particles and k = 0 chunks of
// L0 particles (the last one of a replica may be shorter); no chunk spans
// two replicas. Chunks are numbered globally, replica by replica.
// Mode tables are structure-of-arrays with R * Kpad entries: replica r owns
// [r * Kpad, (r + 1) * Kpad), padded with zero-weight modes; see ModeTab.
// Chunk aggregates and carries: [dir][chunk][state][Kpad] complex, with
// state 0 = beta = k and states 1+2p, 2+2p = SOE pair p driven by the real
// inputs q cos(k.rho) and q sin(k.rho); the mode index is replica-local.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qslab {

constexpr int kMaxPairs = 16;     // SOE pair representatives (M <= 32)
constexpr int kWarp = 32;

template <typename T> struct Cplx { T re, im; };

// Per-precision fixed-point phase type.
template <typename T> struct PhaseT;
template <> struct PhaseT<float>  { using type = uint32_t; };
template <> struct PhaseT<double> { using type = uint64_t; };

// Structure-of-arrays mode table (device pointers), R * Kpad entries. For
// the SOE pair representative p of a mode:
//   cp   = m_p gam_k c_{k,p},          c_{k,p} = -2 k w_p / (a_p^2 - k^2)
//   cbp  = m_p gam_k c_{k,p} a_p
// for beta = k:
//   ck   = gam_k c_kk,  c_kk = sum_l 2 a_l w_l / (a_l^2 - k^2) (real)
//   ckk  = gam_k c_kk k
//   sY   = ck  + sum_p Re cp     (coefficient of the j = i term in Y)
//   sZ   = ckk + sum_p Re cbp
// with gam_k the full prefactor (pi/A) C_k w_k and m_p = 2 for a complex
// pair, 1 for a real node.
template <typename T>
struct ModeTab {
  int32_t* mx;
  int32_t* my;
  T* kx;
  T* ky;
  T* kk;      // |k|
  T* ck;
  T* ckk;
  T* sY;
  T* sZ;
  T* cp;      // [4][NP][R * Kpad]: cp.re, cp.im, cbp.re, cbp.im
};

// SOE pair representatives, shared by all modes and replicas.
struct PairTab {
  int np;                 // number of representatives (padded entries have w = 0)
  double a_re[kMaxPairs]; // a_p = alpha s_p
  double a_im[kMaxPairs];
  double w_re[kMaxPairs];
  double w_im[kMaxPairs];
  double s_re[kMaxPairs];
  double s_im[kMaxPairs];
  double mult[kMaxPairs]; // 2 (complex pair) or 1 (real node) or 0 (padding)
};

// One replica of a call (device array of R).
struct RepInfo {
  int64_t off;            // first particle
  int32_t n;              // particles (may be 0)
  int32_t c0, nch;        // k-space chunks [c0, c0 + nch)
  int32_t z0, nz;         // k = 0 chunks [z0, z0 + nz)
  int32_t g0, ng;         // carry groups [g0, g0 + ng)
  int32_t zg0, nzg;       // k = 0 carry groups [zg0, zg0 + nzg)
  int32_t K;              // modes (half-plane list length, or P)
  int32_t list0;          // offset (in modes) into the concatenated full-k lists
  int32_t cdfx0, nx;      // sampler tables: offsets into the concatenated
  int32_t cdfy0, ny;      //   cumulative tables and their lengths
  int32_t mxmax, mymax;
  double Lx, Ly, Lz, area, H, diagq;
  double k0pre;           // 2 pi / area, the k = 0 term's prefactor
};

// Geometry of a call, passed to kernels by value.
struct Reps {
  int R;
  int L, L0;              // particles per k-space / k = 0 chunk
  int nchunks, nzchunks, ngroups, nzgroups;
  // 1 when every replica's k-space (kflat) or k = 0 (zflat) carry chain is
  // one group: the carries then come from one replay from zero
  int kflat, zflat;
  int Kpad;               // modes per replica (multiple of 32)
  int64_t N;              // particles in all replicas
  const RepInfo* info;        // [R]
  const int32_t* chunk_rep;   // [nchunks]
  const int32_t* zchunk_rep;  // [nzchunks]
  const int32_t* gstart;      // [ngroups + 1] first k-space chunk of each carry group
  const int32_t* group_rep;   // [ngroups]
  const int32_t* zgstart;     // [nzgroups + 1] first k = 0 chunk of each k = 0 carry group
  const int32_t* zgroup_rep;  // [nzgroups]
  unsigned* status;           // the call's status word (debug-build index checks)
};

// Charged walls at z = 0 (bottom) and z = Lz (top), the same for every
// replica (Section 2.4, Thm 2.4): surface charge densities per unit area
// sigma(rho) = s0 + sum_w 2 Re[c_w e^{i k_w.rho}], k_w = 2 pi (mx/Lx, my/Ly).
// Passed to kernels by value (__grid_constant__).
constexpr int kMaxWallModes = 64;
struct WallTab {
  int on;                          // walls set (else the particles must be neutral)
  int nw;                          // Fourier modes, each pair (m, -m) once
  double sb0, st0;                 // uniform parts of sigma_bot, sigma_top
  int32_t m[kMaxWallModes][2];     // (mx, my)
  double c[kMaxWallModes][4];      // c_bot re, im, c_top re, im
};

// Status flags set by kernels (bitwise OR into a device word).
enum StatusBits : unsigned {
  kStNonfinite = 1u,
  kStZRange = 2u,
  kStNonneutral = 4u,
  kStTimeout = 8u,
  kStDebug = 16u,     // debug builds: an internal index check failed
};

// Index checks of the debug build (compiled with -DQSLAB_DEBUG): a failed
// check sets kStDebug in the status word and the kernel skips the access it
// guards (no trap); in the release build the check is `true` and costs
// nothing.
#ifdef QSLAB_DEBUG
__device__ __forceinline__ bool qs_dcheck(bool ok, unsigned* status) {
  if (!ok && status) atomicOr(status, (unsigned)kStDebug);
  return ok;
}
#define QS_DCHECK(ok, status) qslab::qs_dcheck((ok), (status))
#else
#define QS_DCHECK(ok, status) (true)
#endif

// ---- sort (qslab_sort.cu)
struct SortWork {
  void* keys[2];          // keys, ping-pong (room for N keys of key_bytes)
  uint32_t* vals[2];      // payload (original index), ping-pong
  uint32_t* counts;       // [256][nblocks]
  uint32_t* totals;       // [passes][256] digit totals
  int nblocks;
  void* os_state;         // single-pass (onesweep) look-back state
  size_t os_bytes;
  unsigned* status;       // status word: debug-build index checks, the
                          // single-pass sort's bounded waits (may be NULL)
};
size_t sort_workspace_bytes(int64_t N, int key_bytes);
void sort_bind_workspace(SortWork& w, void* base, int64_t N, int key_bytes);
// Stable sort of keys[src]/vals[src] (keys of key_bytes = 4 or 8) on their
// low `passes` bytes; returns the index (0 or 1) of the buffer holding the
// result. onesweep (needs w.status): one kernel per digit with a bounded
// decoupled look-back instead of three; a wait that gives up sets
// kStTimeout, and the sorted arrays are then unspecified (the indices in
// vals may be out of range: consumers clamp them).
int radix_sort(SortWork& w, int64_t N, int key_bytes, int passes, int src, cudaStream_t st,
               bool onesweep = false);
// kernels radix_sort() launches for N keys and `passes` digits
int sort_launches(int64_t N, int passes, bool onesweep = false);
// test hook: in the next single-pass sort, the tile of this ticket in the
// first pass publishes nothing (its successor's bounded wait runs out)
void sort_debug_stall(int tile);

// ---- kernels (qslab_prep.cu: checks, gather, combine, mode tables;
//      qslab_kspace.cu: k != 0 passes; qslab_carry.cu: their carries;
//      qslab_kzero.cu: the k = 0 term)
// Input checks and z keys, one CTA per k-space chunk; per-chunk sums of q
// and |q| (sums[2c], sums[2c+1]); rid (may be NULL) receives the replica of
// every particle.
template <typename T>
void launch_prepare(const Reps& rp, const T* pos, const T* q, void* keys, uint32_t* vals,
                    int32_t* rid, double* sums, unsigned* status, cudaStream_t st);
// Per-replica neutrality check of particles and walls together, from the
// chunk sums of launch_prepare:
// |sum q + area (sb0 + st0)| <= tol (sum |q| + area (|sb0| + |st0|)), with
// sb0 = st0 = 0 without walls; when ctr is not NULL also advances the
// random-batch counter: ctr[1] = ctr[0]++ (the counter this call uses).
void launch_check_neutral(const Reps& rp, const double* sums, double tol, double sb0,
                          double st0, unsigned* status, uint64_t* ctr, cudaStream_t st);
// Second sort key: keys[i] = rid[perm[i]].
void launch_rep_keys(int64_t N, const uint32_t* perm, const int32_t* rid, uint32_t* keys,
                     cudaStream_t st);
// zkeys: the sorted z keys (single-slab calls) or NULL (z gathered from pos)
template <typename T>
void launch_gather(const Reps& rp, const T* pos, const T* q, const uint32_t* perm,
                   const void* zkeys, T* zs, T* dz, T* qs, typename PhaseT<T>::type* xh,
                   typename PhaseT<T>::type* yh, int32_t* perm_out, cudaStream_t st);

struct ScanPlan {
  int KR;           // modes per CTA (threads), multiple of 32
  int nkr;          // number of mode ranges (KR * nkr = Kpad)
  int np;           // pair representatives compiled for (4, 8, 12, 16)
  int nstates;      // 1 + 2 np
  // FP32 pass B: 1 when some warp of some replica holds at most 8 real
  // modes (K mod 32 in 1..8: it runs as a remainder warp, both directions at
  // once, two lanes per mode) or none (K <= Kpad - 32: it only clears its
  // output slots)
  int rem;
};

template <typename T>
void launch_kspace(const ScanPlan& plan, const Reps& rp, const ModeTab<T>& modes,
                   const PairTab& pairs, const T* zs, const T* dz, const T* qs,
                   const typename PhaseT<T>::type* xh,
                   const typename PhaseT<T>::type* yh,
                   const float2* trig,   // FP32: [256] (cos, sin) of j/256 turns
                   Cplx<T>* agg, Cplx<T>* carry, void* dec, T* part,
                   cudaStream_t st, cudaEvent_t* ev3,   // ev3: 3 events or NULL
                   int stage = 0);  // 0: all; 1: pass A + carries; 2: pass B (carries in place)
// bytes of the chunk-to-chunk decay tables and carry-group transfers
size_t kspace_decay_bytes(const ScanPlan& pl, const Reps& rp, int fp64);
// (qslab_carry.cu) the carries of every chunk from the pass-A aggregates;
// dec: kspace_decay_bytes of scratch
template <typename T>
void launch_kspace_carries(const ScanPlan& pl, const Reps& rp, const PairTab& pairs, const T* zs,
                           const T* kk, const Cplx<T>* agg, Cplx<T>* carry, void* dec,
                           cudaStream_t st);
// pair decays between chunk reference points (see qslab_carry.cu); pdec:
// [2][nchunks][np] complex and gaps (may be NULL): [2][nchunks], both in the
// carry type
template <typename T>
void launch_pair_decay(const Reps& rp, int zero_chunks, int np, const T* zs, const PairTab& pairs,
                       void* pdec, void* gaps, cudaStream_t st);

// phi0 / fz0: per sorted particle, in the carry type (FP64 on the FP64 path,
// double-float on the FP32 path)
template <typename T>
void launch_kzero(const Reps& rp, const PairTab& pairs, double alpha, const T* zs,
                  const T* dz, const T* qs, double* work, void* phi0, void* fz0,
                  cudaStream_t st);
size_t kzero_work_doubles(int nzchunks, int nzgroups, int R, int np);

// Potential, forces and per-chunk energies (echunk[nchunks]) back in the
// caller's order; energies[r] (if not NULL) = the sum over replica r's chunks.
// With walls (W.on) the particle-slab potential and its forces are added,
// and the energy gains sum_i q_i phi_p-s,i (zs, xh, yh: sorted z and phases).
template <typename T>
void launch_combine(const Reps& rp, int nkr, const T* part, const void* phi0,
                    const void* fz0, const T* qs, const T* zs,
                    const typename PhaseT<T>::type* xh, const typename PhaseT<T>::type* yh,
                    const WallTab& W, const int32_t* perm, double* echunk,
                    T* phi_out, T* force_out, double* energies, cudaStream_t st);

// Mode tables of all replicas. rbe = 0: modes from `list` (the replicas'
// half-plane lists, concatenated). rbe = 1: K_r = P modes per replica drawn
// on the device from the replica's sampler tables, with the counter ctr[1];
// the drawn (mx, my) go to `sampled` ([R][P] pairs) if it is not NULL.
// rbe = 2: random-batch weights for the modes already in `sampled` (the
// Metropolis chain's). npc = pair count the table is laid out for (compiled
// NP).
//
// Sampler tables per replica (in `cdf`, from cdfx0): the cumulative tables
// of x (nx entries, m = -mxmax..mxmax) and y (ny entries), then the
// Metropolis log-weights -(pi m/(alpha L))^2 - log q(m) of x and y on the
// same ranges (App. G), at cdfx0 + nx + ny and cdfy0 + nx + ny.
template <typename T>
void launch_mode_coef(const Reps& rp, int npc, const int32_t* list, int rbe, uint64_t seed,
                      const uint64_t* ctr, const double* cdf, const PairTab& pairs,
                      double alpha, ModeTab<T> modes, int32_t* sampled, cudaStream_t st);
// The independence Metropolis chain of App. G, one cluster of 8 CTAs per
// replica: P samples (every thin-th state of P * thin steps) per replica
// into `sampled` ([R][P] pairs), with the counter ctr[1].
void launch_mh_chain(const Reps& rp, int P, int thin, uint64_t seed, const uint64_t* ctr,
                     const double* cdf, double alpha, int32_t* sampled, cudaStream_t st);

}  // namespace qslab
