// Internal declarations shared by the qslab CUDA translation units.
//
// Data layout in HBM (all arrays indexed by the z-sorted particle index i):
//   zs[i], dz[i] = zs[i] - zs[i-1] (dz[0] = 0), qs[i]          type T
//   xh[i], yh[i]  fixed-point fractions x/Lx, y/Ly              uint32 (FP32C)
//                 (2^32 or 2^64 units of a turn)                uint64 (FP64)
//   perm[i]       original index of sorted particle i           int32
// Mode tables (one entry per k vector, padded to a multiple of 32 with
// zero-weight modes) are structure-of-arrays, see ModeTab.
// Chunk aggregates and carries: [dir][chunk][state][mode] complex, with
// state 0 = beta = k and states 1+2p, 2+2p = SOE pair p driven by the real
// inputs q cos(k.rho) and q sin(k.rho).
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

// Structure-of-arrays mode table (device pointers). For the SOE pair
// representative p of a mode:
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
  T* cp;      // [4][NP][Kpad]: cp.re, cp.im, cbp.re, cbp.im
};

// SOE pair representatives, shared by all modes (constant over a call).
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

// Status flags set by kernels (bitwise OR into a device word).
enum StatusBits : unsigned {
  kStNonfinite = 1u,
  kStZRange = 2u,
  kStNonneutral = 4u,
  kStTimeout = 8u,
};

// Launch wrappers implemented in the .cu files. All take the caller's stream.
// ---- sort (qslab_sort.cu)
struct SortWork {
  void* keys[2];          // uint32 or uint64 keys, ping-pong
  uint32_t* vals[2];      // payload (original index), ping-pong
  uint32_t* counts;       // [256][nblocks]
  uint32_t* totals;       // [passes][256] digit totals
  int nblocks;
};
size_t sort_workspace_bytes(int64_t N, int key_bytes);
void sort_bind_workspace(SortWork& w, void* base, int64_t N, int key_bytes);
// Sorts keys[0]/vals[0]; returns the index (0 or 1) of the buffer holding the result.
int radix_sort(SortWork& w, int64_t N, int key_bytes, cudaStream_t st);

// ---- kernels (qslab_kernels.cu)
template <typename T>
void launch_prepare(int64_t N, const T* pos, const T* q, double Lz, void* keys,
                    uint32_t* vals, double* sums, unsigned* status,
                    cudaStream_t st);
template <typename T>
void launch_gather(int64_t N, const T* pos, const T* q, const uint32_t* perm,
                   double Lx, double Ly, T* zs, T* dz, T* qs,
                   typename PhaseT<T>::type* xh, typename PhaseT<T>::type* yh,
                   int32_t* perm_out, cudaStream_t st);
void launch_check_neutral(const double* sums, double tol, unsigned* status,
                          cudaStream_t st);

struct ScanPlan {
  int64_t N;
  int L;            // particles per chunk
  int nchunks;
  int Kpad;         // modes, multiple of 32
  int KR;           // modes per CTA (threads), multiple of 32
  int nkr;          // number of mode ranges
  int np;           // pair representatives compiled for (4, 8, 12, 16)
  int nstates;      // 1 + 2 np
};

template <typename T>
void launch_kspace(const ScanPlan& plan, const ModeTab<T>& modes,
                   const PairTab& pairs, const T* zs, const T* dz, const T* qs,
                   const typename PhaseT<T>::type* xh,
                   const typename PhaseT<T>::type* yh, Cplx<T>* agg,
                   Cplx<T>* carry, void* dec, T* part,
                   cudaStream_t st, cudaEvent_t* ev3);  // ev3: 3 events or NULL
// bytes of the chunk-to-chunk decay tables (pair and mode decays)
size_t kspace_decay_bytes(const ScanPlan& pl, int fp64);

// phi0 / fz0: per sorted particle, in the carry type (FP64 on the FP64 path,
// double-float on the FP32 path)
template <typename T>
void launch_kzero(int64_t N, int L0, int nchunks0, const PairTab& pairs,
                  double alpha, double area, const T* zs, const T* dz,
                  const T* qs, double* work, void* phi0, void* fz0,
                  cudaStream_t st);

template <typename T>
void launch_combine(int64_t N, int nkr, const T* part, const void* phi0,
                    const void* fz0, const T* qs, const int32_t* perm,
                    double diagq, double* eblock, int nblk, T* phi_out,
                    T* force_out, double* energy, cudaStream_t st);

// Mode table fill. rbe = 0: modes from `list` (host half-plane list, 2K
// int32). rbe = 1: K = P modes drawn on the device; if `sampled` is not NULL
// the drawn (mx, my) are stored there. npc = pair count the table is laid out
// for (compiled NP).
struct SamplerTab {
  const double* cdfx;
  const double* cdfy;
  int nx, ny;       // table lengths (2 mmax + 1)
  int mxmax, mymax;
};
template <typename T>
void launch_mode_coef(int K, int Kpad, int npc, const int32_t* list, int rbe,
                      uint64_t seed, uint64_t counter, const SamplerTab& sp,
                      const PairTab& pairs, double alpha, double Lx, double Ly,
                      double H, ModeTab<T> modes, int32_t* sampled,
                      cudaStream_t st);

size_t kzero_work_doubles(int nchunks0, int np);

}  // namespace qslab
