// Chunk geometry shared by the qslab kernels: which particles a chunk of a
// replica owns, and the z gap between neighbouring chunks' reference points.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "qslab_internal.h"

namespace qslab {

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

// A chunk of L (or L0) particles inside the particle arrays (debug-build
// checks of the chunk tables).
__device__ __forceinline__ bool chunk_ok(const Reps& rp, const CRange& ch, int L) {
  return ch.r >= 0 && ch.r < rp.R && ch.cnt >= 1 && ch.cnt <= L && ch.start >= 0 &&
         ch.start + ch.cnt <= rp.N;
}

inline int chunk_threads(int L) {
  const int t = ((L + 31) / 32) * 32;
  return t < 256 ? t : 256;
}

// Gap between the reference points of chunk ch and its predecessor along
// direction dir: forward z_end(c) - z_end(c-1), backward z_start(c+1) -
// z_start(c). 0 where the chain of a replica starts (its carry is 0).
template <typename T>
__device__ inline double chunk_gap(const T* zs, const CRange& ch, int dir, int L) {
  if (dir == 0) {
    if (ch.first) return 0.0;
    return (double)zs[ch.start + ch.cnt - 1] - (double)zs[ch.start - 1];
  }
  if (ch.last) return 0.0;
  return (double)zs[ch.start + L] - (double)zs[ch.start];   // chunk c is full
}

}  // namespace qslab
