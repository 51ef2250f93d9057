// Stable LSD radix sort of z keys with a 32-bit payload (the particle index).
//
// The paper sorts particles by z before the recursions (Section 3.2; it
// notes that a bucket sort makes this O(N), Section 3.4). The recursions need
// the exact order z_1 <= ... <= z_N (Remark 3.3: every exponent must be
// non-positive), so the keys are the IEEE bits of z >= 0 themselves, which
// order exactly like the values; no quantisation.
//
// One pass per 8-bit digit, three kernels per pass:
//   hist    per-tile digit counts, counts[digit][tile]
//   scan    exclusive prefix over counts in digit-major order (one CTA)
//   scatter stable placement: within a warp, keys are ranked in input order
//           with __match_any_sync; warps of a tile are ordered by a per-digit
//           prefix over their counts; tiles by the global scan.
// Up to one tile of keys (kTile = 2048) one CTA does the whole sort in one
// launch instead (small_sort_kernel: a bitonic network over (key, input
// position), which gives the same stable order).
// Several slabs of one call are sorted by z first and then, stably, by their
// slab index (a second LSD sort over one or two more digits), which leaves
// every slab in its own index range and ordered by z within it.
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "qslab_internal.h"

namespace qslab {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kItems = 8;
constexpr int kTile = kSortThreads * kItems;
constexpr int kRadix = 256;

template <typename K>
__global__ void __launch_bounds__(kSortThreads)
hist_kernel(const K* __restrict__ keys, int64_t N, int shift, uint32_t* counts,
            uint32_t* totals, int nblocks) {
  __shared__ uint32_t h[kRadix];
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) h[d] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile;
  for (int s = 0; s < kItems; ++s) {
    int64_t idx = base + (int64_t)s * kSortThreads + threadIdx.x;
    if (idx < N) atomicAdd(&h[(unsigned)(keys[idx] >> shift) & 0xFFu], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
    counts[(int64_t)d * nblocks + blockIdx.x] = h[d];
    if (h[d]) atomicAdd(&totals[d], h[d]);
  }
}

// Exclusive scan of counts[digit][tile] in digit-major order: one CTA per
// digit scans its row (coalesced) and starts from the sum of the totals of
// the smaller digits.
__global__ void __launch_bounds__(kSortThreads)
scan_kernel(uint32_t* counts, const uint32_t* totals, int nblocks) {
  __shared__ uint32_t wsum[kSortWarps];
  __shared__ uint32_t carry;
  const int d = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  // offset of this digit: sum of totals[0..d)
  uint32_t v = (t < d) ? totals[t] : 0u;
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) wsum[w] = v;
  __syncthreads();
  if (t == 0) {
    uint32_t a = 0;
    for (int j = 0; j < kSortWarps; ++j) a += wsum[j];
    carry = a;
  }
  __syncthreads();
  uint32_t* row = counts + (int64_t)d * nblocks;
  for (int b0 = 0; b0 < nblocks; b0 += kSortThreads) {
    const int b = b0 + t;
    const uint32_t x = b < nblocks ? row[b] : 0u;
    uint32_t y = x;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    __syncthreads();
    if (lane == 31) wsum[w] = y;
    __syncthreads();
    uint32_t before = carry;
    for (int j = 0; j < w; ++j) before += wsum[j];
    if (b < nblocks) row[b] = before + y - x;
    __syncthreads();
    if (t == kSortThreads - 1) carry = before + y;
    __syncthreads();
  }
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads)
scatter_kernel(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
               K* __restrict__ kout, uint32_t* __restrict__ vout, int64_t N,
               int shift, const uint32_t* __restrict__ offsets, int nblocks,
               unsigned* status) {
  __shared__ uint32_t wcnt[kSortWarps][kRadix];
  __shared__ uint32_t goff[kRadix];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
    goff[d] = offsets[(int64_t)d * nblocks + blockIdx.x];
    for (int ww = 0; ww < kSortWarps; ++ww) wcnt[ww][d] = 0;
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)w * 32 * kItems;
  K key[kItems];
  uint32_t val[kItems], loc[kItems], dig[kItems];
  for (int s = 0; s < kItems; ++s) {
    const int64_t idx = base + s * 32 + lane;
    const bool valid = idx < N;
    key[s] = valid ? kin[idx] : (K)0;
    val[s] = valid ? vin[idx] : 0u;
    const unsigned d = valid ? ((unsigned)(key[s] >> shift) & 0xFFu) : 0x100u;
    dig[s] = d;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned before = valid ? wcnt[w][d & 0xFFu] : 0u;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[w][d & 0xFFu] = before + __popc(peers);
    __syncwarp();
    loc[s] = before + __popc(peers & lt);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
    uint32_t run = 0;
    for (int ww = 0; ww < kSortWarps; ++ww) {
      uint32_t c = wcnt[ww][d];
      wcnt[ww][d] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int s = 0; s < kItems; ++s) {
    if (dig[s] < 0x100u) {
      const uint32_t pos = goff[dig[s]] + wcnt[w][dig[s]] + loc[s];
      if (QS_DCHECK(pos < (uint64_t)N, status)) {
        kout[pos] = key[s];
        vout[pos] = val[s];
      }
    }
  }
}

// At most one tile (N <= kTile): a bitonic sort in shared memory of the
// pairs (key restricted to its low `passes` bytes, input position). The
// positions are distinct, so the order is total and equals the stable order
// the LSD passes give; one CTA with one thread per compare-exchange pair.
// A stage with stride j <= 32 keeps every warp inside its own 64 elements,
// so only a warp barrier separates two such stages.
template <typename K>
__global__ void __launch_bounds__(1024)
small_sort_kernel(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                  K* __restrict__ kout, uint32_t* __restrict__ vout, int N, int n2, int passes,
                  unsigned* status) {
  __shared__ K sk[kTile];
  __shared__ uint16_t si[kTile];
  const K mask = passes * 8 >= (int)(8 * sizeof(K)) ? ~(K)0 : (((K)1 << (8 * passes)) - 1);
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    // padding sorts after every key: the largest key and position
    sk[t] = t < N ? (kin[t] & mask) : ~(K)0;
    si[t] = t < N ? (uint16_t)t : (uint16_t)0xFFFFu;
  }
  __syncthreads();
  const int half = n2 >> 1;
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < half; t += blockDim.x) {
        const int a = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        const int b = a | j;
        const K ka = sk[a], kb = sk[b];
        const uint16_t ia = si[a], ib = si[b];
        const bool gt = ka > kb || (ka == kb && ia > ib);
        if (gt == ((a & k) == 0)) {     // ascending where bit k of a is clear
          sk[a] = kb; sk[b] = ka;
          si[a] = ib; si[b] = ia;
        }
      }
      const int jn = j > 1 ? j >> 1 : k;  // the next stage's stride
      if (j <= 32 && jn <= 32 && blockDim.x >= half) __syncwarp();
      else __syncthreads();
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const int i = si[t];
    if (!QS_DCHECK(i < N, status)) continue;
    kout[t] = kin[i];
    vout[t] = vin[i];
  }
}

// ---------------------------------------------------------------- onesweep
// One kernel per digit pass, with the offsets of earlier tiles found by a
// decoupled look-back (Merrill and Garland's single-pass prefix scan, as
// used for radix sorting by Adinets and Merrill's Onesweep): tiles take
// tickets in launch order; each publishes its digit counts at once
// (aggregate), reads back through the earlier tiles' words until an
// inclusive prefix, and publishes its own inclusive prefix. The global digit
// offsets come from one histogram of every pass's digit over all keys,
// taken before the first pass. A tile waits only on tiles with smaller
// tickets, which are already running, so every wait ends; each wait is
// still bounded: after kSpinLimit polls the tile records a timeout in the
// status word, publishes an error word (its successors stop there), and
// scatters nothing. Every later pass of the sort then does nothing, and the
// consumers of the permutation clamp its entries, so a timed-out sort leaves
// wrong values but no access out of range.
constexpr int kOsItems = 16;
constexpr int kOsTile = kSortThreads * kOsItems;   // 4096 keys per tile
constexpr uint32_t kFlagAgg = 1u, kFlagInc = 2u, kFlagErr = 3u;
constexpr int kSpinLimit = 1 << 20;
constexpr int kOsWindow = 8;       // earlier tiles' words read per round of the look-back

// all passes' digit histograms in one read of the keys
template <typename K>
__global__ void __launch_bounds__(kSortThreads)
os_hist_kernel(const K* __restrict__ keys, int64_t N, int passes, uint32_t* gtot) {
  __shared__ uint32_t h[8][kRadix];
  for (int e = threadIdx.x; e < passes * kRadix; e += blockDim.x) h[e / kRadix][e % kRadix] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const K k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(unsigned)(k >> (8 * p)) & 0xFFu], 1u);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < passes * kRadix; e += blockDim.x) {
    const uint32_t v = h[e / kRadix][e % kRadix];
    if (v) atomicAdd(&gtot[e], v);
  }
}

__device__ __forceinline__ uint64_t os_word(uint32_t flag, uint32_t count) {
  return ((uint64_t)flag << 32) | count;
}

// stall: the tile of this ticket publishes nothing (a test of the bounded
// wait; -1 in normal use)
template <typename K>
__global__ void __launch_bounds__(kSortThreads)
os_pass_kernel(const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
               uint32_t* __restrict__ vout, int64_t N, int shift, const uint32_t* __restrict__ gtot,
               unsigned long long* tstat, unsigned* ticket, unsigned* status, int stall) {
  __shared__ uint32_t wcnt[kSortWarps][kRadix];
  __shared__ uint32_t toff[kRadix];
  __shared__ uint32_t goff[kRadix];
  __shared__ uint32_t wsum[kSortWarps];
  __shared__ int tile_s, bad_s;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    tile_s = (int)atomicAdd(ticket, 1u);
    bad_s = (status && (*(volatile unsigned*)status & kStTimeout)) ? 1 : 0;
  }
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x)
    for (int ww = 0; ww < kSortWarps; ++ww) wcnt[ww][d] = 0;
  __syncthreads();
  const int tile = tile_s;
  unsigned long long* my = tstat + (size_t)tile * kRadix;
  if (bad_s) {   // an earlier pass timed out: publish errors, move nothing
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) atomicExch(&my[d], os_word(kFlagErr, 0));
    return;
  }
  // ranks within the tile: per warp in input order (match_any), then warps
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)tile * kOsTile + (int64_t)w * 32 * kOsItems;
  K key[kOsItems];
  uint32_t val[kOsItems], loc[kOsItems], dig[kOsItems];
#pragma unroll
  for (int s = 0; s < kOsItems; ++s) {
    const int64_t idx = base + s * 32 + lane;
    const bool valid = idx < N;
    key[s] = valid ? kin[idx] : (K)0;
    val[s] = valid ? vin[idx] : 0u;
    const unsigned d = valid ? ((unsigned)(key[s] >> shift) & 0xFFu) : 0x100u;
    dig[s] = d;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned before = valid ? wcnt[w][d & 0xFFu] : 0u;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[w][d & 0xFFu] = before + __popc(peers);
    __syncwarp();
    loc[s] = before + __popc(peers & lt);
  }
  __syncthreads();
  // one thread per digit: warp prefix, the tile's count, publish, look back
  const int d = threadIdx.x;      // kSortThreads == kRadix
  uint32_t run = 0;
  for (int ww = 0; ww < kSortWarps; ++ww) {
    const uint32_t c = wcnt[ww][d];
    wcnt[ww][d] = run;
    run += c;
  }
  const bool stalled = tile == stall;
  if (!stalled) atomicExch(&my[d], os_word(tile == 0 ? kFlagInc : kFlagAgg, run));
  uint32_t prefix = 0;
  bool err = stalled;
  if (tile > 0 && !stalled) {
    // read back eight earlier tiles' words at a time (independent loads),
    // consume them in order up to an inclusive prefix, or up to a word not
    // yet published, which is polled again
    int j = tile - 1;
    int spins = 0;
    bool done = false;
    while (!done) {
      uint64_t v[kOsWindow];
#pragma unroll
      for (int u = 0; u < kOsWindow; ++u)
        v[u] = j - u >= 0 ? *(volatile unsigned long long*)&tstat[(size_t)(j - u) * kRadix + d]
                          : os_word(kFlagInc, 0);
      int used = 0;
      bool wait = false;
#pragma unroll
      for (int u = 0; u < kOsWindow; ++u) {
        if (done || wait) continue;
        const uint32_t f = (uint32_t)(v[u] >> 32);
        if (f == 0u) { wait = true; continue; }
        if (f == kFlagErr) { err = true; done = true; continue; }
        prefix += (uint32_t)v[u];
        ++used;
        if (f == kFlagInc) done = true;
      }
      if (done) break;
      j -= used;
      if (wait) {
        if (++spins > kSpinLimit) { err = true; break; }
        __nanosleep(64);
      }
    }
    atomicExch(&my[d], err ? os_word(kFlagErr, 0) : os_word(kFlagInc, prefix + run));
  }
  toff[d] = prefix;
  // exclusive scan of the global digit totals (the same in every tile)
  const uint32_t g = gtot[d];
  uint32_t y = g;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
    if (lane >= o) y += z;
  }
  if (lane == 31) wsum[w] = y;
  const unsigned anyerr = __syncthreads_or(err ? 1 : 0);
  uint32_t b = 0;
  for (int ww = 0; ww < w; ++ww) b += wsum[ww];
  goff[d] = b + y - g;
  __syncthreads();
  if (anyerr) {
    if (threadIdx.x == 0 && status) atomicOr(status, (unsigned)kStTimeout);
    return;
  }
#pragma unroll
  for (int s = 0; s < kOsItems; ++s) {
    if (dig[s] < 0x100u) {
      const uint64_t pos = (uint64_t)goff[dig[s]] + toff[dig[s]] + wcnt[w][dig[s]] + loc[s];
      if (pos < (uint64_t)N) {
        kout[pos] = key[s];
        vout[pos] = val[s];
      }
    }
  }
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// onesweep state: [passes][tiles][256] look-back words, [passes] tickets,
// [passes][256] global digit totals (cleared together before a sort)
size_t os_state_bytes(int64_t N, int passes) {
  const int64_t nt = (N + kOsTile - 1) / kOsTile;
  return align256((size_t)passes * nt * kRadix * 8) + align256((size_t)passes * 4) +
         align256((size_t)passes * kRadix * 4);
}

size_t sort_workspace_bytes(int64_t N, int key_bytes) {
  const int64_t nb = (N + kTile - 1) / kTile;
  return 2 * align256((size_t)N * key_bytes) + 2 * align256((size_t)N * 4) +
         align256((size_t)nb * kRadix * 4) + align256(8 * kRadix * 4) +
         os_state_bytes(N, key_bytes);
}

void sort_bind_workspace(SortWork& w, void* base, int64_t N, int key_bytes) {
  char* p = static_cast<char*>(base);
  w.nblocks = (int)((N + kTile - 1) / kTile);
  w.keys[0] = p; p += align256((size_t)N * key_bytes);
  w.keys[1] = p; p += align256((size_t)N * key_bytes);
  w.vals[0] = reinterpret_cast<uint32_t*>(p); p += align256((size_t)N * 4);
  w.vals[1] = reinterpret_cast<uint32_t*>(p); p += align256((size_t)N * 4);
  w.counts = reinterpret_cast<uint32_t*>(p);
  p += align256((size_t)w.nblocks * kRadix * 4);
  w.totals = reinterpret_cast<uint32_t*>(p);
  p += align256(8 * kRadix * 4);
  w.os_state = p;
  w.os_bytes = os_state_bytes(N, key_bytes);
  w.status = nullptr;
}

namespace {
std::atomic<int> g_sort_stall{-1};
}

void sort_debug_stall(int tile) { g_sort_stall.store(tile); }

int sort_launches(int64_t N, int passes, bool onesweep) {
  if (N <= kTile) return 1;
  return onesweep ? 1 + passes : 3 * passes;
}

template <typename K>
static int onesweep_sort(SortWork& w, int64_t N, int passes, int src, cudaStream_t st) {
  const int64_t nt = (N + kOsTile - 1) / kOsTile;
  char* p = static_cast<char*>(w.os_state);
  auto* tstat = reinterpret_cast<unsigned long long*>(p);
  p += align256((size_t)passes * nt * kRadix * 8);
  auto* tickets = reinterpret_cast<unsigned*>(p);
  p += align256((size_t)passes * 4);
  auto* gtot = reinterpret_cast<uint32_t*>(p);
  cudaMemsetAsync(w.os_state, 0, os_state_bytes(N, passes), st);
  int hb = (int)((N + kSortThreads * 16 - 1) / (kSortThreads * 16));
  if (hb > 152 * 8) hb = 152 * 8;
  os_hist_kernel<K><<<hb, kSortThreads, 0, st>>>(static_cast<const K*>(w.keys[src]), N, passes,
                                                  gtot);
  const int stall = g_sort_stall.exchange(-1);
  int cur = src;
  for (int q = 0; q < passes; ++q) {
    os_pass_kernel<K><<<(unsigned)nt, kSortThreads, 0, st>>>(
        static_cast<const K*>(w.keys[cur]), w.vals[cur], static_cast<K*>(w.keys[cur ^ 1]),
        w.vals[cur ^ 1], N, 8 * q, gtot + (size_t)q * kRadix, tstat + (size_t)q * nt * kRadix,
        tickets + q, w.status, q == 0 ? stall : -1);
    cur ^= 1;
  }
  return cur;
}

int radix_sort(SortWork& w, int64_t N, int key_bytes, int passes, int src, cudaStream_t st,
               bool onesweep) {
  int cur = src;
  if (N <= kTile) {
    // small sorts: one CTA, buffer src in, the other out
    int n2 = 2;
    while (n2 < N) n2 <<= 1;
    const int thr = n2 / 2 < 32 ? 32 : n2 / 2;
    if (key_bytes == 4)
      small_sort_kernel<uint32_t><<<1, thr, 0, st>>>(
          static_cast<const uint32_t*>(w.keys[cur]), w.vals[cur],
          static_cast<uint32_t*>(w.keys[cur ^ 1]), w.vals[cur ^ 1], (int)N, n2, passes, w.status);
    else
      small_sort_kernel<uint64_t><<<1, thr, 0, st>>>(
          static_cast<const uint64_t*>(w.keys[cur]), w.vals[cur],
          static_cast<uint64_t*>(w.keys[cur ^ 1]), w.vals[cur ^ 1], (int)N, n2, passes, w.status);
    return cur ^ 1;
  }
  if (onesweep && w.status) {
    if (key_bytes == 4) return onesweep_sort<uint32_t>(w, N, passes, src, st);
    return onesweep_sort<uint64_t>(w, N, passes, src, st);
  }
  cudaMemsetAsync(w.totals, 0, (size_t)passes * kRadix * 4, st);
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    uint32_t* tot = w.totals + p * kRadix;
    if (key_bytes == 4) {
      auto* kin = static_cast<const uint32_t*>(w.keys[cur]);
      auto* kout = static_cast<uint32_t*>(w.keys[cur ^ 1]);
      hist_kernel<uint32_t><<<w.nblocks, kSortThreads, 0, st>>>(kin, N, shift, w.counts, tot, w.nblocks);
      scan_kernel<<<kRadix, kSortThreads, 0, st>>>(w.counts, tot, w.nblocks);
      scatter_kernel<uint32_t><<<w.nblocks, kSortThreads, 0, st>>>(
          kin, w.vals[cur], kout, w.vals[cur ^ 1], N, shift, w.counts, w.nblocks, w.status);
    } else {
      auto* kin = static_cast<const uint64_t*>(w.keys[cur]);
      auto* kout = static_cast<uint64_t*>(w.keys[cur ^ 1]);
      hist_kernel<uint64_t><<<w.nblocks, kSortThreads, 0, st>>>(kin, N, shift, w.counts, tot, w.nblocks);
      scan_kernel<<<kRadix, kSortThreads, 0, st>>>(w.counts, tot, w.nblocks);
      scatter_kernel<uint64_t><<<w.nblocks, kSortThreads, 0, st>>>(
          kin, w.vals[cur], kout, w.vals[cur ^ 1], N, shift, w.counts, w.nblocks, w.status);
    }
    cur ^= 1;
  }
  return cur;
}

}  // namespace qslab
