// LSD radix machinery for the tensor-path sort (paper Sec. 4.2: the sort is a
// relocation of rows along the key axis, digit by digit) on sm_103a.
//
//   k_stats      : min / max of the keys of every array (one read of the keys);
//                  the planner turns them into (lo, significant bits).
//   k_histogram  : the counts of every digit of every pass, in one read of the
//                  keys (per-CTA shared-memory histograms merged into global).
//   k_digit_scan : exclusive scan of each pass's digit counts (digit bases).
//   k_onesweep   : one digit pass: a tile of 1536 to 3840 rows is copied to
//                  shared memory, publishes its digit counts to a decoupled
//                  look-back chain, is ranked stably inside the CTA (digit
//                  groups of a warp matched by a shared lane-mask table or by
//                  ballots, + per-warp counters), and is
//                  written out in tile-sorted order so that each digit's run
//                  lands contiguously.
//
// Every kernel takes an array of jobs so that one launch serves any number of
// arrays (both sides of a join, or thousands of joins of a batch).
#include "tj_internal.cuh"
#include "tj_warp.cuh"

namespace tj {

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
template <typename Job>
__device__ __forceinline__ int find_job(const Job* jobs, int num_jobs, int64_t t) {
  int lo = 0, hi = num_jobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile0 <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_volatile_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.volatile.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long order_u(int32_t k) {
  return (unsigned long long)((uint32_t)k ^ 0x80000000u);
}
__device__ __forceinline__ unsigned long long order_u(int64_t k) {
  return (unsigned long long)k ^ 0x8000000000000000ull;
}

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, typename UnsignedOf<K>::type lo, int shift,
                                             uint32_t mask) {
  using U = typename UnsignedOf<K>::type;
  return (uint32_t)((((U)key) - lo) >> shift) & mask;
}

// Route through the radix index: the cuts <= key are all cuts before the key's
// bucket plus those of its bucket that are <= key, found by `steps` halvings
// of the bucket (the same count on every lane: no divergence).
template <typename K>
__device__ __forceinline__ uint32_t route_idx(K key, typename UnsignedOf<K>::type lo,
                                              const K* s_cuts, const uint16_t* s_tab, int steps,
                                              int ushift) {
  using U = typename UnsignedOf<K>::type;
  // keys below lo (a range estimated from a sample) take bucket 0
  const unsigned long long x = key < (K)lo ? 0ull : (unsigned long long)(U)((U)key - lo);
  uint32_t b;
  if (ushift >= 0) {
    // uniform index; keys of the range give b < kRouteBuckets - 1, the clamp
    // keeps any other value (a tile's padding rows) inside the table
    const unsigned long long u = x >> ushift;
    b = u < (unsigned long long)(kRouteBuckets - 1) ? (uint32_t)u : (uint32_t)(kRouteBuckets - 1);
  } else {
    const int nb = 64 - __clzll(x);  // significant bits of x
    b = nb < 6 ? (uint32_t)x : (uint32_t)((nb << 5) | ((x >> (nb - 6)) & 31ull));
  }
  int a = s_tab[b];
  int n = (int)s_tab[b + 1] - a;
  for (int i = 0; i < steps; ++i) {
    const int half = n >> 1;
    const bool go = n > 0 && s_cuts[a + half] <= key;  // a + half < ncuts when n > 0
    a = go ? a + half + 1 : a;
    n = go ? n - half - 1 : half;
  }
  return (uint32_t)a;
}

// Exclusive scan of in[0, bins) into out[0, bins) by the whole CTA
// (bins <= 2 * kThreads).  Ends with a barrier.
__device__ __forceinline__ void block_excl_scan_bins(const uint32_t* in, uint32_t* out, int bins,
                                                     uint32_t* s_warp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int d0 = tid * 2;
  const uint32_t a = d0 < bins ? in[d0] : 0u;
  const uint32_t b = d0 + 1 < bins ? in[d0 + 1] : 0u;
  const uint32_t s = a + b;
  uint32_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  uint32_t wpre = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w)
    if (w < warp) wpre += s_warp[w];
  const uint32_t excl = wpre + x - s;
  if (d0 < bins) out[d0] = excl;
  if (d0 + 1 < bins) out[d0 + 1] = excl + a;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// K1: min / max of every array's keys
// ---------------------------------------------------------------------------
template <typename K>
__global__ void __launch_bounds__(kThreads) k_stats(const RadixJob<K>* __restrict__ jobs,
                                                    int num_jobs, int64_t total_tiles,
                                                    KeyStats* __restrict__ stats, int tile) {
  __shared__ unsigned long long s_mn[kWarps], s_mx[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // a contiguous run of tiles per CTA: one reduction and one pair of atomics
  // per job the run touches
  const int64_t per = (total_tiles + gridDim.x - 1) / gridDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(total_tiles, t0 + per);
  int cur = -1;
  int64_t cur_end = 0;  // first tile after the current job
  unsigned long long mn = ~0ull, mx = 0ull;
  auto flush = [&]() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long a = __shfl_xor_sync(0xFFFFFFFFu, mn, o);
      unsigned long long b = __shfl_xor_sync(0xFFFFFFFFu, mx, o);
      mn = a < mn ? a : mn;
      mx = b > mx ? b : mx;
    }
    if (lane == 0) {
      s_mn[warp] = mn;
      s_mx[warp] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kWarps; ++w) {
        mn = s_mn[w] < mn ? s_mn[w] : mn;
        mx = s_mx[w] > mx ? s_mx[w] : mx;
      }
      atomicMin(&stats[cur].min_u, mn);
      atomicMin(&stats[cur].max_u, ~mx);  // stored inverted so both fields use atomicMin
    }
    __syncthreads();
    mn = ~0ull;
    mx = 0ull;
  };
  for (int64_t t = t0; t < t1; ++t) {
    if (cur < 0 || t >= cur_end) {
      if (cur >= 0) flush();
      cur = find_job(jobs, num_jobs, t);
      cur_end = jobs[cur].tile0 + (jobs[cur].n + tile - 1) / tile;
    }
    const K* __restrict__ keys = jobs[cur].keys;
    const int64_t row0 = (t - jobs[cur].tile0) * tile;
    const int64_t row1 = min(jobs[cur].n, row0 + tile);
#pragma unroll 4
    for (int64_t r = row0 + threadIdx.x; r < row1; r += kThreads) {
      const unsigned long long u = order_u(keys[r]);
      mn = u < mn ? u : mn;
      mx = u > mx ? u : mx;
    }
  }
  if (cur >= 0) flush();
}

// ---------------------------------------------------------------------------
// K2: digit histograms of every pass in one read of the keys
// ---------------------------------------------------------------------------
// passes x 2^digit_bits never exceeds this (64-bit keys: 8 x 2^8 or 7 x 2^9;
// 32-bit keys: <= 4 x 2^8 or 3 x 2^10; a route pass: 1 x 2^10)
constexpr int kHistWords = 4096;

// Counts of every pass's digit for the rows a thread loaded (P passes known at
// compile time; NARROW: all digits lie in the low 32 bits of key - lo).
template <typename K, int P, bool NARROW, int N>
__device__ __forceinline__ void hist_rows(const K (&kv)[N], int row1,
                                          typename UnsignedOf<K>::type lo, const int (&sh)[kMaxPasses],
                                          const uint32_t (&mk)[kMaxPasses], uint32_t* s_h, int hs) {
  using U = typename UnsignedOf<K>::type;
#pragma unroll
  for (int u = 0; u < N; ++u) {
    if ((int)threadIdx.x + u * kThreads < row1) {
      if (NARROW) {
        const uint32_t x = (uint32_t)kv[u] - (uint32_t)lo;
#pragma unroll
        for (int p = 0; p < P; ++p) atomicAdd(&s_h[p * hs + ((x >> sh[p]) & mk[p])], 1u);
      } else {
        const U x = (U)kv[u] - lo;
#pragma unroll
        for (int p = 0; p < P; ++p)
          atomicAdd(&s_h[p * hs + ((uint32_t)(x >> sh[p]) & mk[p])], 1u);
      }
    }
  }
}

template <typename K>
__global__ void __launch_bounds__(kThreads, 6) k_histogram(const RadixJob<K>* __restrict__ jobs,
                                                        int num_jobs, int64_t total_tiles,
                                                        const int32_t* __restrict__ tile_job,
                                                        int tile) {
  using U = typename UnsignedOf<K>::type;
  __shared__ uint32_t s_h[kHistWords];
  __shared__ int s_shift[kMaxPasses];
  __shared__ uint32_t s_mask[kMaxPasses];
  __shared__ K s_cuts[kMaxCuts];
  __shared__ uint16_t s_tab[kRouteBuckets + 1];
  int cur = -1, passes = 0, ncuts = -1, hs = 0, rsteps = 0, rshift = -1;
  bool narrow = false;
  U lo = 0;
  int sh[kMaxPasses];
  uint32_t mk[kMaxPasses];
#pragma unroll
  for (int p = 0; p < kMaxPasses; ++p) {
    sh[p] = 0;
    mk[p] = 0u;
  }
  auto flush = [&](int job) {
    __syncthreads();
    for (int p = 0; p < passes; ++p)
      for (int d = threadIdx.x; d <= (int)s_mask[p]; d += kThreads) {
        const uint32_t c = s_h[p * hs + d];
        if (c) atomicAdd(&jobs[job].hist[p * jobs[job].hist_stride + d], c);
      }
  };
  // a contiguous run of tiles per CTA: one flush per job the run touches
  const int64_t per = (total_tiles + gridDim.x - 1) / gridDim.x;
  const int64_t t_end = min(total_tiles, (int64_t)(blockIdx.x + 1) * per);
  for (int64_t t = (int64_t)blockIdx.x * per; t < t_end; ++t) {
    const int j = tile_job ? tile_job[t] : find_job(jobs, num_jobs, t);
    if (j != cur) {
      if (cur >= 0) flush(cur);
      __syncthreads();
      cur = j;
      passes = jobs[j].passes;
      lo = (U)jobs[j].lo;
      ncuts = jobs[j].cuts ? jobs[j].ncuts : -1;
      rsteps = jobs[j].route_steps;
      rshift = jobs[j].route_shift;
      int mb = 0;
      for (int p = 0; p < passes; ++p) mb = max(mb, jobs[j].bits[p]);
      hs = 1 << mb;
      if (ncuts >= 0) {
        for (int i = threadIdx.x; i < kMaxCuts; i += kThreads) s_cuts[i] = jobs[j].cuts[i];
        for (int i = threadIdx.x; i <= kRouteBuckets; i += kThreads) s_tab[i] = jobs[j].route_tab[i];
      }
      if (threadIdx.x < kMaxPasses) {
        s_shift[threadIdx.x] = jobs[j].shift[threadIdx.x];
        s_mask[threadIdx.x] =
            threadIdx.x < passes ? (1u << jobs[j].bits[threadIdx.x]) - 1u : 0u;
      }
#pragma unroll
      for (int p = 0; p < kMaxPasses; ++p) {
        sh[p] = p < passes ? jobs[j].shift[p] : 0;
        mk[p] = p < passes ? (1u << jobs[j].bits[p]) - 1u : 0u;
      }
      narrow = passes > 0 && jobs[j].shift[passes - 1] + jobs[j].bits[passes - 1] <= 32;
      for (int i = threadIdx.x; i < passes * hs; i += kThreads) s_h[i] = 0;
      __syncthreads();
    }
    const K* __restrict__ keys = jobs[j].keys;
    const int64_t row0 = (t - jobs[j].tile0) * tile;
    const int row1 = (int)min((int64_t)tile, jobs[j].n - row0);  // tile <= kTile
    const K* __restrict__ kp = keys + row0;
    constexpr int kU = kTile / kThreads;  // up to 16 rows per thread, loads issued together
    K kv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = threadIdx.x + u * kThreads;
      kv[u] = r < row1 ? kp[r] : K(0);
    }
    if (ncuts >= 0) {
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if ((int)threadIdx.x + u * kThreads < row1)
          atomicAdd(&s_h[route_idx<K>(kv[u], lo, s_cuts, s_tab, rsteps, rshift)], 1u);
    } else {
#define TJ_HIST_CASE(P)                                                   \
  case P:                                                                 \
    if (narrow)                                                           \
      hist_rows<K, P, true>(kv, row1, lo, sh, mk, s_h, hs);               \
    else                                                                  \
      hist_rows<K, P, false>(kv, row1, lo, sh, mk, s_h, hs);              \
    break;
      switch (passes) {
        TJ_HIST_CASE(1)
        TJ_HIST_CASE(2)
        TJ_HIST_CASE(3)
        TJ_HIST_CASE(4)
        TJ_HIST_CASE(5)
        TJ_HIST_CASE(6)
        TJ_HIST_CASE(7)
        TJ_HIST_CASE(8)
        default: break;
      }
#undef TJ_HIST_CASE
    }
  }
  if (cur >= 0) flush(cur);
}

// ---------------------------------------------------------------------------
// K3: exclusive scan of each (job, pass) digit histogram, in place
// ---------------------------------------------------------------------------
template <typename K>
__global__ void k_digit_scan(const RadixJob<K>* __restrict__ jobs, int num_jobs, int passes) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= (int64_t)num_jobs * passes) return;
  const int j = (int)(gw / passes), p = (int)(gw % passes);
  if (p >= jobs[j].passes) return;
  const int bins = 1 << jobs[j].bits[p];
  uint32_t* h = jobs[j].hist + p * jobs[j].hist_stride;
  uint32_t carry = 0;
  for (int base = 0; base < bins; base += 32) {
    const uint32_t v = (base + lane < bins) ? h[base + lane] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (base + lane < bins) h[base + lane] = carry + x - v;
    carry += __shfl_sync(0xFFFFFFFFu, x, 31);
  }
}

// ---------------------------------------------------------------------------
// K4: one onesweep digit pass
// ---------------------------------------------------------------------------
// Shared memory (bins = 2^bits of this pass, set at launch; hb = ceil(bins/2)):
//   keys[tile + 16 B] K | ids[tile + 16 B] K   rows in input order (never moved),
//                                       each starting where its source's address
//                                       modulo 16 puts it
//   src[tile] u16                       input row of each tile-sorted slot
//   warp counters[kSortWarps][hb] u32   two 16-bit digit counters per word
//   tile count[bins] u32 | tile exclusive[bins] u32 | global base[bins] i64
//   [route passes by the cut table: cut keys[bins] K | radix index[kRouteBuckets + 8]
//    u16 | digit of each tile-sorted slot[tile] u8 (<= 256 bins) or u16]
//   (a route pass has fewer than bins cuts)
//   [route passes whose regions are sized ahead: end of each batch's region[bins] u32]
template <typename K>
__host__ __device__ constexpr size_t onesweep_smem_bytes(int bins, int mode, int tile = kTile,
                                                         bool guard = false) {
  return 2 * sizeof(K) * (size_t)tile + 2 * 16 + sizeof(uint16_t) * (size_t)tile +
         sizeof(uint32_t) * (size_t)kSortWarps * (size_t)((bins + 1) / 2) +
         sizeof(uint32_t) * 3 * (size_t)bins +
         (mode == kModeCuts ? sizeof(K) * (size_t)bins + sizeof(uint16_t) * (kRouteBuckets + 8) +
                                  (bins <= 256 ? 1 : (bins <= 512 || !guard) ? 2 : 0) * (size_t)tile
                            : 0) +
         (mode != kModeSort && guard ? sizeof(uint32_t) * (size_t)bins : 0);
}

// Exclusive scan of in[0, bins) by a CTA of kSortThreads (bins <= kMaxBins):
// thread t scans entries [t * kPer, (t + 1) * kPer).  Ends with a barrier.
__device__ __forceinline__ void sort_block_excl_scan(const uint32_t* in, uint32_t* out, int bins,
                                                     uint32_t* s_warp) {
  constexpr int kPer = (kMaxBins + kSortThreads - 1) / kSortThreads;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int d0 = tid * kPer;
  uint32_t v[kPer];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    v[i] = d0 + i < bins ? in[d0 + i] : 0u;
    s += v[i];
  }
  uint32_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  uint32_t run = x - s;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w)
    if (w < warp) run += s_warp[w];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    if (d0 + i < bins) out[d0 + i] = run;
    run += v[i];
  }
  __syncthreads();
}

// Sum look-back words v[0..W) (newest predecessor first) into `prefix` up to
// and including the first inclusive word; stop early at a predecessor that
// has published nothing yet.  Returns the number of words consumed.
template <int W>
__device__ __forceinline__ int lookback_consume(const uint32_t (&v)[W], uint32_t& prefix,
                                                bool& done) {
  int used = 0;
  uint32_t acc = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    if (used != w) break;
    const uint32_t f = v[w] & ~kValMask;
    if (f == 0u) break;
    acc += v[w] & kValMask;
    ++used;
    if (f == kFlagInc) {
      done = true;
      break;
    }
  }
  prefix += acc;
  return used;
}

// Asynchronous global -> shared copy of n <= TILE elements of K (no registers
// held) into `area` (TILE + 16 / sizeof(K) elements, 16-byte aligned).  The
// copy starts at area + (src mod 16) / sizeof(K), so both ends agree modulo
// 16 and all but a head and a tail element move in 16-byte chunks whatever
// the source's alignment; returns where it starts.  Every loop has a fixed
// trip count (predicated), so the compiler unrolls it.
template <typename K, int TILE>
__device__ __forceinline__ K* copy_rows_async(K* area, const K* __restrict__ src, int n) {
  constexpr int kPer = 16 / (int)sizeof(K);
  const uint32_t mis = (uint32_t)((uintptr_t)src & 15u);  // a multiple of sizeof(K)
  K* d = area + mis / sizeof(K);
  const uint32_t sd = (uint32_t)__cvta_generic_to_shared(d);
  const int head = min(n, mis ? (int)((16u - mis) / sizeof(K)) : 0);
  const int chunks = (n - head) / kPer;
  const int tail0 = head + chunks * kPer;
  const int tid = threadIdx.x;
  if (tid < head)
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sd + (uint32_t)(tid * sizeof(K))),
                 "l"(src + tid), "n"(sizeof(K))
                 : "memory");
  constexpr int kIters = (TILE / kPer + kSortThreads - 1) / kSortThreads;
#pragma unroll
  for (int it = 0; it < kIters; ++it) {
    const int c = tid + it * kSortThreads;
    if (c < chunks)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                       sd + (uint32_t)(head * sizeof(K)) + 16u * c),
                   "l"(src + head + c * kPer)
                   : "memory");
  }
  if (tid < n - tail0)
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(
                     sd + (uint32_t)((tail0 + tid) * sizeof(K))),
                 "l"(src + tail0 + tid), "n"(sizeof(K))
                 : "memory");
  return d;
}

// One LSD pass over a tile of kSortThreads * ITEMS rows:
//   1. copy the tile's keys and ids into shared memory (cp.async, 16-byte
//      chunks) where they stay in input order;
//   2. take every row's digit, count the tile's digits (shared atomics) and
//      publish the counts to the look-back chain at once, so that successors
//      rarely wait on this tile;
//   3. rank stably inside each warp (rank_items_or / rank_items; warp w owns rows
//      [w*32*ITEMS, (w+1)*32*ITEMS), item i covers 32 consecutive rows);
//   4. record, for every tile-sorted slot, its input row (a 16-bit index)
//      while the first look-back window is in flight, then finish the
//      look-back (bounded wait; on timeout report TJ_ERR_TIMEOUT and go on);
//   5. walk the slots in order and write each row to its global position:
//      consecutive slots of one digit go to consecutive addresses.
// MODE: kModeSort (digit = bits of key - lo), kModeCuts (route pass, pass 0:
// digit = batch index from the cut table) or kModeRadix (route pass, pass 0:
// digit = bits of clamp(key, lo, hi) - lo, equal-width batches).
template <typename K, int ITEMS, int MODE>
__global__ void __launch_bounds__(kSortThreads, TJ_SORT_MINB)
    k_onesweep(const RadixJob<K>* __restrict__ jobs, int num_jobs, int64_t total_tiles, int pass,
               uint32_t* __restrict__ tile_counter, int* __restrict__ err,
               const int32_t* __restrict__ tile_job) {
  using U = typename UnsignedOf<K>::type;
  constexpr int TILE = kSortThreads * ITEMS;
  static_assert(TILE <= 65536, "slot indices are 16-bit");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_warp[kSortWarps];
  __shared__ uint32_t s_t;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_t = atomicAdd(tile_counter, 1u);
  __syncthreads();
  const int64_t t = s_t;
  if (t >= total_tiles) return;
  const int j = tile_job ? tile_job[t] : find_job(jobs, num_jobs, t);
  const RadixJob<K>* J = jobs + j;
  if (pass >= J->passes) return;  // this array needs fewer passes than the batch
  const int64_t lt = t - J->tile0;
  const int64_t row0 = lt * TILE;
  const int nvalid = (int)min((int64_t)TILE, J->n - row0);
  const int shift = J->shift[pass];
  const int nbits = J->bits[pass];
  const int bins = 1 << nbits;
  const int hb = (bins + 1) >> 1;
  const uint32_t mask = (uint32_t)bins - 1u;
  const U lo = (U)J->lo;
  uint32_t* lb_base = J->lookback + pass * J->lb_stride;
  uint32_t* lb_mine = lb_base + lt * bins;

  constexpr int kPad = 16 / (int)sizeof(K);
  K* const a_keys = reinterpret_cast<K*>(smem);  // staging areas (16-byte aligned)
  K* const a_vals = a_keys + TILE + kPad;
  uint16_t* s_src = reinterpret_cast<uint16_t*>(a_vals + TILE + kPad);
  uint32_t* s_whist = reinterpret_cast<uint32_t*>(s_src + TILE);
  uint32_t* s_count = s_whist + kSortWarps * hb;  // contiguous with s_whist
  uint32_t* s_excl = s_count + bins;
  // a digit's first output position minus its first slot (positions are
  // 32-bit, as the digit histograms are: arithmetic modulo 2^32)
  uint32_t* s_gbase = s_excl + bins;
  K* s_cuts = reinterpret_cast<K*>(s_gbase + bins);
  uint16_t* s_tab = reinterpret_cast<uint16_t*>(s_cuts + bins);
  uint16_t* s_dig = s_tab + (kRouteBuckets + 8);  // u16 slots; u8 when bins <= 256
  uint8_t* s_dig8 = reinterpret_cast<uint8_t*>(s_dig);
  // slot digits kept, except beyond 512 batches with sized regions: there the
  // scatter searches the cut table again (their 2 bytes a row, beside the
  // regions' ends, would cost the multiprocessor a CTA)
  const bool keep_dig = bins <= 512 || J->route_end == nullptr;
  uint32_t* s_rend =  // end of each batch's region (route passes with sized regions)
      MODE == kModeCuts
          ? reinterpret_cast<uint32_t*>(s_dig8 + (bins <= 256 ? 1 : keep_dig ? 2 : 0) * TILE)
          : s_gbase + bins;
  const bool dig8 = bins <= 256;
  constexpr bool route = MODE == kModeCuts;  // digits from the cut table, kept per slot
  constexpr bool radix = MODE == kModeRadix;
  const K c_lo = (K)lo, c_hi = (K)J->route_hi;  // clamp of a radix route
  // sort digits within the low 32 bits of key - lo: 32-bit arithmetic
  const bool narrow = shift + nbits <= 32;
  const uint32_t lo32 = (uint32_t)lo;

  // 1. tile -> shared memory (asynchronous), counters zeroed meanwhile
  const K* s_keys = copy_rows_async<K, TILE>(a_keys, J->src_k[pass] + row0, nvalid);
  const K* s_vals = copy_rows_async<K, TILE>(a_vals, J->src_v[pass] + row0, nvalid);
  asm volatile("cp.async.commit_group;" ::: "memory");
  const bool guard = MODE != kModeSort && J->route_end != nullptr;
  if (route) {
    for (int i = tid; i < bins; i += kSortThreads) s_cuts[i] = J->cuts[i];
    for (int i = tid; i <= kRouteBuckets; i += kSortThreads) s_tab[i] = J->route_tab[i];
  }
  if (guard)
    for (int i = tid; i < bins; i += kSortThreads) s_rend[i] = J->route_end[i];
  for (int i = tid; i < kSortWarps * hb + bins; i += kSortThreads) s_whist[i] = 0u;
  // lane-mask tables of the ranking (one word per value of the digit's low
  // 7 bits), in the slot-index array, which is not live before step 4
  const int mwords = bins < 128 ? bins : 128;
  const bool rank_or = kSortWarps * mwords * 4 <= TILE * 2;
  if (rank_or)
    for (int i = tid; i < kSortWarps * mwords; i += kSortThreads)
      reinterpret_cast<uint32_t*>(s_src)[i] = 0u;
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();

  // 2. digits (low 16 bits of dr; the rank goes to the high 16 bits later)
  const int wbase = warp * 32 * ITEMS;
  uint32_t dr[ITEMS];
  if (route) {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const K k = s_keys[wbase + i * 32 + lane];  // padding rows: unused values
      dr[i] = route_idx<K>(k, lo, s_cuts, s_tab, J->route_steps, J->route_shift);
    }
  } else if (radix) {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const K k = s_keys[wbase + i * 32 + lane];
      const K c = k < c_lo ? c_lo : (c_hi < k ? c_hi : k);
      dr[i] = narrow ? (((uint32_t)c - lo32) >> shift) & mask : digit_of<K>(c, lo, shift, mask);
    }
  } else if (narrow) {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
      dr[i] = (((uint32_t)s_keys[wbase + i * 32 + lane] - lo32) >> shift) & mask;
  } else {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
      dr[i] = digit_of<K>(s_keys[wbase + i * 32 + lane], lo, shift, mask);
  }
#pragma unroll
  for (int i = 0; i < ITEMS; ++i)
    if (wbase + i * 32 + lane < nvalid) atomicAdd(&s_count[dr[i]], 1u);
  __syncthreads();
  for (int d = tid; d < bins; d += kSortThreads)
    st_volatile_u32(lb_mine + d, (lt == 0 ? kFlagInc : kFlagAgg) | s_count[d]);

  // 3. stable rank inside the warp: lane-mask tables when they fit (tiles of
  //    at least 3072 rows), else one ballot per digit bit (digit width fixed
  //    at compile time so that the ballots of several items interleave)
  {
    uint32_t* wh = s_whist + warp * hb;
    const int nv = nvalid - wbase;  // valid rows of this warp (may be <= 0)
    uint32_t* wm = reinterpret_cast<uint32_t*>(s_src) + warp * mwords;
    if (rank_or)
      switch (nbits) {
        case 8: rank_items_or<1, ITEMS>(dr, nv, wh, wm); break;
        case 9: rank_items_or<2, ITEMS>(dr, nv, wh, wm); break;
        case 10: rank_items_or<3, ITEMS>(dr, nv, wh, wm); break;
        default: rank_items_or<0, ITEMS>(dr, nv, wh, wm); break;
      }
    else
      switch (nbits) {
        case 1: rank_items<1, ITEMS>(dr, nv, wh); break;
        case 2: rank_items<2, ITEMS>(dr, nv, wh); break;
        case 3: rank_items<3, ITEMS>(dr, nv, wh); break;
        case 4: rank_items<4, ITEMS>(dr, nv, wh); break;
        case 5: rank_items<5, ITEMS>(dr, nv, wh); break;
        case 6: rank_items<6, ITEMS>(dr, nv, wh); break;
        case 7: rank_items<7, ITEMS>(dr, nv, wh); break;
        case 8: rank_items<8, ITEMS>(dr, nv, wh); break;
        case 9: rank_items<9, ITEMS>(dr, nv, wh); break;
        default: rank_items<10, ITEMS>(dr, nv, wh); break;
      }
  }
  __syncthreads();

  // per pair of digits: exclusive prefix over the warps (16-bit halves; the
  // tile's totals are already in s_count)
  for (int p = tid; p < hb; p += kSortThreads) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = s_whist[w * hb + p];
      s_whist[w * hb + p] = run;
      run += c;
    }
  }
  sort_block_excl_scan(s_count, s_excl, bins, s_warp);  // its barriers order the loop above

  // 4. first look-back window in flight while the slots are recorded
  constexpr int kDPer = (kMaxBins + kSortThreads - 1) / kSortThreads;
  uint32_t win[kLookWindow];
#pragma unroll
  for (int w = 0; w < kLookWindow; ++w)
    win[w] = (tid < bins && lt - 1 - w >= 0) ? ld_volatile_u32(lb_base + (lt - 1 - w) * bins + tid)
                                             : kFlagInc;
  {
    const uint32_t* wx = s_whist + warp * hb;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int r = wbase + i * 32 + lane;
      if (r < nvalid) {
        const uint32_t d = dr[i] & 0xFFFFu;
        const uint32_t wpre = (wx[d >> 1] >> ((d & 1u) * 16u)) & 0xFFFFu;
        const uint32_t pos = s_excl[d] + wpre + (dr[i] >> 16);
        s_src[pos] = (uint16_t)r;
        if (route) {
          if (dig8)
            s_dig8[pos] = (uint8_t)d;
          else if (keep_dig)
            s_dig[pos] = (uint16_t)d;
        }
      }
    }
  }
  const uint32_t* hist = J->hist + pass * J->hist_stride;
#pragma unroll
  for (int e = 0; e < kDPer; ++e) {
    const int d = tid + e * kSortThreads;
    if (d >= bins) break;
    uint32_t prefix = 0;
    if (lt > 0) {
      int64_t k = lt - 1;  // newest predecessor not yet summed
      bool done = false;
      if (e == 0) k -= lookback_consume<kLookWindow>(win, prefix, done);
      int spins = 0;
      while (!done) {
        uint32_t v[kLookWide];
#pragma unroll
        for (int w = 0; w < kLookWide; ++w)
          v[w] = (k - w >= 0) ? ld_volatile_u32(lb_base + (k - w) * bins + d) : kFlagInc;
        const int used = lookback_consume<kLookWide>(v, prefix, done);
        k -= used;
        if (used == 0) {
          if (++spins > kSpinLimit) {
            atomicExch(err, (int)TJ_ERR_TIMEOUT);
            break;
          }
          __nanosleep(32);
        }
      }
      st_volatile_u32(lb_mine + d, kFlagInc | ((prefix + s_count[d]) & kValMask));
    }
    s_gbase[d] = hist[d] + prefix - s_excl[d];
  }
  __syncthreads();

  // 5. slots in order -> global
  K* __restrict__ dst_k = J->dst_k[pass];
  K* __restrict__ dst_v = J->dst_v[pass];
  if (route) {
    if (guard) {
      // batch regions sized in advance: a row past its region's end is
      // dropped and reported (the caller then routes again with exact sizes)
      bool over = false;
#pragma unroll
      for (int it = 0; it < ITEMS; ++it) {
        const int q = tid + it * kSortThreads;
        if (q < nvalid) {
          const int r = s_src[q];
          const uint32_t d = dig8       ? (uint32_t)s_dig8[q]
                             : keep_dig ? (uint32_t)s_dig[q]
                                        : route_idx<K>(s_keys[r], lo, s_cuts, s_tab,
                                                       J->route_steps, J->route_shift);
          const uint32_t g = s_gbase[d] + (uint32_t)q;
          const bool in = g < s_rend[d];
          over |= !in;
          if (in) {
            dst_k[g] = s_keys[r];
            dst_v[g] = s_vals[r];
          }
        }
      }
      if (over) atomicCAS(err, 0, (int)TJ_ERR_CAPACITY);
      return;
    }
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const int q = tid + it * kSortThreads;
      if (q < nvalid) {
        const int r = s_src[q];
        const uint32_t d = dig8       ? (uint32_t)s_dig8[q]
                           : keep_dig ? (uint32_t)s_dig[q]
                                      : route_idx<K>(s_keys[r], lo, s_cuts, s_tab,
                                                     J->route_steps, J->route_shift);
        const uint32_t g = s_gbase[d] + (uint32_t)q;
        dst_k[g] = s_keys[r];
        dst_v[g] = s_vals[r];
      }
    }
    return;
  }
  if (radix) {
    // digit recomputed from the key (cheaper than keeping it per slot)
    bool over = false;
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const int q = tid + it * kSortThreads;
      if (q < nvalid) {
        const int r = s_src[q];
        const K k = s_keys[r];
        const K c = k < c_lo ? c_lo : (c_hi < k ? c_hi : k);
        const uint32_t d =
            narrow ? (((uint32_t)c - lo32) >> shift) & mask : digit_of<K>(c, lo, shift, mask);
        const uint32_t g = s_gbase[d] + (uint32_t)q;
        const bool in = !guard || g < s_rend[d];
        over |= !in;
        if (in) {
          dst_k[g] = k;
          dst_v[g] = s_vals[r];
        }
      }
    }
    if (over) atomicCAS(err, 0, (int)TJ_ERR_CAPACITY);
    return;
  }
  if (narrow) {
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const int q = tid + it * kSortThreads;
      if (q < nvalid) {
        const int r = s_src[q];
        const K k = s_keys[r];
        const uint32_t d = (((uint32_t)k - lo32) >> shift) & mask;
        const uint32_t g = s_gbase[d] + (uint32_t)q;
        dst_k[g] = k;
        dst_v[g] = s_vals[r];
      }
    }
  } else {
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const int q = tid + it * kSortThreads;
      if (q < nvalid) {
        const int r = s_src[q];
        const K k = s_keys[r];
        const uint32_t d = digit_of<K>(k, lo, shift, mask);
        const uint32_t g = s_gbase[d] + (uint32_t)q;
        dst_k[g] = k;
        dst_v[g] = s_vals[r];
      }
    }
  }
}

// next[d] = base[d] + inclusive count of digit d over one route launch's tiles
__global__ void k_route_chain(const uint32_t* __restrict__ base,
                              const uint32_t* __restrict__ lookback, int64_t last_tile, int bins,
                              uint32_t* __restrict__ next) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= bins) return;
  next[d] = base[d] + (lookback[last_tile * bins + d] & kValMask);
}

cudaError_t launch_route_chain(const uint32_t* base, const uint32_t* lookback, int64_t last_tile,
                               int bins, uint32_t* next, cudaStream_t st) {
  k_route_chain<<<(bins + kThreads - 1) / kThreads, kThreads, 0, st>>>(base, lookback, last_tile,
                                                                       bins, next);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename K>
cudaError_t launch_stats(const RadixJob<K>* d_jobs, int num_jobs, int64_t total_tiles,
                         KeyStats* d_stats, cudaStream_t st, int tile) {
  if (total_tiles <= 0) return cudaSuccess;
  const int64_t grid = total_tiles < 152 * 8 ? total_tiles : 152 * 8;
  k_stats<K><<<(unsigned)grid, kThreads, 0, st>>>(d_jobs, num_jobs, total_tiles, d_stats, tile);
  return cudaGetLastError();
}

template <typename K>
cudaError_t launch_histogram(const RadixJob<K>* d_jobs, int num_jobs, int64_t total_tiles,
                             cudaStream_t st, const int32_t* d_tile_job, int tile) {
  if (total_tiles <= 0) return cudaSuccess;
  const int64_t grid = total_tiles < 152 * 6 ? total_tiles : 152 * 6;
  k_histogram<K><<<(unsigned)grid, kThreads, 0, st>>>(d_jobs, num_jobs, total_tiles, d_tile_job,
                                                      tile);
  return cudaGetLastError();
}

template <typename K>
__global__ void k_fill_tile_job(const RadixJob<K>* __restrict__ jobs, int32_t* __restrict__ map,
                                int tile) {
  const int j = blockIdx.x;
  const int64_t t0 = jobs[j].tile0;
  const int64_t nt = (jobs[j].n + tile - 1) / tile;
  for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) map[t0 + t] = j;
}

template <typename K>
cudaError_t launch_fill_tile_job(const RadixJob<K>* d_jobs, int num_jobs, int32_t* d_map,
                                 cudaStream_t st, int tile) {
  if (num_jobs <= 0) return cudaSuccess;
  k_fill_tile_job<K><<<num_jobs, 128, 0, st>>>(d_jobs, d_map, tile);
  return cudaGetLastError();
}

template <typename K>
cudaError_t launch_digit_scan(const RadixJob<K>* d_jobs, int num_jobs, int passes,
                              cudaStream_t st) {
  if (passes <= 0 || num_jobs <= 0) return cudaSuccess;
  const int64_t warps = (int64_t)num_jobs * passes;
  const int64_t grid = (warps * 32 + kThreads - 1) / kThreads;
  k_digit_scan<K><<<(unsigned)grid, kThreads, 0, st>>>(d_jobs, num_jobs, passes);
  return cudaGetLastError();
}

template <typename K, int MODE>
cudaError_t launch_onesweep_t(const RadixJob<K>* d_jobs, int num_jobs, int64_t total_tiles,
                              int pass, int max_bits, uint32_t* d_tile_counter, int* d_err,
                              cudaStream_t st, const int32_t* d_tile_job, int items, bool guard) {
  if (items == 4) {
    const size_t smem = onesweep_smem_bytes<K>(1 << max_bits, MODE, kSortThreads * 4, guard);
    k_onesweep<K, 4, MODE><<<(unsigned)total_tiles, kSortThreads, smem, st>>>(
        d_jobs, num_jobs, total_tiles, pass, d_tile_counter, d_err, d_tile_job);
  } else if (items == kItemsRoute && kItemsRoute != kItems && kItemsRoute != kItemsWide) {
    if constexpr (MODE == kModeCuts) {  // route passes by the cut table only
      const size_t smem = onesweep_smem_bytes<K>(1 << max_bits, MODE, kTileRoute, guard);
      k_onesweep<K, kItemsRoute, MODE><<<(unsigned)total_tiles, kSortThreads, smem, st>>>(
          d_jobs, num_jobs, total_tiles, pass, d_tile_counter, d_err, d_tile_job);
    } else {
      return cudaErrorInvalidValue;
    }
  } else if (items == kItemsWide) {
    const size_t smem = onesweep_smem_bytes<K>(1 << max_bits, MODE, kTileWide, guard);
    k_onesweep<K, kItemsWide, MODE><<<(unsigned)total_tiles, kSortThreads, smem, st>>>(
        d_jobs, num_jobs, total_tiles, pass, d_tile_counter, d_err, d_tile_job);
  } else {
    const size_t smem = onesweep_smem_bytes<K>(1 << max_bits, MODE, kTile, guard);
    k_onesweep<K, kItems, MODE><<<(unsigned)total_tiles, kSortThreads, smem, st>>>(
        d_jobs, num_jobs, total_tiles, pass, d_tile_counter, d_err, d_tile_job);
  }
  return cudaGetLastError();
}

template <typename K>
cudaError_t launch_onesweep(const RadixJob<K>* d_jobs, int num_jobs, int64_t total_tiles,
                            int pass, int max_bits, int mode, uint32_t* d_tile_counter,
                            int* d_err, cudaStream_t st, const int32_t* d_tile_job, int items,
                            bool guard) {
  if (total_tiles <= 0) return cudaSuccess;
  if (mode == kModeCuts)
    return launch_onesweep_t<K, kModeCuts>(d_jobs, num_jobs, total_tiles, pass, max_bits,
                                           d_tile_counter, d_err, st, d_tile_job, items, guard);
  if (mode == kModeRadix)
    return launch_onesweep_t<K, kModeRadix>(d_jobs, num_jobs, total_tiles, pass, max_bits,
                                            d_tile_counter, d_err, st, d_tile_job, items, guard);
  return launch_onesweep_t<K, kModeSort>(d_jobs, num_jobs, total_tiles, pass, max_bits,
                                         d_tile_counter, d_err, st, d_tile_job, items, false);
}

// Largest dynamic shared memory of every onesweep instantiation (route passes
// with sized regions need the most).
template <typename K, int ITEMS, int MODE>
cudaError_t onesweep_attr() {
  // the larger of a launch with and without sized regions (a cut-table route
  // over more than 512 batches keeps slot digits only without them)
  const size_t a = onesweep_smem_bytes<K>(kMaxBins, MODE, kSortThreads * ITEMS, false);
  const size_t b = onesweep_smem_bytes<K>(kMaxBins, MODE, kSortThreads * ITEMS, MODE != kModeSort);
  return cudaFuncSetAttribute(k_onesweep<K, ITEMS, MODE>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(a > b ? a : b));
}

template <typename K>
cudaError_t onesweep_attrs() {
  cudaError_t e;
  if ((e = onesweep_attr<K, kItems, kModeSort>()) != cudaSuccess) return e;
  if ((e = onesweep_attr<K, kItems, kModeCuts>()) != cudaSuccess) return e;
  if ((e = onesweep_attr<K, kItems, kModeRadix>()) != cudaSuccess) return e;
  if ((e = onesweep_attr<K, kItemsWide, kModeSort>()) != cudaSuccess) return e;
  if ((e = onesweep_attr<K, kItemsWide, kModeCuts>()) != cudaSuccess) return e;
  if ((e = onesweep_attr<K, kItemsWide, kModeRadix>()) != cudaSuccess) return e;
  if ((e = onesweep_attr<K, 4, kModeSort>()) != cudaSuccess) return e;
  if ((e = onesweep_attr<K, 4, kModeCuts>()) != cudaSuccess) return e;
  if ((e = onesweep_attr<K, 4, kModeRadix>()) != cudaSuccess) return e;
  if (kItemsRoute != kItems && kItemsRoute != kItemsWide)
    if ((e = onesweep_attr<K, kItemsRoute, kModeCuts>()) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t radix_init_attributes() {
  cudaError_t e = onesweep_attrs<int32_t>();
  if (e != cudaSuccess) return e;
  return onesweep_attrs<int64_t>();
}

#define TJ_INSTANTIATE_RADIX(K)                                                                 \
  template cudaError_t launch_stats<K>(const RadixJob<K>*, int, int64_t, KeyStats*,             \
                                       cudaStream_t, int);                                      \
  template cudaError_t launch_histogram<K>(const RadixJob<K>*, int, int64_t, cudaStream_t,      \
                                           const int32_t*, int);                                \
  template cudaError_t launch_fill_tile_job<K>(const RadixJob<K>*, int, int32_t*, cudaStream_t, \
                                               int);                                            \
  template cudaError_t launch_digit_scan<K>(const RadixJob<K>*, int, int, cudaStream_t);        \
  template cudaError_t launch_onesweep<K>(const RadixJob<K>*, int, int64_t, int, int, int,     \
                                          uint32_t*, int*, cudaStream_t, const int32_t*, int,   \
                                          bool);
TJ_INSTANTIATE_RADIX(int32_t)
TJ_INSTANTIATE_RADIX(int64_t)

}  // namespace tj
