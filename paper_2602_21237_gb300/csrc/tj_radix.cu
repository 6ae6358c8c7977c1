// LSD radix machinery for the tensor-path sort (paper Sec. 4.2: the sort is a
// relocation of rows along the key axis, digit by digit) on sm_103a.
//
//   k_stats      : min / max of the keys of every array (one read of the keys);
//                  the planner turns them into (lo, significant bits).
//   k_histogram  : the counts of every digit of every pass, in one read of the
//                  keys (per-CTA shared-memory histograms merged into global).
//   k_digit_scan : exclusive scan of each pass's digit counts (digit bases).
//   k_onesweep   : one digit pass: a tile of 4096 rows is ranked stably inside
//                  the CTA (warp __match_any_sync groups + per-warp counters),
//                  its per-digit counts are published to a decoupled look-back
//                  chain, and the rows are scattered through shared memory so
//                  that each digit's run is written contiguously.
//
// Every kernel takes an array of jobs so that one launch serves any number of
// arrays (both sides of a join, or thousands of joins of a batch).
#include "tj_internal.cuh"

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

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
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

// Number of cut keys <= key in a sorted table padded to kMaxCuts entries with
// the key type's maximum (branch-free binary search; pads only count for the
// maximum key and are clipped by ncuts).
template <typename K>
__device__ __forceinline__ uint32_t route_of(K key, const K* s_cuts, int ncuts) {
  int pos = 0;
#pragma unroll
  for (int step = kMaxCuts / 2; step >= 1; step >>= 1)
    if (s_cuts[pos + step - 1] <= key) pos += step;
  return (uint32_t)min(pos, ncuts);
}

// Route through the radix index: the cuts <= key are all cuts before the key's
// bucket plus those of its bucket that are <= key (a short binary search).
template <typename K>
__device__ __forceinline__ uint32_t route_idx(K key, typename UnsignedOf<K>::type lo,
                                              const K* s_cuts, const uint16_t* s_tab) {
  using U = typename UnsignedOf<K>::type;
  const unsigned long long x = (unsigned long long)(U)((U)key - lo);
  const int nb = 64 - __clzll(x);  // significant bits of x
  const uint32_t b = nb < 6 ? (uint32_t)x : (uint32_t)((nb << 5) | ((x >> (nb - 6)) & 31ull));
  int a = s_tab[b], e = s_tab[b + 1];
  while (a < e) {
    const int mid = (a + e) >> 1;
    if (s_cuts[mid] <= key)
      a = mid + 1;
    else
      e = mid;
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
  for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    const int j = find_job(jobs, num_jobs, t);
    const K* __restrict__ keys = jobs[j].keys;
    const int64_t row0 = (t - jobs[j].tile0) * tile;
    const int64_t row1 = min(jobs[j].n, row0 + tile);
    unsigned long long mn = ~0ull, mx = 0ull;
    for (int64_t r = row0 + threadIdx.x; r < row1; r += kThreads) {
      const unsigned long long u = order_u(keys[r]);
      mn = u < mn ? u : mn;
      mx = u > mx ? u : mx;
    }
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
      atomicMin(&stats[j].min_u, mn);
      atomicMin(&stats[j].max_u, ~mx);  // stored inverted so both fields use atomicMin
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// K2: digit histograms of every pass in one read of the keys
// ---------------------------------------------------------------------------
// passes x 2^digit_bits never exceeds this (64-bit keys: 8 x 2^8 or 7 x 2^9;
// 32-bit keys: <= 4 x 2^8 or 3 x 2^10; a route pass: 1 x 2^10)
constexpr int kHistWords = 4096;

template <typename K>
__global__ void __launch_bounds__(kThreads) k_histogram(const RadixJob<K>* __restrict__ jobs,
                                                        int num_jobs, int64_t total_tiles,
                                                        const int32_t* __restrict__ tile_job,
                                                        int tile) {
  using U = typename UnsignedOf<K>::type;
  __shared__ uint32_t s_h[kHistWords];
  __shared__ int s_shift[kMaxPasses];
  __shared__ uint32_t s_mask[kMaxPasses];
  __shared__ K s_cuts[kMaxCuts];
  __shared__ uint16_t s_tab[kRouteBuckets + 1];
  int cur = -1, passes = 0, ncuts = -1, hs = 0;
  U lo = 0;
  auto flush = [&](int job) {
    __syncthreads();
    for (int p = 0; p < passes; ++p)
      for (int d = threadIdx.x; d <= (int)s_mask[p]; d += kThreads) {
        const uint32_t c = s_h[p * hs + d];
        if (c) atomicAdd(&jobs[job].hist[p * jobs[job].hist_stride + d], c);
      }
  };
  // grid-stride over tiles: one flush per job a CTA touched
  for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    const int j = tile_job ? tile_job[t] : find_job(jobs, num_jobs, t);
    if (j != cur) {
      if (cur >= 0) flush(cur);
      __syncthreads();
      cur = j;
      passes = jobs[j].passes;
      lo = (U)jobs[j].lo;
      ncuts = jobs[j].cuts ? jobs[j].ncuts : -1;
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
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = threadIdx.x + u * kThreads;
      if (r < row1) {
        if (ncuts >= 0) {
          atomicAdd(&s_h[route_idx<K>(kv[u], lo, s_cuts, s_tab)], 1u);
        } else {
          const U x = (U)kv[u] - lo;
          for (int p = 0; p < passes; ++p)
            atomicAdd(&s_h[p * hs + ((uint32_t)(x >> s_shift[p]) & s_mask[p])], 1u);
        }
      }
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
// Shared memory (bins = 2^bits of this pass, set at launch):
//   keys[kTile] K | ids[kTile] K | warp counters[kSortWarps][bins] u32 |
//   tile count[bins] u32 | tile exclusive[bins] u32 | global base[bins] i64
//   [cut keys[kMaxCuts] K, when the pass routes by a cut table]
//   [cut keys[bins] K, radix index[kRouteBuckets + 1] u16, when routing: a
//    route pass has at most bins - 1 cuts]
template <typename K>
__host__ __device__ constexpr size_t onesweep_smem_bytes(int bins, bool route, int tile = kTile) {
  return 2 * sizeof(K) * (size_t)tile + sizeof(uint32_t) * (size_t)(kSortWarps + 2) * bins +
         sizeof(long long) * (size_t)bins +
         (route ? sizeof(K) * (size_t)bins + sizeof(uint16_t) * (kRouteBuckets + 8) : 0);
}

// Exclusive scan of in[0, bins) by a CTA of kSortThreads (bins <= 2 * kSortThreads).
__device__ __forceinline__ void sort_block_excl_scan(const uint32_t* in, uint32_t* out, int bins,
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
  for (int w = 0; w < kSortWarps; ++w)
    if (w < warp) wpre += s_warp[w];
  const uint32_t excl = wpre + x - s;
  if (d0 < bins) out[d0] = excl;
  if (d0 + 1 < bins) out[d0 + 1] = excl + a;
  __syncthreads();
}

template <typename K, int ITEMS>
__global__ void __launch_bounds__(kSortThreads, TJ_SORT_MINB)
    k_onesweep(const RadixJob<K>* __restrict__ jobs, int num_jobs, int64_t total_tiles, int pass,
               uint32_t* __restrict__ tile_counter, int* __restrict__ err,
               const int32_t* __restrict__ tile_job) {
  using U = typename UnsignedOf<K>::type;
  constexpr int TILE = kSortThreads * ITEMS;
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
  const int bins = 1 << J->bits[pass];
  const uint32_t mask = (uint32_t)bins - 1u;
  const U lo = (U)J->lo;
  const K* __restrict__ src_k = J->src_k[pass] + row0;
  const K* __restrict__ src_v = J->src_v[pass] + row0;
  K* __restrict__ dst_k = J->dst_k[pass];
  K* __restrict__ dst_v = J->dst_v[pass];
  uint32_t* lb_base = J->lookback;
  uint32_t* lb_mine = lb_base + lt * bins;
  const uint32_t* hist = J->hist + pass * J->hist_stride;

  K* s_keys = reinterpret_cast<K*>(smem);
  K* s_vals = s_keys + TILE;
  uint32_t* s_whist = reinterpret_cast<uint32_t*>(s_vals + TILE);
  uint32_t* s_count = s_whist + kSortWarps * bins;
  uint32_t* s_excl = s_count + bins;
  long long* s_gbase = reinterpret_cast<long long*>(s_excl + bins);
  K* s_cuts = reinterpret_cast<K*>(s_gbase + bins);
  uint16_t* s_tab = reinterpret_cast<uint16_t*>(s_cuts + bins);
  const int ncuts = J->cuts ? J->ncuts : -1;
  if (ncuts >= 0) {
    for (int i = tid; i < bins; i += kSortThreads) s_cuts[i] = J->cuts[i];
    for (int i = tid; i <= kRouteBuckets; i += kSortThreads) s_tab[i] = J->route_tab[i];
  }
  // the digit of a row in this pass: a radix digit of key - lo, or its route
  auto dig = [&](K k) -> uint32_t {
    return ncuts >= 0 ? route_idx<K>(k, lo, s_cuts, s_tab)
                      : digit_of<K>(k, lo, shift, mask);
  };

  // Warp-striped rows: warp w owns rows [w*32*ITEMS, (w+1)*32*ITEMS) of the
  // tile; item i covers 32 consecutive rows, so ranks follow row order.
  const int wbase = warp * 32 * ITEMS;
  K key[ITEMS];
  K val[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int r = wbase + i * 32 + lane;
    key[i] = r < nvalid ? src_k[r] : K(0);
  }
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int r = wbase + i * 32 + lane;
    val[i] = r < nvalid ? src_v[r] : K(0);
  }
  for (int i = tid; i < kSortWarps * bins; i += kSortThreads) s_whist[i] = 0u;
  __syncthreads();

  // 1. peer groups of equal digits for every item (independent -> pipelined)
  uint32_t peers[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int r = wbase + i * 32 + lane;
    const uint32_t d = r < nvalid ? dig(key[i]) : 0xFFFFFFFFu;
    peers[i] = __match_any_sync(0xFFFFFFFFu, d);
  }
  // 2. one shared-memory atomicAdd per group, issued by the group's highest
  //    lane; it returns the warp's running count of that digit (items in order)
  uint32_t* wh = s_whist + warp * bins;
  uint32_t rk[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int r = wbase + i * 32 + lane;
    rk[i] = 0u;
    if (r < nvalid && (peers[i] >> lane) == 1u)
      rk[i] = atomicAdd(&wh[dig(key[i])], (uint32_t)__popc(peers[i]));
  }
  // 3. broadcast the group's base and add the rank inside the group
  const uint32_t ltm = lanemask_lt();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int leader = 31 - __clz(peers[i]);
    const uint32_t base = __shfl_sync(0xFFFFFFFFu, rk[i], leader);
    rk[i] = base + __popc(peers[i] & ltm);
  }
  __syncthreads();

  // per digit: exclusive prefix over warps and the tile's count; publish it
  for (int d = tid; d < bins; d += kSortThreads) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = s_whist[w * bins + d];
      s_whist[w * bins + d] = run;
      run += c;
    }
    s_count[d] = run;
    st_volatile_u32(lb_mine + d, (lt == 0 ? kFlagInc : kFlagAgg) | run);
  }
  __syncthreads();
  sort_block_excl_scan(s_count, s_excl, bins, s_warp);

  // Look-back and placement overlap: each digit thread first issues the loads
  // of its first look-back window, then every thread places its rows at their
  // tile-sorted position in shared memory, then the digit threads finish the
  // decoupled look-back (summing predecessors' counts of their digit until an
  // inclusive prefix, kLookWindow words per round trip; bounded wait, on
  // timeout report and go on).
  constexpr int kDPer = (kMaxBins + kSortThreads - 1) / kSortThreads;
  uint32_t win[kLookWindow];  // first window of this thread's first digit
#pragma unroll
  for (int w = 0; w < kLookWindow; ++w)
    win[w] = (tid < bins && lt - 1 - w >= 0) ? ld_volatile_u32(lb_base + (lt - 1 - w) * bins + tid)
                                             : 0u;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int r = wbase + i * 32 + lane;
    if (r < nvalid) {
      const uint32_t d = dig(key[i]);
      const uint32_t pos = s_excl[d] + s_whist[warp * bins + d] + rk[i];
      s_keys[pos] = key[i];
      s_vals[pos] = val[i];
    }
  }
#pragma unroll
  for (int e = 0; e < kDPer; ++e) {
    const int d = tid + e * kSortThreads;
    if (d >= bins) break;
    uint32_t prefix = 0;
    if (lt > 0) {
      int64_t k = lt - 1;  // newest predecessor not yet summed
      int spins = 0;
      bool done = false;
      bool first = (e == 0);
      while (!done) {
        uint32_t v[kLookWindow];
#pragma unroll
        for (int w = 0; w < kLookWindow; ++w)
          v[w] = first ? win[w]
                       : ((k - w >= 0) ? ld_volatile_u32(lb_base + (k - w) * bins + d) : kFlagInc);
        if (first)
#pragma unroll
          for (int w = 0; w < kLookWindow; ++w)
            if (k - w < 0) v[w] = kFlagInc;
        first = false;
        int used = 0;
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < kLookWindow; ++w) {
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
        k -= used;
        if (done || k < 0) break;
        if (used == 0) {
          if (++spins > kSpinLimit) {
            atomicExch(err, (int)TJ_ERR_TIMEOUT);
            break;
          }
          __nanosleep(32);
        } else {
          spins = 0;
        }
      }
      st_volatile_u32(lb_mine + d, kFlagInc | ((prefix + s_count[d]) & kValMask));
    }
    s_gbase[d] = (long long)hist[d] + (long long)prefix - (long long)s_excl[d];
  }
  __syncthreads();

  // scatter: consecutive staged rows of one digit go to consecutive addresses
#pragma unroll 4
  for (int q = tid; q < nvalid; q += kSortThreads) {
    const K k = s_keys[q];
    const uint32_t d = dig(k);
    const long long g = s_gbase[d] + q;
    dst_k[g] = k;
    dst_v[g] = s_vals[q];
  }
}

// ---------------------------------------------------------------------------
// K4': persistent onesweep pass with TMA prefetch of the next tile
// ---------------------------------------------------------------------------
// One CTA per SM loops over tiles taken from the atomic tile counter.  While
// it ranks and scatters tile t from shared buffer b, the next tile's keys and
// ids are already being copied into buffer b ^ 1 by the tensor memory
// accelerator (cp.async.bulk, completion counted on an mbarrier), so HBM reads
// stay in flight for the whole tile instead of only at its start.  Tiles whose
// rows are not 16-byte aligned in global memory (a job starting at an odd
// offset, a ragged last tile) are copied by the threads instead.  A CTA takes
// tile ids in increasing order and finishes them in that order, so the tile a
// look-back waits on is always being processed (no deadlock).
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  uint64_t g;
  asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(g), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Bounded wait for a buffer's copy; false (and the error word set) on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err) {
  for (int i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 64) __nanosleep(32);
  }
  atomicExch(err, (int)TJ_ERR_TIMEOUT);
  return false;
}

// Shared memory: two tile buffers (keys | ids) | warp counters[kSortWarps][bins]
// | tile count[bins] | tile exclusive[bins] | global base[bins] | [cuts, index]
template <typename K>
__host__ __device__ constexpr size_t onesweep_pf_smem_bytes(int bins, bool route) {
  return 4 * sizeof(K) * (size_t)kTile + sizeof(uint32_t) * (size_t)(kSortWarps + 2) * bins +
         sizeof(long long) * (size_t)bins +
         (route ? sizeof(K) * (size_t)bins + sizeof(uint16_t) * (kRouteBuckets + 8) : 0);
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads, 1)
    k_onesweep_pf(const RadixJob<K>* __restrict__ jobs, int num_jobs, int64_t total_tiles,
                  int pass, int max_bins, uint32_t* __restrict__ tile_counter,
                  int* __restrict__ err, const int32_t* __restrict__ tile_job) {
  using U = typename UnsignedOf<K>::type;
  constexpr int TILE = kTile;
  extern __shared__ __align__(128) unsigned char smem[];
  K* s_buf = reinterpret_cast<K*>(smem);  // buffer b: keys at 2*b*TILE, ids at (2*b+1)*TILE
  uint32_t* s_whist = reinterpret_cast<uint32_t*>(s_buf + 4 * TILE);
  uint32_t* s_count = s_whist + kSortWarps * max_bins;
  uint32_t* s_excl = s_count + max_bins;
  long long* s_gbase = reinterpret_cast<long long*>(s_excl + max_bins);
  K* s_cuts = reinterpret_cast<K*>(s_gbase + max_bins);
  uint16_t* s_tab = reinterpret_cast<uint16_t*>(s_cuts + max_bins);
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ long long s_tile[2];
  __shared__ int s_mode[2];  // 0: nothing to do, 1: copied by TMA, 2: threads copy it
  __shared__ uint32_t s_warp[kSortWarps];
  __shared__ int s_route_job, s_stop;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t parity[2] = {0u, 0u};

  // thread 0 only: take the next tile id and start copying it into buffer b
  auto fetch = [&](int b) {
    const long long t = (long long)atomicAdd(tile_counter, 1u);
    int mode = 0;
    if (t < total_tiles) {
      const int j = tile_job ? tile_job[t] : find_job(jobs, num_jobs, t);
      const RadixJob<K>* J = jobs + j;
      if (pass < J->passes) {
        const int64_t row0 = (t - J->tile0) * TILE;
        const int nvalid = (int)min((int64_t)TILE, J->n - row0);
        const K* sk = J->src_k[pass] + row0;
        const K* sv = J->src_v[pass] + row0;
        const uint32_t bytes = (uint32_t)nvalid * (uint32_t)sizeof(K);
        mode = 2;
        if ((((uintptr_t)sk | (uintptr_t)sv) & 15u) == 0 && (bytes & 15u) == 0) {
          mode = 1;
          // the buffer's previous contents were written through the generic proxy
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_expect_tx(&s_bar[b], 2 * bytes);
          bulk_g2s(s_buf + 2 * b * TILE, sk, bytes, &s_bar[b]);
          bulk_g2s(s_buf + (2 * b + 1) * TILE, sv, bytes, &s_bar[b]);
        }
      }
    }
    s_tile[b] = t;
    s_mode[b] = mode;
  };

  if (tid == 0) {
    mbar_init(&s_bar[0]);
    mbar_init(&s_bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_route_job = -1;
    s_stop = 0;
    fetch(0);
  }
  __syncthreads();
  int b = 0;
  while (true) {
    const long long t = s_tile[b];
    const int mode = s_mode[b];
    if (t >= total_tiles || s_stop) break;
    if (tid == 0) fetch(b ^ 1);  // buffer b ^ 1 was released at the end of the last tile
    if (mode == 0) {
      __syncthreads();
      b ^= 1;
      continue;
    }
    const int j = tile_job ? tile_job[t] : find_job(jobs, num_jobs, t);
    const RadixJob<K>* J = jobs + j;
    const int64_t lt = t - J->tile0;
    const int64_t row0 = lt * TILE;
    const int nvalid = (int)min((int64_t)TILE, J->n - row0);
    const int shift = J->shift[pass];
    const int bins = 1 << J->bits[pass];
    const uint32_t mask = (uint32_t)bins - 1u;
    const U lo = (U)J->lo;
    K* __restrict__ dst_k = J->dst_k[pass];
    K* __restrict__ dst_v = J->dst_v[pass];
    uint32_t* lb_base = J->lookback;
    uint32_t* lb_mine = lb_base + lt * bins;
    const uint32_t* hist = J->hist + pass * J->hist_stride;
    const int ncuts = J->cuts ? J->ncuts : -1;
    K* bk = s_buf + 2 * b * TILE;
    K* bv = s_buf + (2 * b + 1) * TILE;
    const bool reload = ncuts >= 0 && s_route_job != j;
    auto dig = [&](K k) -> uint32_t {
      return ncuts >= 0 ? route_idx<K>(k, lo, s_cuts, s_tab) : digit_of<K>(k, lo, shift, mask);
    };

    if (mode == 1) {
      mbar_wait_bounded(&s_bar[b], parity[b], err);
      parity[b] ^= 1u;
    } else {
      const K* __restrict__ src_k = J->src_k[pass] + row0;
      const K* __restrict__ src_v = J->src_v[pass] + row0;
      for (int i = tid; i < nvalid; i += kSortThreads) {
        bk[i] = src_k[i];
        bv[i] = src_v[i];
      }
    }
    if (reload) {
      for (int i = tid; i < bins; i += kSortThreads) s_cuts[i] = J->cuts[i];
      for (int i = tid; i <= kRouteBuckets; i += kSortThreads) s_tab[i] = J->route_tab[i];
    }
    for (int i = tid; i < kSortWarps * bins; i += kSortThreads) s_whist[i] = 0u;
    __syncthreads();
    if (tid == 0 && reload) s_route_job = j;

    const int wbase = warp * 32 * kItems;
    K key[kItems];
    K val[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const int r = wbase + i * 32 + lane;
      key[i] = r < nvalid ? bk[r] : K(0);
      val[i] = r < nvalid ? bv[r] : K(0);
    }
    uint32_t peers[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const int r = wbase + i * 32 + lane;
      const uint32_t d = r < nvalid ? dig(key[i]) : 0xFFFFFFFFu;
      peers[i] = __match_any_sync(0xFFFFFFFFu, d);
    }
    uint32_t* wh = s_whist + warp * bins;
    uint32_t rk[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const int r = wbase + i * 32 + lane;
      rk[i] = 0u;
      if (r < nvalid && (peers[i] >> lane) == 1u)
        rk[i] = atomicAdd(&wh[dig(key[i])], (uint32_t)__popc(peers[i]));
    }
    const uint32_t ltm = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const int leader = 31 - __clz(peers[i]);
      const uint32_t base = __shfl_sync(0xFFFFFFFFu, rk[i], leader);
      rk[i] = base + __popc(peers[i] & ltm);
    }
    __syncthreads();

    for (int d = tid; d < bins; d += kSortThreads) {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t c = s_whist[w * bins + d];
        s_whist[w * bins + d] = run;
        run += c;
      }
      s_count[d] = run;
      st_volatile_u32(lb_mine + d, (lt == 0 ? kFlagInc : kFlagAgg) | run);
    }
    __syncthreads();
    sort_block_excl_scan(s_count, s_excl, bins, s_warp);

    // placement into the tile buffer (every row has been read into registers)
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const int r = wbase + i * 32 + lane;
      if (r < nvalid) {
        const uint32_t d = dig(key[i]);
        const uint32_t pos = s_excl[d] + s_whist[warp * bins + d] + rk[i];
        bk[pos] = key[i];
        bv[pos] = val[i];
      }
    }
    // decoupled look-back, kLookWindow predecessors per round trip, bounded
    for (int d = tid; d < bins; d += kSortThreads) {
      uint32_t prefix = 0;
      if (lt > 0) {
        int64_t k = lt - 1;
        int spins = 0;
        bool done = false;
        while (!done) {
          uint32_t v[kLookWindow];
#pragma unroll
          for (int w = 0; w < kLookWindow; ++w)
            v[w] = (k - w >= 0) ? ld_volatile_u32(lb_base + (k - w) * bins + d) : kFlagInc;
          int used = 0;
          uint32_t acc = 0;
#pragma unroll
          for (int w = 0; w < kLookWindow; ++w) {
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
          k -= used;
          if (done || k < 0) break;
          if (used == 0) {
            if (++spins > kSpinLimit) {
              atomicExch(err, (int)TJ_ERR_TIMEOUT);
              break;
            }
            __nanosleep(32);
          } else {
            spins = 0;
          }
        }
        st_volatile_u32(lb_mine + d, kFlagInc | ((prefix + s_count[d]) & kValMask));
      }
      s_gbase[d] = (long long)hist[d] + (long long)prefix - (long long)s_excl[d];
    }
    __syncthreads();

#pragma unroll 4
    for (int q = tid; q < nvalid; q += kSortThreads) {
      const K k = bk[q];
      const long long g = s_gbase[dig(k)] + q;
      dst_k[g] = k;
      dst_v[g] = bv[q];
    }
    if (tid == 0) s_stop = ld_volatile_u32(reinterpret_cast<const uint32_t*>(err)) != 0u;
    // order this tile's generic-proxy reads and writes of buffer b before the
    // bulk copy that will refill it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();  // buffer b is free again
    b ^= 1;
  }
  // a copy started for a tile this CTA will not process must land before exit
  if (tid == 0 && s_tile[b] < total_tiles && s_mode[b] == 1)
    mbar_wait_bounded(&s_bar[b], parity[b], err);
  __syncthreads();
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

template <typename K>
cudaError_t launch_onesweep(const RadixJob<K>* d_jobs, int num_jobs, int64_t total_tiles,
                            int pass, int max_bits, bool route, uint32_t* d_tile_counter,
                            int* d_err, cudaStream_t st, const int32_t* d_tile_job, int items) {
  if (total_tiles <= 0) return cudaSuccess;
#if TJ_ONESWEEP_PF
  if (items == kItems) {
    // persistent: one CTA per SM, each prefetching its next tile
    static int sms[256] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 256 && sms[dev] == 0) {
      e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
    }
    const int nsm = (dev >= 0 && dev < 256 && sms[dev] > 0) ? sms[dev] : 152;
    const int64_t grid = total_tiles < nsm ? total_tiles : nsm;
    const size_t smem = onesweep_pf_smem_bytes<K>(1 << max_bits, route);
    k_onesweep_pf<K><<<(unsigned)grid, kSortThreads, smem, st>>>(
        d_jobs, num_jobs, total_tiles, pass, 1 << max_bits, d_tile_counter, d_err, d_tile_job);
    return cudaGetLastError();
  }
#endif
  if (items == 4) {
    const size_t smem = onesweep_smem_bytes<K>(1 << max_bits, route, kSortThreads * 4);
    k_onesweep<K, 4><<<(unsigned)total_tiles, kSortThreads, smem, st>>>(
        d_jobs, num_jobs, total_tiles, pass, d_tile_counter, d_err, d_tile_job);
  } else {
    const size_t smem = onesweep_smem_bytes<K>(1 << max_bits, route);
    k_onesweep<K, kItems><<<(unsigned)total_tiles, kSortThreads, smem, st>>>(
        d_jobs, num_jobs, total_tiles, pass, d_tile_counter, d_err, d_tile_job);
  }
  return cudaGetLastError();
}

cudaError_t radix_init_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_onesweep<int32_t, kItems>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)onesweep_smem_bytes<int32_t>(kMaxBins, true));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_onesweep<int64_t, kItems>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)onesweep_smem_bytes<int64_t>(kMaxBins, true));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_onesweep_pf<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)onesweep_pf_smem_bytes<int32_t>(kMaxBins, true));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_onesweep_pf<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)onesweep_pf_smem_bytes<int64_t>(kMaxBins, true));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_onesweep<int32_t, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)onesweep_smem_bytes<int32_t>(kMaxBins, true, kSortThreads * 4));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_onesweep<int64_t, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)onesweep_smem_bytes<int64_t>(kMaxBins, true, kSortThreads * 4));
}

#define TJ_INSTANTIATE_RADIX(K)                                                                 \
  template cudaError_t launch_stats<K>(const RadixJob<K>*, int, int64_t, KeyStats*,             \
                                       cudaStream_t, int);                                      \
  template cudaError_t launch_histogram<K>(const RadixJob<K>*, int, int64_t, cudaStream_t,      \
                                           const int32_t*, int);                                \
  template cudaError_t launch_fill_tile_job<K>(const RadixJob<K>*, int, int32_t*, cudaStream_t, \
                                               int);                                            \
  template cudaError_t launch_digit_scan<K>(const RadixJob<K>*, int, int, cudaStream_t);        \
  template cudaError_t launch_onesweep<K>(const RadixJob<K>*, int, int64_t, int, int, bool,    \
                                          uint32_t*, int*, cudaStream_t, const int32_t*, int);
TJ_INSTANTIATE_RADIX(int32_t)
TJ_INSTANTIATE_RADIX(int64_t)

}  // namespace tj
