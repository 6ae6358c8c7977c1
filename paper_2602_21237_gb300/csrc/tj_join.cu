// Join of two key-sorted relations on their common key axis (paper Sec. 4.1)
// with a single final materialisation of (r_id, s_id) pairs (Sec. 3.1).
//
//   k_tile_ranges : for every tile of kJTile sorted S rows, the range [a, b)
//                   of sorted R rows whose keys lie between the tile's first
//                   and last key (two searches per tile), written with the
//                   tile's rows and job as one 64-byte descriptor;
//   k_join        : per S tile, fused count -> scan -> write:
//                     1. read the tile's descriptor, stage its S rows and its
//                        R range (in chunks of kRCap rows, up to 4) in shared
//                        memory with cp.async;
//                     2. build an open-addressing hash table of each chunk's
//                        distinct keys with shared-memory atomicCAS: slot ->
//                        (first, end) of the key's run of R rows;
//                     3. probe it once per S row -> match count, run start;
//                     4. a decoupled look-back over all tiles of all jobs gives
//                        the tile's first output index;
//                     5. write the pairs, ordered by key, S position, R
//                        position, if they fit the caller's capacity.
//                   Tiles whose R range exceeds the on-chip chunks (S sparse
//                   against R) search a strided sample of the range on chip,
//                   then one stride of R in global memory.
#include "tj_internal.cuh"

namespace tj {

template <typename Job>
__device__ __forceinline__ int find_job_j(const Job* jobs, int num_jobs, int64_t t) {
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

// multiplicative hashing onto the table's log2(kHTSlots) bits
constexpr int kHTBits = kHTSlots == 1024 ? 10 : kHTSlots == 2048 ? 11 : kHTSlots == 4096 ? 12 : 13;
static_assert((1 << kHTBits) == kHTSlots, "hash table slots: 2^10 .. 2^13");
__device__ __forceinline__ uint32_t ht_hash(int32_t k) {
  return ((uint32_t)k * 0x9E3779B9u) >> (32 - kHTBits);
}
__device__ __forceinline__ uint32_t ht_hash(int64_t k) {
  return (uint32_t)(((uint64_t)k * 0x9E3779B97F4A7C15ull) >> (64 - kHTBits));
}
static_assert(kRCap < 0xFFFF, "run bounds are packed in 16 bits");

constexpr uint32_t kHTEmpty = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t lanemask_lt_j() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_volatile_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---------------------------------------------------------------------------
// k_tile_ranges: one warp per S tile.  Lanes 0-15 find the first R row with
// key >= the tile's first key, lanes 16-31 the first R row with key > the
// tile's last key, each by a 16-ary search (16 probes per round trip); lane 0
// writes the tile's descriptor, so a join tile needs one load to start.
template <typename K>
__global__ void k_tile_ranges(const JoinJob<K>* __restrict__ jobs, int num_jobs,
                              int64_t total_tiles, JTile<K>* __restrict__ tiles,
                              const int32_t* __restrict__ tile_job) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (t >= total_tiles) return;  // whole warps leave together
  const int lane = threadIdx.x & 31, sub = lane & 15;
  const bool upper = lane >= 16;
  const uint32_t half = upper ? 0xFFFF0000u : 0x0000FFFFu;
  const int j = tile_job ? tile_job[t] : find_job_j(jobs, num_jobs, t);
  const JoinJob<K>* J = jobs + j;
  const int64_t row0 = (t - J->tile0) * kJTile;
  const int64_t row1 = min(J->ns, row0 + kJTile);
  const K key = upper ? J->sk[row1 - 1] : J->sk[row0];
  const K* __restrict__ r = J->rk;
  // invariant: every row before lo satisfies the predicate, none from hi on
  // (predicate: r[i] < key for the lower bound, r[i] <= key for the upper)
  int64_t lo = 0, hi = J->nr;
  while (true) {
    const int64_t len = hi - lo;
    if (__all_sync(0xFFFFFFFFu, len <= 16)) break;
    const int64_t step = (len + 15) / 16;
    const int64_t p = lo + sub * step;
    bool pred = false;
    if (len > 16 && p < hi) pred = upper ? !(key < r[p]) : (r[p] < key);
    const int c = __popc(__ballot_sync(0xFFFFFFFFu, pred) & half);
    if (len > 16) {
      // probes 0..c-1 satisfy the predicate, probe c (if any) does not
      const int64_t lo0 = lo;
      if (c > 0) lo = lo0 + (int64_t)(c - 1) * step + 1;
      if (c < 16) hi = min(hi, lo0 + (int64_t)c * step);
    }
  }
  const int64_t p = lo + sub;
  const bool pred = p < hi && (upper ? !(key < r[p]) : (r[p] < key));
  const int64_t res = lo + __popc(__ballot_sync(0xFFFFFFFFu, pred) & half);
  const int64_t b = __shfl_sync(0xFFFFFFFFu, res, 16);
  if (lane == 0) {
    JTile<K> d;
    d.sk = J->sk + row0;
    d.sv = J->sv + row0;
    d.rk = J->rk + res;
    d.rv = J->rv + res;
    d.lt = t - J->tile0;
    d.nrr = b - res;
    d.nv = (int32_t)(row1 - row0);
    d.j = j;
    d.pad = 0;
    tiles[t] = d;
  }
}

// ---------------------------------------------------------------------------
#ifndef TJ_JTHREADS
#define TJ_JTHREADS 512
#endif
#ifndef TJ_JMINB
#define TJ_JMINB 2
#endif
constexpr int kJThreads = TJ_JTHREADS;          // threads per join CTA
constexpr int kJWarps = kJThreads / 32;
constexpr int kJItems = kJTile / kJThreads;     // S rows per thread
static_assert(kJItems * kJThreads == kJTile, "join tile = threads x items");

// Shared memory: S keys | S ids (kJTile + kPad each) | R keys | R ids (kRCap +
// kPad each) | hash table[kHTSlots] u32.  Each staged array starts up to kPad
// elements into its area (its first element keeps the source's address modulo
// 16, so that all but a head and a tail move in 16-byte copies).  After the
// probe the many-matches write path (which reads ids from global memory)
// keeps per-row offsets (u64) and run starts (u32) from the start of it.
template <typename K>
__host__ __device__ constexpr int join_pad() {
  return 16 / (int)sizeof(K);
}
template <typename K>
constexpr size_t join_smem_bytes() {
  return sizeof(K) * (size_t)(2 * (kJTile + join_pad<K>()) + 2 * (kRCap + join_pad<K>())) +
         sizeof(uint32_t) * kHTSlots;
}
static_assert(sizeof(int32_t) * (2 * kJTile + 2 * kRCap) >=
                  (sizeof(uint64_t) + sizeof(uint32_t)) * kJTile,
              "offsets and run starts fit in the join's shared memory");

// Asynchronous global -> shared copy of n elements into dst (16-byte aligned,
// kPad elements of slack): returns where the copy starts, dst plus the
// source's misalignment, so both sides agree modulo 16; the head and tail
// elements around the 16-byte chunks are copied one by one.  Every thread of
// the CTA calls it.
template <typename K>
__device__ __forceinline__ K* join_copy_async(K* dst, const K* __restrict__ src, int n) {
  const uint32_t mis = (uint32_t)((uintptr_t)src & 15u);  // a multiple of sizeof(K)
  K* d = dst + mis / sizeof(K);
  const uint32_t sd = (uint32_t)__cvta_generic_to_shared(d);
  constexpr int kPer = 16 / (int)sizeof(K);
  const int head = min(n, mis ? (int)((16u - mis) / sizeof(K)) : 0);
  const int chunks = (n - head) / kPer;
  for (int i = threadIdx.x; i < head; i += kJThreads)
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sd + (uint32_t)(i * sizeof(K))),
                 "l"(src + i), "n"(sizeof(K))
                 : "memory");
  for (int c = threadIdx.x; c < chunks; c += kJThreads)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sd + (uint32_t)(head * sizeof(K)) +
                                                                   16u * c),
                 "l"(src + head + c * kPer)
                 : "memory");
  for (int i = head + chunks * kPer + threadIdx.x; i < n; i += kJThreads)
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sd + (uint32_t)(i * sizeof(K))),
                 "l"(src + i), "n"(sizeof(K))
                 : "memory");
  return d;
}

// One join tile: kJTile consecutive rows of sorted S against the range [a, b)
// of sorted R whose keys lie between the tile's first and last key.
//   1. S keys and ids and the first chunk of the R range go to shared memory
//      (cp.async); warp w owns S rows [w*32*kJItems, ...), item u = 32 rows;
//   2. per chunk of the R range (kRCap rows, at most kMaxChunks): an
//      open-addressing table of the chunk's distinct keys is built with
//      shared-memory atomicCAS (slot -> first and end of the key's run), and
//      every S row probes it -> match count, run start and the R id of the
//      first match; wider R ranges are searched through a strided sample
//      staged on chip, then within one stride in global memory;
//   3. the tile's total goes to the decoupled look-back chain over all tiles
//      (warp 0, 32 predecessors per round trip), which yields the tile's
//      first output index;
//   4. at most one match per row (a foreign-key join): each row's output index
//      comes from ballots over the warp and the warps' totals; otherwise the
//      tile's counts are scanned and each output index finds its S row.
// Output order: key, then S position, then R position.
template <typename K>
__global__ void __launch_bounds__(kJThreads, TJ_JMINB)
    k_join(int64_t total_tiles, const JTile<K>* __restrict__ tiles,
           uint64_t* __restrict__ lookback, uint32_t* __restrict__ tile_counter,
           K* __restrict__ out, int64_t capacity, const int64_t* __restrict__ out_base,
           int64_t* __restrict__ job_out, int64_t* __restrict__ total, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int kPad = join_pad<K>();
  K* const b_sk = reinterpret_cast<K*>(smem);  // staging areas (16-byte aligned)
  K* const b_sv = b_sk + kJTile + kPad;
  K* const b_rk = b_sv + kJTile + kPad;
  K* const b_rv = b_rk + kRCap + kPad;
  uint32_t* s_ht = reinterpret_cast<uint32_t*>(b_rv + kRCap + kPad);
  __shared__ uint64_t s_wsum[kJWarps];
  __shared__ uint64_t s_base;
  __shared__ uint32_t s_t;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_t = atomicAdd(tile_counter, 1u);
  __syncthreads();
  const int64_t t = s_t;
  if (t >= total_tiles) return;
  const JTile<K> T = tiles[t];
  const int j = T.j;
  const int64_t nrr = T.nrr;
  const int64_t lt = T.lt;
  const int nv = T.nv;
  const K* __restrict__ rk_g = T.rk;
  const K* __restrict__ rv_g = T.rv;
  const int64_t nchunks = (nrr + kRCap - 1) / kRCap;
  const bool onchip = nchunks <= kMaxChunks;

  // 1. stage S and the first R chunk
  const K* s_sk = join_copy_async<K>(b_sk, T.sk, nv);
  const K* s_sv = join_copy_async<K>(b_sv, T.sv, nv);
  K* s_rk = b_rk;  // the staged R chunk (where its copy starts)
  K* s_rv = b_rv;
  if (onchip && nchunks > 0) {
    const int nc0 = (int)min((int64_t)kRCap, nrr);
    s_rk = join_copy_async<K>(b_rk, rk_g, nc0);
    s_rv = join_copy_async<K>(b_rv, rv_g, nc0);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");

  // 2. probe
  const int wbase = warp * 32 * kJItems;
  uint32_t cnt[kJItems], start[kJItems];
#pragma unroll
  for (int u = 0; u < kJItems; ++u) cnt[u] = start[u] = 0u;
  if (onchip) {
    for (int64_t c = 0; c < nchunks; ++c) {
      const int c0 = (int)(c * kRCap);
      const int nc = (int)min((int64_t)kRCap, nrr - c0);
      if (c > 0) {
        __syncthreads();  // the previous chunk's probes are done
        s_rk = join_copy_async<K>(b_rk, rk_g + c0, nc);
        s_rv = join_copy_async<K>(b_rv, rv_g + c0, nc);
        asm volatile("cp.async.commit_group;" ::: "memory");
      }
      for (int i = tid; i < kHTSlots; i += kJThreads) s_ht[i] = kHTEmpty;
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
      // insert the first row of every run of equal keys; keys are distinct, so
      // an occupied slot is never this key and insertion needs no comparison
      for (int i = tid; i < nc; i += kJThreads) {
        if (i == 0 || s_rk[i] != s_rk[i - 1]) {
          uint32_t h = ht_hash(s_rk[i]);
          while (atomicCAS(&s_ht[h], kHTEmpty, (uint32_t)i | 0xFFFF0000u) != kHTEmpty)
            h = (h + 1) & (kHTSlots - 1);
        }
      }
      __syncthreads();
      // the last row of every run records the run's end
      for (int i = tid; i < nc; i += kJThreads) {
        if (i == nc - 1 || s_rk[i] != s_rk[i + 1]) {
          const K key = s_rk[i];
          uint32_t h = ht_hash(key);
          while (true) {
            const uint32_t w = s_ht[h];
            if (s_rk[w & 0xFFFFu] == key) {
              s_ht[h] = (w & 0xFFFFu) | ((uint32_t)(i + 1) << 16);
              break;
            }
            h = (h + 1) & (kHTSlots - 1);
          }
        }
      }
      __syncthreads();
      const K cf = s_rk[0], cl = s_rk[nc - 1];
#pragma unroll
      for (int u = 0; u < kJItems; ++u) {
        const int q = wbase + u * 32 + lane;
        if (q >= nv) continue;
        const K key = s_sk[q];
        if (key < cf || cl < key) continue;
        uint32_t h = ht_hash(key);
        while (true) {
          const uint32_t w = s_ht[h];
          if (w == kHTEmpty) break;
          const uint32_t f = w & 0xFFFFu;
          if (s_rk[f] == key) {
            if (cnt[u] == 0u) start[u] = (uint32_t)c0 + f;
            cnt[u] += (w >> 16) - f;
            break;
          }
          h = (h + 1) & (kHTSlots - 1);
        }
      }
    }
    if (nchunks == 0) asm volatile("cp.async.wait_all;" ::: "memory");
  } else {
    // Wide R range (S sparse against R): every stride-th R key goes to shared
    // memory; a row's bound is found among those samples on chip, then inside
    // one stride of R in global memory, all rows of a thread in lockstep
    // (independent loads in flight together).
    const int64_t stride = (nrr + kRCap - 1) / kRCap;
    const int m = (int)((nrr + stride - 1) / stride);
    for (int i = tid; i < m; i += kJThreads) s_rk[i] = rk_g[(int64_t)i * stride];
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    int steps = 0;  // halvings that empty a range of `stride` rows
    while (((int64_t)1 << steps) <= stride) ++steps;
    K key[kJItems];
#pragma unroll
    for (int u = 0; u < kJItems; ++u) {
      const int q = wbase + u * 32 + lane;
      key[u] = q < nv ? s_sk[q] : K(0);
    }
    // bound 0: first R row with key >= the row's key; 1: first with key >
    // (offsets into the range: nrr < 2^30)
    const int nr32 = (int)nrr;
    auto search = [&](int bound, int (&lo)[kJItems]) {
      int n[kJItems];
#pragma unroll
      for (int u = 0; u < kJItems; ++u) {
        // samples before a satisfy the predicate (sample < key, or <= key)
        int a = 0, c = m;
        while (a < c) {
          const int mid = (a + c) >> 1;
          const bool pr = bound ? !(key[u] < s_rk[mid]) : (s_rk[mid] < key[u]);
          a = pr ? mid + 1 : a;
          c = pr ? c : mid;
        }
        // rows up to sample a - 1 satisfy it, sample a (if any) does not
        lo[u] = a == 0 ? 0 : (int)((a - 1) * stride + 1);
        const int hi = a == m ? nr32 : (int)(a * stride);
        n[u] = hi - lo[u];
      }
      for (int it = 0; it < steps; ++it) {
#pragma unroll
        for (int u = 0; u < kJItems; ++u) {
          const int half = n[u] >> 1;
          const K r = rk_g[min(lo[u] + half, nr32 - 1)];  // in range even when n == 0
          const bool go = n[u] > 0 && (bound ? !(key[u] < r) : (r < key[u]));
          lo[u] = go ? lo[u] + half + 1 : lo[u];
          n[u] = go ? n[u] - half - 1 : half;
        }
      }
    };
    int lo[kJItems];
    search(0, lo);
    // a match and no equal key right after it: one match (the common case of
    // unique R keys); otherwise the upper bound is searched too
    uint32_t more = 0u;
#pragma unroll
    for (int u = 0; u < kJItems; ++u) {
      const bool valid = wbase + u * 32 + lane < nv;
      const K r0 = rk_g[min(lo[u], nr32 - 1)];
      const K r1 = rk_g[min(lo[u] + 1, nr32 - 1)];
      const bool e0 = valid && lo[u] < nr32 && r0 == key[u];
      const bool e1 = e0 && lo[u] + 1 < nr32 && r1 == key[u];
      start[u] = (uint32_t)lo[u];
      cnt[u] = e0 ? 1u : 0u;
      more |= (e1 ? 1u : 0u) << u;
    }
    if (__any_sync(0xFFFFFFFFu, more != 0u)) {
      int hi[kJItems];
      search(1, hi);
#pragma unroll
      for (int u = 0; u < kJItems; ++u)
        if ((more >> u) & 1u) cnt[u] = (uint32_t)(hi[u] - lo[u]);
    }
  }

  // 3. the tile's total, its warps' prefixes and the chained scan over tiles
  uint64_t mysum = 0;
  uint32_t mymax = 0;
#pragma unroll
  for (int u = 0; u < kJItems; ++u) {
    mysum += cnt[u];
    mymax = max(mymax, cnt[u]);
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) mysum += __shfl_xor_sync(0xFFFFFFFFu, mysum, o);
  if (lane == 0) s_wsum[warp] = mysum;
  const bool multi = __syncthreads_or(mymax > 1u) != 0;  // also publishes s_wsum
  uint64_t C = 0, wpre = 0;
#pragma unroll
  for (int w = 0; w < kJWarps; ++w) {
    const uint64_t x = s_wsum[w];
    if (w < warp) wpre += x;
    C += x;
  }
  // chained scan over all tiles by warp 0: each round trip reads the 32 newest
  // predecessors not yet summed (lane l: tile k - l), sums the run of ready
  // words up to the first inclusive one, and stops there
  if (warp == 0) {
    uint64_t* mine = lookback + t;
    uint64_t prefix = 0;
    if (t == 0) {
      if (lane == 0) st_volatile_u64(mine, kFlagInc64 | (C & kValMask64));
    } else {
      if (lane == 0) st_volatile_u64(mine, kFlagAgg64 | (C & kValMask64));
      int64_t k = t - 1;  // newest predecessor not yet summed
      int spins = 0;
      while (true) {
        const int64_t idx = k - lane;
        const uint64_t v = idx >= 0 ? ld_volatile_u64(lookback + idx) : kFlagInc64;
        const uint64_t f = v & ~kValMask64;
        const uint32_t notready = __ballot_sync(0xFFFFFFFFu, f == 0ull);
        const uint32_t inc = __ballot_sync(0xFFFFFFFFu, f == kFlagInc64);
        const int first_nr = notready ? __ffs(notready) - 1 : 32;
        const int first_inc = inc ? __ffs(inc) - 1 : 32;
        const int take = first_inc < first_nr ? first_inc + 1 : first_nr;  // lanes summed
        uint64_t x = lane < take ? (v & kValMask64) : 0ull;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
        prefix += x;
        if (first_inc < first_nr) break;
        k -= take;
        if (take == 0) {
          if (++spins > kSpinLimit) {
            if (lane == 0) atomicExch(err, (int)TJ_ERR_TIMEOUT);
            break;
          }
          __nanosleep(32);
        } else {
          spins = 0;
        }
      }
      if (lane == 0) st_volatile_u64(mine, kFlagInc64 | ((prefix + C) & kValMask64));
    }
    if (lane == 0) {
      s_base = prefix;
      if (lt == 0 && job_out) job_out[j] = (int64_t)prefix;
      // the end of this launch's output (absolute when the launch has a base)
      if (t == total_tiles - 1) *total = (int64_t)(prefix + C) + (out_base ? *out_base : 0);
    }
  }
  __syncthreads();
  // output index of this tile's first pair: the group's base (the partitioned
  // join writes several groups one after another) plus the chained prefix
  const uint64_t E = s_base + (out_base ? (uint64_t)*out_base : 0ull);
  if (E + C > (uint64_t)capacity) return;  // the host reports TJ_ERR_CAPACITY

  // 4. write
  if (!multi) {
    using P = typename PairOf<K>::type;
    const bool vec = (((uintptr_t)out) & (2 * sizeof(K) - 1)) == 0;
    const uint32_t ltm = lanemask_lt_j();
    // R rows of the chunk still in shared memory (the last one) are read
    // there, earlier ones from global memory
    const int64_t cres = onchip && nchunks > 0 ? (nchunks - 1) * kRCap : INT64_MAX;
    uint64_t off = E + wpre;
#pragma unroll
    for (int u = 0; u < kJItems; ++u) {
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, cnt[u] != 0u);
      if (cnt[u] != 0u) {
        const uint64_t o = off + __popc(m & ltm);
        const int64_t st0 = (int64_t)start[u];
        const K sid = s_sv[wbase + u * 32 + lane];
        const K rid = st0 >= cres ? s_rv[st0 - cres] : rv_g[st0];
        if (vec) {
          P pr;
          pr.x = rid;
          pr.y = sid;
          *reinterpret_cast<P*>(out + 2 * o) = pr;
        } else {
          out[2 * o] = rid;
          out[2 * o + 1] = sid;
        }
      }
      off += __popc(m);
    }
  } else {
    // many matches: per-row counts -> exclusive offsets, then each output
    // index finds its S row by binary search
    uint64_t* s_off = reinterpret_cast<uint64_t*>(smem);
    uint32_t* s_rs = reinterpret_cast<uint32_t*>(s_off + kJTile);
#pragma unroll
    for (int u = 0; u < kJItems; ++u) {
      const int q = wbase + u * 32 + lane;
      if (q < nv) {
        s_off[q] = cnt[u];
        s_rs[q] = start[u];
      }
    }
    __syncthreads();
    {
      constexpr int kPer = kJTile / kJThreads;
      uint64_t v[kPer];
      uint64_t sum = 0;
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int q = tid * kPer + i;
        v[i] = q < nv ? s_off[q] : 0ull;
        sum += v[i];
      }
      uint64_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
      }
      __syncthreads();  // every thread has read its counts
      if (lane == 31) s_wsum[warp] = x;
      __syncthreads();
      uint64_t pre = 0;
#pragma unroll
      for (int w = 0; w < kJWarps; ++w)
        if (w < warp) pre += s_wsum[w];
      uint64_t run = pre + x - sum;
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int q = tid * kPer + i;
        if (q < nv) s_off[q] = run;
        run += v[i];
      }
    }
    __syncthreads();
    const K* __restrict__ sv_g = T.sv;
    K* __restrict__ o = out + 2 * E;
    for (uint64_t x = tid; x < C; x += kJThreads) {
      int lo = 0, hi = nv - 1;  // last q with s_off[q] <= x
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= x)
          lo = mid;
        else
          hi = mid - 1;
      }
      const uint64_t r = s_rs[lo] + (x - s_off[lo]);
      o[2 * x] = rv_g[r];
      o[2 * x + 1] = sv_g[lo];
    }
  }
}

// ---------------------------------------------------------------------------
template <typename K>
cudaError_t launch_tile_ranges(const JoinJob<K>* d_jobs, int num_jobs, int64_t total_tiles,
                               JTile<K>* d_tiles, cudaStream_t st, const int32_t* d_tile_job) {
  if (total_tiles <= 0) return cudaSuccess;
  const int64_t grid = (total_tiles * 32 + kThreads - 1) / kThreads;
  k_tile_ranges<K><<<(unsigned)grid, kThreads, 0, st>>>(d_jobs, num_jobs, total_tiles, d_tiles,
                                                        d_tile_job);
  return cudaGetLastError();
}

// Tile -> job maps of one group of a partitioned join: blocks [0, nr) fill
// the radix map from the radix jobs, the rest the join map from the join jobs.
template <typename K>
__global__ void k_group_maps(const RadixJob<K>* __restrict__ rjobs, int nr,
                             int32_t* __restrict__ rmap, const JoinJob<K>* __restrict__ jjobs,
                             int32_t* __restrict__ jmap, int tile) {
  const int b = blockIdx.x;
  if (b < nr) {
    const int64_t t0 = rjobs[b].tile0;
    const int64_t nt = (rjobs[b].n + tile - 1) / tile;
    for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) rmap[t0 + t] = b;
  } else {
    const int j = b - nr;
    const int64_t t0 = jjobs[j].tile0;
    const int64_t nt = (jjobs[j].ns + kJTile - 1) / kJTile;
    for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) jmap[t0 + t] = j;
  }
}

template <typename K>
cudaError_t launch_group_maps(const RadixJob<K>* d_rjobs, int nr, int32_t* d_rmap,
                              const JoinJob<K>* d_jjobs, int nj, int32_t* d_jmap,
                              cudaStream_t st, int tile) {
  if (nr + nj <= 0) return cudaSuccess;
  k_group_maps<K><<<nr + nj, 256, 0, st>>>(d_rjobs, nr, d_rmap, d_jjobs, d_jmap, tile);
  return cudaGetLastError();
}

template <typename K>
__global__ void k_fill_join_tile_job(const JoinJob<K>* __restrict__ jobs,
                                     int32_t* __restrict__ map) {
  const int j = blockIdx.x;
  const int64_t t0 = jobs[j].tile0;
  const int64_t nt = (jobs[j].ns + kJTile - 1) / kJTile;
  for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) map[t0 + t] = j;
}

template <typename K>
cudaError_t launch_fill_join_tile_job(const JoinJob<K>* d_jobs, int num_jobs, int32_t* d_map,
                                      cudaStream_t st) {
  if (num_jobs <= 0) return cudaSuccess;
  k_fill_join_tile_job<K><<<num_jobs, 128, 0, st>>>(d_jobs, d_map);
  return cudaGetLastError();
}

template <typename K>
cudaError_t launch_join(int64_t total_tiles, const JTile<K>* d_tiles, uint64_t* d_lookback,
                        uint32_t* d_tile_counter, K* out, int64_t capacity,
                        const int64_t* d_out_base, int64_t* d_job_out, int64_t* d_total,
                        int* d_err, cudaStream_t st) {
  if (total_tiles <= 0) return cudaSuccess;
  const size_t smem = join_smem_bytes<K>();
  k_join<K><<<(unsigned)total_tiles, kJThreads, smem, st>>>(
      total_tiles, d_tiles, d_lookback, d_tile_counter, out, capacity, d_out_base, d_job_out,
      d_total, d_err);
  return cudaGetLastError();
}

// Jobs without join tiles (empty S, or skipped) take the first output index of
// the next job that has tiles, or the total; entry num_jobs is the total.
template <typename K>
__global__ void k_fix_job_out(const JoinJob<K>* __restrict__ jobs, int num_jobs,
                              int64_t total_tiles, int64_t* __restrict__ job_out,
                              const int64_t* __restrict__ total) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > num_jobs) return;
  if (j == num_jobs) {
    job_out[j] = total_tiles > 0 ? *total : 0;
    return;
  }
  const int64_t t0 = jobs[j].tile0;
  const bool has_tiles = jobs[j].ns > 0;
  if (has_tiles) return;
  if (t0 >= total_tiles) {
    job_out[j] = total_tiles > 0 ? *total : 0;
  } else {
    const int k = find_job_j(jobs, num_jobs, t0);
    job_out[j] = job_out[k];
  }
}

template <typename K>
cudaError_t launch_fix_job_out(const JoinJob<K>* d_jobs, int num_jobs, int64_t total_tiles,
                               int64_t* d_job_out, const int64_t* d_total, cudaStream_t st) {
  const int grid = (num_jobs + 1 + kThreads - 1) / kThreads;
  k_fix_job_out<K><<<grid, kThreads, 0, st>>>(d_jobs, num_jobs, total_tiles, d_job_out, d_total);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// k_cross: the pairs of single-key batches, streamed (one CTA per kXPairs
// consecutive pairs of a batch): pair p = i * nr + j of a batch is (R id j,
// S id i), so for nr = 1 (a foreign key's heavy value) a CTA reads 4096
// consecutive S ids and writes 4096 consecutive pairs.
template <typename K>
__global__ void __launch_bounds__(kXThreads)
    k_cross(const CrossJob<K>* __restrict__ jobs, int num_jobs, K* __restrict__ out,
            int64_t capacity, const int64_t* __restrict__ base_in, int64_t* __restrict__ base_out,
            int64_t run_pairs) {
  const int64_t b = blockIdx.x;
  int lo = 0, hi = num_jobs - 1;  // last job whose first CTA is <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].blk0 <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  const CrossJob<K> J = jobs[lo];
  const int64_t base = *base_in;
  if (b == 0 && threadIdx.x == 0) *base_out = base + run_pairs;
  const int64_t np = J.nr * J.ns;
  const int64_t o = base + J.off;
  if (o + np > capacity) return;  // the host reports TJ_ERR_CAPACITY
  const int64_t p0 = (b - J.blk0) * kXPairs;
  const int64_t p1 = min(np, p0 + kXPairs);
  using P = typename PairOf<K>::type;
  const bool vec = (((uintptr_t)out) & (2 * sizeof(K) - 1)) == 0;
  if (J.nr == 1) {
    const K r = J.rv[0];
    for (int64_t p = p0 + threadIdx.x; p < p1; p += kXThreads) {
      const K sid = J.sv[p];
      if (vec) {
        P v;
        v.x = r;
        v.y = sid;
        *reinterpret_cast<P*>(out + 2 * (o + p)) = v;
      } else {
        out[2 * (o + p)] = r;
        out[2 * (o + p) + 1] = sid;
      }
    }
  } else {
    for (int64_t p = p0 + threadIdx.x; p < p1; p += kXThreads) {
      const int64_t i = p / J.nr, j = p - i * J.nr;
      out[2 * (o + p)] = J.rv[j];
      out[2 * (o + p) + 1] = J.sv[i];
    }
  }
}

template <typename K>
cudaError_t launch_cross(const CrossJob<K>* d_jobs, int num_jobs, int64_t blocks, K* out,
                         int64_t capacity, const int64_t* d_base, int64_t* d_next,
                         int64_t run_pairs, cudaStream_t st) {
  if (num_jobs <= 0 || blocks <= 0) return cudaErrorInvalidValue;
  k_cross<K><<<(unsigned)blocks, kXThreads, 0, st>>>(d_jobs, num_jobs, out, capacity, d_base,
                                                     d_next, run_pairs);
  return cudaGetLastError();
}

cudaError_t join_init_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_join<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)join_smem_bytes<int32_t>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_join<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)join_smem_bytes<int64_t>());
}

#define TJ_INSTANTIATE_JOIN(K)                                                                  \
  template cudaError_t launch_tile_ranges<K>(const JoinJob<K>*, int, int64_t, JTile<K>*,        \
                                             cudaStream_t, const int32_t*);                     \
  template cudaError_t launch_fill_join_tile_job<K>(const JoinJob<K>*, int, int32_t*,            \
                                                    cudaStream_t);                              \
  template cudaError_t launch_join<K>(int64_t, const JTile<K>*, uint64_t*, uint32_t*, K*,        \
                                      int64_t, const int64_t*, int64_t*, int64_t*, int*,          \
                                      cudaStream_t);                                              \
  template cudaError_t launch_cross<K>(const CrossJob<K>*, int, int64_t, K*, int64_t,            \
                                       const int64_t*, int64_t*, int64_t, cudaStream_t);        \
  template cudaError_t launch_fix_job_out<K>(const JoinJob<K>*, int, int64_t, int64_t*,          \
                                             const int64_t*, cudaStream_t);                     \
  template cudaError_t launch_group_maps<K>(const RadixJob<K>*, int, int32_t*, const JoinJob<K>*, \
                                            int, int32_t*, cudaStream_t, int);
TJ_INSTANTIATE_JOIN(int32_t)
TJ_INSTANTIATE_JOIN(int64_t)

}  // namespace tj
