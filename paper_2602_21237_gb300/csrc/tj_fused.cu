// Partition-resident phase of the partitioned join (paper Sec. 4.1: align
// both relations on the common key axis; Sec. 3.1: materialise once; Sec. 6:
// every pass within the working memory).
//
// After the route pass has cut R and S into key-range batches and one MSD
// onesweep pass has cut each batch into sub-batches of kFKeys consecutive key
// values (S and R rows of a sub-batch contiguous, in input order), one CTA
// per tile of a sub-batch (at most kFCapS S rows, all of the sub-batch's R
// rows) finishes the join on chip:
//   1. count the R rows per 10-bit key offset (key - the sub-batch's first
//      key) and keep each key's R id in a table (keys with several R rows:
//      the R rows sorted stably by key offset in shared memory, two LSD
//      passes of 5-bit digits);
//   2. hold the S rows in registers, count them per key offset and rank each
//      stably among the warp's rows of its key (tj_warp.cuh);
//   3. per key offset: the S rows of earlier warps and the offset of the
//      key's first pair, Sum_{k' < k} |S_k'| |R_k'| (an exclusive scan);
//   4. a decoupled look-back over the items of the group (in key order) gives
//      the tile's first output index;
//   5. write every pair (r_id, s_id) once, straight to its place: key order,
//      then S position, then R position.
// A sub-batch with more than kFCapS S rows (skewed keys) is split into tiles
// processed by separate CTAs: k_fused_hist adds each tile's counts into the
// sub-batch's totals first, and inside k_fused_join a second decoupled
// look-back over per-key count vectors gives every tile the counts of the
// tiles before it, so a hot key's rows spread over many CTAs.
//
//   k_fused_info  : per batch, the number of items (tiles), of tiles and
//                   sub-batches that need the multi-tile counts, and the
//                   largest R sub-batch (the host checks it fits on chip);
//   k_fused_items : the item list of a group in key order;
//   k_fused_hist  : per-key totals of the multi-tile sub-batches;
//   k_fused_join  : the join of one item.
#include "tj_internal.cuh"
#include "tj_warp.cuh"

namespace tj {

namespace {

constexpr int kFWarps = kFThreads / 32;
constexpr int kFItemsS = kFCapS / kFThreads;  // S rows per thread (9)
static_assert(kFItemsS * kFThreads == kFCapS, "S tile = threads x rows per thread");
constexpr int kFItemsR = kFCapR / kFThreads;  // R rows per thread (4)
constexpr int kFDigit = kFKeyBits / 2;        // bits per in-smem sort pass (5)
constexpr int kFBins = 1 << kFDigit;          // 32
static_assert(kFDigit * 2 == kFKeyBits, "two in-smem passes cover the key offset");
static_assert(kFKeys == 2 * kFThreads, "two key offsets per thread in the scans");
static_assert(kFCapS <= 65536 && kFCapR <= 65536, "16-bit row indices");

__device__ __forceinline__ uint32_t ld_vol_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_vol_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.volatile.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_vol_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_vol_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Rows of sub-batch d of a job: its R and S row ranges (exclusive bases of
// the MSD histogram; a job without an MSD pass is one sub-batch).
template <typename K>
struct Sub {
  int64_t r0, nr, s0, ns;
};
template <typename K>
__device__ __forceinline__ Sub<K> sub_of(const FusedJob<K>& J, int d) {
  Sub<K> x;
  if (J.m == 0) {
    x.r0 = 0;
    x.nr = J.nr;
    x.s0 = 0;
    x.ns = J.ns;
  } else {
    const int nd = 1 << J.m;
    x.r0 = J.hr[d];
    x.nr = (d + 1 < nd ? (int64_t)J.hr[d + 1] : J.nr) - x.r0;
    x.s0 = J.hs[d];
    x.ns = (d + 1 < nd ? (int64_t)J.hs[d + 1] : J.ns) - x.s0;
  }
  return x;
}

// tiles of a sub-batch (0 if it cannot produce pairs)
__device__ __forceinline__ int64_t tiles_of(int64_t nr, int64_t ns) {
  return (nr > 0 && ns > 0) ? (ns + kFCapS - 1) / kFCapS : 0;
}

// Exclusive scan of v (one value per thread of a CTA of NT threads); the
// CTA's total goes to *total.  Ends with a barrier.
template <int NT, typename T>
__device__ __forceinline__ T block_excl(T v, T* s_warp, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  T pre = 0, all = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) {
    const T z = s_warp[w];
    if (w < warp) pre += z;
    all += z;
  }
  *total = all;
  __syncthreads();
  return pre + x - v;
}

}  // namespace

// ---------------------------------------------------------------------------
// k_fused_info: one CTA per job
// ---------------------------------------------------------------------------
template <typename K>
__global__ void __launch_bounds__(kFThreads) k_fused_info(const FusedJob<K>* __restrict__ jobs,
                                                          int64_t* __restrict__ info) {
  __shared__ int64_t s_w[kFWarps];
  __shared__ int64_t s_max[kFWarps];
  const FusedJob<K>& J = jobs[blockIdx.x];
  const int nd = J.m == 0 ? 1 : 1 << J.m;
  int64_t items = 0, kbt = 0, kbs = 0, maxr = 0;
  for (int d = threadIdx.x; d < nd; d += kFThreads) {
    const Sub<K> x = sub_of(J, d);
    const int64_t t = tiles_of(x.nr, x.ns);
    items += t;
    if (t > 1) {
      kbt += t;
      kbs += 1;
    }
    if (t > 0) maxr = max(maxr, x.nr);
  }
  int64_t tot;
  int64_t* outs[3] = {&items, &kbt, &kbs};
  for (int i = 0; i < 3; ++i) {
    block_excl<kFThreads, int64_t>(*outs[i], s_w, &tot);
    if (threadIdx.x == 0) info[4 * blockIdx.x + i] = tot;
  }
  // largest R sub-batch that produces pairs
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) maxr = max(maxr, __shfl_xor_sync(0xFFFFFFFFu, maxr, o));
  if (lane == 0) s_max[warp] = maxr;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kFWarps; ++w) maxr = max(maxr, s_max[w]);
    info[4 * blockIdx.x + 3] = maxr;
  }
}

// ---------------------------------------------------------------------------
// k_fused_items: one CTA per job writes its items (sub-batches in key order,
// tiles in row order) from its first item index on
// ---------------------------------------------------------------------------
template <typename K>
__global__ void __launch_bounds__(kFThreads) k_fused_items(const FusedJob<K>* __restrict__ jobs,
                                                           FItem* __restrict__ items) {
  __shared__ int64_t s_w[kFWarps];
  const int j = blockIdx.x;
  const FusedJob<K>& J = jobs[j];
  const int nd = J.m == 0 ? 1 : 1 << J.m;
  int64_t base_i = J.item0, base_t = J.kbt0, base_s = J.kbs0;
  for (int c = 0; c < nd; c += kFThreads) {
    const int d = c + (int)threadIdx.x;
    int64_t t = 0;
    if (d < nd) {
      const Sub<K> x = sub_of(J, d);
      t = tiles_of(x.nr, x.ns);
    }
    const bool multi = t > 1;
    int64_t ti, tt, ts;
    const int64_t ei = block_excl<kFThreads, int64_t>(t, s_w, &ti);
    const int64_t et = block_excl<kFThreads, int64_t>(multi ? t : 0, s_w, &tt);
    const int64_t es = block_excl<kFThreads, int64_t>(multi ? 1 : 0, s_w, &ts);
    Sub<K> x = {0, 0, 0, 0};
    if (d < nd) x = sub_of(J, d);
    using U = typename UnsignedOf<K>::type;
    for (int64_t k = 0; k < t; ++k) {
      FItem it;
      it.rk = (uint64_t)(uintptr_t)(J.rk + x.r0);
      it.rv = (uint64_t)(uintptr_t)(J.rv + x.r0);
      it.sk = (uint64_t)(uintptr_t)(J.sk + x.s0 + k * kFCapS);
      it.sv = (uint64_t)(uintptr_t)(J.sv + x.s0 + k * kFCapS);
      it.sublo = (uint64_t)((U)J.lo + ((U)d << kFKeyBits));
      it.nr = (int32_t)x.nr;
      it.ns = (int32_t)min((int64_t)kFCapS, x.ns - k * kFCapS);
      it.job = j;
      it.dt = (uint32_t)d | ((uint32_t)k << 11);
      it.kbt = multi ? (int32_t)(base_t + et + k) : -1;
      it.kbs = multi ? (int32_t)(base_s + es) : -1;
      items[base_i + ei + k] = it;
    }
    base_i += ti;
    base_t += tt;
    base_s += ts;
  }
}

// ---------------------------------------------------------------------------
// k_fused_hist: per-key totals of the multi-tile sub-batches (one CTA per
// item; items of single-tile sub-batches return at once)
// ---------------------------------------------------------------------------
template <typename K>
__global__ void __launch_bounds__(256) k_fused_hist(const FusedJob<K>* __restrict__ jobs,
                                                    const FItem* __restrict__ items,
                                                    uint32_t* __restrict__ tot) {
  __shared__ uint32_t h[kFKeys];
  const FItem it = items[blockIdx.x];
  if (it.kbt < 0) return;
  using U = typename UnsignedOf<K>::type;
  const U sublo = (U)it.sublo;
  for (int i = threadIdx.x; i < kFKeys; i += 256) h[i] = 0u;
  __syncthreads();
  const int n = it.ns;
  const K* __restrict__ sk = reinterpret_cast<const K*>(it.sk);
  for (int i = threadIdx.x; i < n; i += 256)
    atomicAdd(&h[(uint32_t)((U)sk[i] - sublo) & (kFKeys - 1)], 1u);
  __syncthreads();
  uint32_t* T = tot + (size_t)it.kbs * kFKeys;
  for (int i = threadIdx.x; i < kFKeys; i += 256)
    if (h[i]) atomicAdd(&T[i], h[i]);
}

// ---------------------------------------------------------------------------
// in-smem stable sort of n <= ITEMS * kFThreads rows by their 10-bit key
// offset: two LSD passes of 5-bit digits; the sorted row order lands in pb
// (pa holds the order after the first pass)
// ---------------------------------------------------------------------------
template <int ITEMS>
__device__ __forceinline__ void sort_offsets(const uint16_t* __restrict__ koff, int n,
                                             uint16_t* __restrict__ pa, uint16_t* __restrict__ pb,
                                             uint32_t* wcnt, uint16_t* wexcl, uint32_t* dbase) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wbase = warp * 32 * ITEMS;
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    const int sh = pass * kFDigit;
    uint16_t* __restrict__ outp = pass ? pb : pa;
    for (int i = tid; i < kFWarps * (kFBins / 2); i += kFThreads) wcnt[i] = 0u;
    __syncthreads();
    uint32_t dr[ITEMS];
    uint16_t idx[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int q = wbase + i * 32 + lane;
      idx[i] = (uint16_t)(q < n ? (pass ? pa[q] : q) : 0);
      dr[i] = q < n ? ((uint32_t)koff[idx[i]] >> sh) & (kFBins - 1) : 0u;
    }
    rank_items<kFDigit, ITEMS>(dr, n - wbase, wcnt + warp * (kFBins / 2));
    __syncthreads();
    // per digit: exclusive prefix over the warps, then the digits' bases
    if (tid < kFBins) {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kFWarps; ++w) {
        const uint32_t c = (wcnt[w * (kFBins / 2) + (tid >> 1)] >> ((tid & 1) * 16)) & 0xFFFFu;
        wexcl[w * kFBins + tid] = (uint16_t)run;
        run += c;
      }
      // warp 0 holds the 32 digits' totals: exclusive scan
      uint32_t x = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
      }
      dbase[tid] = x - run;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int q = wbase + i * 32 + lane;
      if (q < n) {
        const uint32_t d = dr[i] & 0xFFFFu;
        outp[dbase[d] + wexcl[warp * kFBins + d] + (dr[i] >> 16)] = idx[i];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// k_fused_join: one CTA per item
// ---------------------------------------------------------------------------
// Shared memory: per-warp counters of the key offsets (two 16-bit counters a
// word) and lane-mask tables of the ranking | per key offset: the
// sub-batch's R rows (two 16-bit counters a word) and the entry a row reads
// to write its pairs | the R rows' key offsets, sorted by key offset
// (stably) when a key has several R rows.  About 75 KB: three CTAs a
// multiprocessor.
// What a row of key offset k needs to write its pairs, in one 16-byte load:
// the position of the key's first pair for this tile's rows within the
// sub-batch's output (~0: no R row has the key), and the key's R id (one R
// row per key) or the start of its sorted R run (several).
template <typename K>
struct alignas(16) KeyEnt {
  uint64_t a;
  K r;
};

template <typename K>
struct FusedSmem {
  uint32_t wh[kFWarps][kFKeys / 2];
  uint32_t wm[kFWarps][128];
  uint32_t cR[kFKeys / 2];
  KeyEnt<K> ent[kFKeys];
  uint16_t r_koff[kFCapR];
  uint16_t r_pa[kFCapR];
  uint16_t r_pb[kFCapR];
  uint32_t wcnt[kFWarps * (kFBins / 2)];
  uint16_t wexcl[kFWarps * kFBins];
  uint32_t dbase[kFBins];
  uint64_t s_w64[kFWarps];
  uint64_t s_wb[kFWarps];
  uint64_t s_wc[kFWarps];
  uint32_t s_w32[kFWarps];
  uint64_t s_base;
  uint32_t s_item;
};

template <typename K>
size_t fused_smem_bytes() {
  return sizeof(FusedSmem<K>);
}

// One item: a tile of <= kFCapS S rows of a sub-batch and all its R rows.
//   1. R rows: count per key offset; a key's first R id goes to a table (a
//      key with several R rows sets a flag: then the R rows are sorted by key
//      offset, stably, and each key's run is used);
//   2. S rows into registers (warp w owns rows [w 256, (w + 1) 256), item u
//      of a lane is row w 256 + 32 u + lane), counted per key offset, ranked
//      stably within the warp by key offset (rank_items_or);
//   3. per key offset: the S rows of earlier warps (prefix over the warps'
//      counters), of earlier tiles of the sub-batch (look-back over count
//      vectors), and the key's first pair, Sum_{k' < k} |S_k'| |R_k'|;
//   4. the chained scan over the group's items gives the tile's first pair;
//   5. each S row's pairs go to their final position straight from registers.
#ifndef TJ_FUSED_MINB
#define TJ_FUSED_MINB 2
#endif
template <typename K>
__global__ void __launch_bounds__(kFThreads, TJ_FUSED_MINB)
    k_fused_join(const FItem* __restrict__ items,
                 int64_t n_items, uint32_t* __restrict__ item_counter,
                 uint64_t* __restrict__ item_lb, uint32_t* __restrict__ kb_lb,
                 const uint32_t* __restrict__ kb_tot, K* __restrict__ out, int64_t capacity,
                 const int64_t* __restrict__ out_base, int64_t* __restrict__ total,
                 int* __restrict__ err) {
  using U = typename UnsignedOf<K>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FusedSmem<K>& S = *reinterpret_cast<FusedSmem<K>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) S.s_item = atomicAdd(item_counter, 1u);
  // counters and tables start at zero
  for (int i = tid; i < kFWarps * (kFKeys / 2); i += kFThreads) (&S.wh[0][0])[i] = 0u;
  for (int i = tid; i < kFWarps * 128; i += kFThreads) (&S.wm[0][0])[i] = 0u;
  for (int i = tid; i < kFKeys / 2; i += kFThreads) S.cR[i] = 0u;
  __syncthreads();
  const int64_t ii = S.s_item;
  if (ii >= n_items) return;
  const FItem it = items[ii];
  const int t = (int)(it.dt >> 11);
  const bool multi_tile = it.kbt >= 0;
  const U sublo = (U)it.sublo;
  const int nr = it.nr;  // <= kFCapR (the host checked)
  const int ns = it.ns;
  const K* __restrict__ g_rv = reinterpret_cast<const K*>(it.rv);
  const K* __restrict__ g_sv = reinterpret_cast<const K*>(it.sv);

  // 1. the tile's global loads in flight at once: S keys, R keys and ids
  //    (the S ids are loaded when the pairs are written)
  const int wrow = warp * 32 * kFItemsS;
  K rkey[kFItemsR], rid_v[kFItemsR], skey[kFItemsS];
  {
    const K* __restrict__ rk = reinterpret_cast<const K*>(it.rk);
    const K* __restrict__ rv = g_rv;
    const K* __restrict__ sk = reinterpret_cast<const K*>(it.sk);
#pragma unroll
    for (int u = 0; u < kFItemsS; ++u) {
      const int row = wrow + u * 32 + lane;
      skey[u] = row < ns ? sk[row] : K(0);
    }
#pragma unroll
    for (int u = 0; u < kFItemsR; ++u) {
      const int i = tid + u * kFThreads;
      rkey[u] = i < nr ? rk[i] : K(0);
      rid_v[u] = i < nr ? rv[i] : K(0);
    }
  }
  // R rows: counts per key offset, a key's first R id in the table
  bool dup = false;
#pragma unroll
  for (int u = 0; u < kFItemsR; ++u) {
    const int i = tid + u * kFThreads;
    if (i < nr) {
      const uint32_t o = (uint32_t)((U)rkey[u] - sublo) & (kFKeys - 1);
      S.r_koff[i] = (uint16_t)o;
      const uint32_t sh = (o & 1u) * 16u;  // counts <= kFCapR: the halves never carry
      if (((atomicAdd(&S.cR[o >> 1], 1u << sh) >> sh) & 0xFFFFu) == 0u)
        S.ent[o].r = rid_v[u];  // the key's R id, kept unless the key has several
      else
        dup = true;
    }
  }
  // 2. S rows counted and ranked
  uint32_t dr[kFItemsS];
#pragma unroll
  for (int u = 0; u < kFItemsS; ++u) dr[u] = (uint32_t)((U)skey[u] - sublo) & (kFKeys - 1);
  rank_items_or<kFKeyBits - 7, kFItemsS>(dr, ns - wrow, &S.wh[warp][0], &S.wm[warp][0]);
  dup = __syncthreads_or(dup) != 0;  // also: counts complete, ranks done

  // 3. per key offset (two per thread: word tid of the warps' counters):
  //    the S rows of earlier warps, and the tile's count
  const int k0 = 2 * tid;
  uint32_t cs[2];
  {
    uint32_t run = 0;  // the two 16-bit halves never carry (counts <= kFCapS)
#pragma unroll
    for (int w = 0; w < kFWarps; ++w) {
      const uint32_t c = S.wh[w][tid];
      S.wh[w][tid] = run;
      run += c;
    }
    cs[0] = run & 0xFFFFu;
    cs[1] = run >> 16;
  }
  // multi-tile sub-batches: publish this tile's counts (look-back over the
  // sub-batch's tiles, one word per key offset)
  uint32_t* lb_mine = multi_tile ? kb_lb + (size_t)it.kbt * kFKeys : nullptr;
  if (multi_tile)
#pragma unroll
    for (int e = 0; e < 2; ++e) st_vol_u32(lb_mine + k0 + e, (t == 0 ? kFlagInc : kFlagAgg) | cs[e]);
  // keys with several R rows: their R rows sorted by key offset
  if (dup) sort_offsets<kFItemsR>(S.r_koff, nr, S.r_pa, S.r_pb, S.wcnt, S.wexcl, S.dbase);
  uint32_t pr[2] = {0u, 0u};
  if (multi_tile && t > 0) {
    // decoupled look-back over the earlier tiles of the sub-batch (a window
    // of kLB predecessors per round trip, both key offsets together; tile 0
    // publishes inclusive counts, so the walk ends there at the latest;
    // bounded wait)
    constexpr int kLB = 8;
    const int64_t first = it.kbt - t;  // a sub-batch's tiles have consecutive slots
    int64_t p[2] = {it.kbt - 1, it.kbt - 1};
    bool done[2] = {false, false};
    int spins = 0;
    while (!(done[0] && done[1])) {
      uint32_t v[2][kLB];
#pragma unroll
      for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int q = 0; q < kLB; ++q)
          v[e][q] = (!done[e] && p[e] - q >= first)
                        ? ld_vol_u32(kb_lb + (size_t)(p[e] - q) * kFKeys + k0 + e)
                        : kFlagInc;
      bool progress = false;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        if (done[e]) continue;
#pragma unroll
        for (int q = 0; q < kLB; ++q) {
          const uint32_t f = v[e][q] & ~kValMask;
          if (f == 0u) break;  // not published yet: wait for it
          pr[e] += v[e][q] & kValMask;
          --p[e];
          progress = true;
          if (f == kFlagInc) {
            done[e] = true;
            break;
          }
        }
      }
      if (!progress) {
        if (++spins > kSpinLimit) {
          atomicExch(err, (int)TJ_ERR_TIMEOUT);
          break;
        }
        __nanosleep(32);
      }
    }
#pragma unroll
    for (int e = 0; e < 2; ++e)
      st_vol_u32(lb_mine + k0 + e, kFlagInc | ((pr[e] + cs[e]) & kValMask));
  }
  uint32_t cr[2];
  uint64_t tot[2];
  {
    const uint32_t c2 = S.cR[tid];
    cr[0] = c2 & 0xFFFFu;
    cr[1] = c2 >> 16;
  }
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    tot[e] = multi_tile ? (uint64_t)kb_tot[(size_t)it.kbs * kFKeys + k0 + e] : (uint64_t)cs[e];
  }
  // one pass over the key offsets: the exclusive scan of the keys' pairs in
  // the sub-batch (the first pair of each key) and of their R rows (run
  // starts), with the sums of this tile's pairs and of earlier tiles' pairs
  uint64_t total_sub, cnt_tile, before;
  {
    const uint64_t p0 = tot[0] * cr[0], p1 = tot[1] * cr[1];
    uint64_t a = p0 + p1;                                              // scanned
    uint64_t b = (uint64_t)cs[0] * cr[0] + (uint64_t)cs[1] * cr[1];   // summed
    uint64_t c = (uint64_t)pr[0] * cr[0] + (uint64_t)pr[1] * cr[1];   // summed
    uint32_t r = cr[0] + cr[1];                                        // scanned
    uint64_t xa = a;
    uint32_t xr = r;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t ya = __shfl_up_sync(0xFFFFFFFFu, xa, o);
      const uint32_t yr = __shfl_up_sync(0xFFFFFFFFu, xr, o);
      if (lane >= o) {
        xa += ya;
        xr += yr;
      }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
      c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    }
    if (lane == 31) {
      S.s_w64[warp] = xa;
      S.s_w32[warp] = xr;
    }
    if (lane == 0) {
      S.s_wb[warp] = b;
      S.s_wc[warp] = c;
    }
    __syncthreads();
    uint64_t pa = 0, ta = 0, tb = 0, tc = 0;
    uint32_t pr32 = 0;
#pragma unroll
    for (int w = 0; w < kFWarps; ++w) {
      const uint64_t va = S.s_w64[w];
      if (w < warp) {
        pa += va;
        pr32 += S.s_w32[w];
      }
      ta += va;
      tb += S.s_wb[w];
      tc += S.s_wc[w];
    }
    const uint64_t eo = pa + xa - a;  // first pair of key k0 in the sub-batch
    const uint32_t er = pr32 + xr - r;  // first sorted R row of key k0
    const uint64_t first[2] = {eo, eo + p0};
    const uint32_t rstart[2] = {er, er + cr[0]};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      // the key's first pair for this tile's rows: after the earlier tiles';
      // with several R rows a key's run start replaces its R id
      S.ent[k0 + e].a = cr[e] ? first[e] + (uint64_t)pr[e] * cr[e] : ~0ull;
      if (dup) S.ent[k0 + e].r = (K)rstart[e];
    }
    total_sub = ta;
    cnt_tile = tb;
    before = tc;
  }

  // the S ids (read when the pairs are written): their loads in flight while
  // warp 0 runs the chained scan (the S keys' registers are free by now)
  K sid[kFItemsS];
  {
    const K* __restrict__ sv = g_sv;
#pragma unroll
    for (int u = 0; u < kFItemsS; ++u) {
      const int row = wrow + u * 32 + lane;
      sid[u] = row < ns ? sv[row] : K(0);
    }
  }
  // 4. chained scan over the group's items (warp 0): the tile's first pair
  if (warp == 0) {
    uint64_t* mine = item_lb + ii;
    uint64_t prefix = 0;
    if (ii == 0) {
      if (lane == 0) st_vol_u64(mine, kFlagInc64 | (cnt_tile & kValMask64));
    } else {
      if (lane == 0) st_vol_u64(mine, kFlagAgg64 | (cnt_tile & kValMask64));
      int64_t k = ii - 1;
      int spins = 0;
      while (true) {
        const int64_t idx = k - lane;
        const uint64_t v = idx >= 0 ? ld_vol_u64(item_lb + idx) : kFlagInc64;
        const uint64_t f = v & ~kValMask64;
        const uint32_t notready = __ballot_sync(0xFFFFFFFFu, f == 0ull);
        const uint32_t inc = __ballot_sync(0xFFFFFFFFu, f == kFlagInc64);
        const int first_nr = notready ? __ffs(notready) - 1 : 32;
        const int first_inc = inc ? __ffs(inc) - 1 : 32;
        const int take = first_inc < first_nr ? first_inc + 1 : first_nr;
        uint64_t y = lane < take ? (v & kValMask64) : 0ull;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) y += __shfl_xor_sync(0xFFFFFFFFu, y, o);
        prefix += y;
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
      if (lane == 0) st_vol_u64(mine, kFlagInc64 | ((prefix + cnt_tile) & kValMask64));
    }
    if (lane == 0) {
      const int64_t gb = out_base ? *out_base : 0;
      S.s_base = (uint64_t)gb + prefix;
      if (ii == n_items - 1) *total = gb + (int64_t)(prefix + cnt_tile);
    }
  }
  __syncthreads();
  const uint64_t E = S.s_base;      // absolute index of this tile's first pair
  const uint64_t base = E - before;  // the sub-batch's first pair
  // the tile's pairs lie anywhere in its sub-batch's: write nothing unless
  // all of them fit (the host reports TJ_ERR_CAPACITY)
  if (base + total_sub > (uint64_t)capacity) return;

  // 5. every S row's pairs, in key order, then S position, then R position
  using P = typename PairOf<K>::type;
  const bool vec = (((uintptr_t)out) & (2 * sizeof(K) - 1)) == 0;
  const uint32_t* wx = &S.wh[warp][0];
#pragma unroll
  for (int u = 0; u < kFItemsS; ++u) {
    if (wrow + u * 32 + lane >= ns) continue;
    const uint32_t k = dr[u] & 0xFFFFu;
    const KeyEnt<K> en = S.ent[k];
    if (en.a == ~0ull) continue;  // no R row has the key
    // S rows of the key before this one in the tile: earlier warps, earlier
    // lanes and items of this warp
    const uint32_t within = ((wx[k >> 1] >> ((k & 1u) * 16u)) & 0xFFFFu) + (dr[u] >> 16);
    if (!dup) {
      const uint64_t pos = base + en.a + within;
      if (vec) {
        P pr2;
        pr2.x = en.r;
        pr2.y = sid[u];
        *reinterpret_cast<P*>(out + 2 * pos) = pr2;
      } else {
        out[2 * pos] = en.r;
        out[2 * pos + 1] = sid[u];
      }
    } else {
      const uint32_t c = (S.cR[k >> 1] >> ((k & 1u) * 16u)) & 0xFFFFu;
      const uint64_t pos = base + en.a + (uint64_t)within * c;
      const uint32_t r0 = (uint32_t)en.r;
      const K* __restrict__ rv = g_rv;  // R ids in the order of the key's run
      for (uint32_t j = 0; j < c; ++j) {
        out[2 * (pos + j)] = rv[S.r_pb[r0 + j]];
        out[2 * (pos + j) + 1] = sid[u];
      }
    }
  }
}

// ---------------------------------------------------------------------------
template <typename K>
cudaError_t launch_fused_info(const FusedJob<K>* d_jobs, int nj, int64_t* d_info,
                              cudaStream_t st) {
  if (nj <= 0) return cudaSuccess;
  k_fused_info<K><<<nj, kFThreads, 0, st>>>(d_jobs, d_info);
  return cudaGetLastError();
}

template <typename K>
cudaError_t launch_fused_prep(const FusedJob<K>* d_jobs, int nj, FItem* d_items, int64_t n_items,
                              bool any_multi, uint32_t* d_kb_tot, cudaStream_t st) {
  if (nj <= 0 || n_items <= 0) return cudaSuccess;
  k_fused_items<K><<<nj, kFThreads, 0, st>>>(d_jobs, d_items);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !any_multi) return e;
  k_fused_hist<K><<<(unsigned)n_items, 256, 0, st>>>(d_jobs, d_items, d_kb_tot);
  return cudaGetLastError();
}

template <typename K>
cudaError_t launch_fused_join(const FusedJob<K>* d_jobs, const FItem* d_items, int64_t n_items,
                              uint32_t* d_item_counter, uint64_t* d_item_lb, uint32_t* d_kb_lb,
                              const uint32_t* d_kb_tot, K* out, int64_t capacity,
                              const int64_t* d_out_base, int64_t* d_total, int* d_err,
                              cudaStream_t st) {
  (void)d_jobs;  // the items carry what the join needs
  if (n_items <= 0) return cudaSuccess;
  k_fused_join<K><<<(unsigned)n_items, kFThreads, fused_smem_bytes<K>(), st>>>(
      d_items, n_items, d_item_counter, d_item_lb, d_kb_lb, d_kb_tot, out, capacity,
      d_out_base, d_total, d_err);
  return cudaGetLastError();
}

cudaError_t fused_init_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_fused_join<int32_t>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fused_smem_bytes<int32_t>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fused_join<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)fused_smem_bytes<int64_t>());
}

#define TJ_INSTANTIATE_FUSED(K)                                                                 \
  template cudaError_t launch_fused_info<K>(const FusedJob<K>*, int, int64_t*, cudaStream_t);   \
  template cudaError_t launch_fused_prep<K>(const FusedJob<K>*, int, FItem*, int64_t, bool,     \
                                            uint32_t*, cudaStream_t);                           \
  template cudaError_t launch_fused_join<K>(const FusedJob<K>*, const FItem*, int64_t,          \
                                            uint32_t*, uint64_t*, uint32_t*, const uint32_t*,   \
                                            K*, int64_t, const int64_t*, int64_t*, int*,        \
                                            cudaStream_t);
TJ_INSTANTIATE_FUSED(int32_t)
TJ_INSTANTIATE_FUSED(int64_t)

}  // namespace tj
