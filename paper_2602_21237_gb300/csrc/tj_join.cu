// Join of two key-sorted relations on their common key axis (paper Sec. 4.1)
// with a single final materialisation of (r_id, s_id) pairs (Sec. 3.1).
//
//   k_tile_ranges : for every tile of 2048 sorted S rows, the range [a, b) of
//                   sorted R rows whose keys lie between the tile's first and
//                   last key (two binary searches per tile).
//   k_join        : per S tile, fused count -> scan -> write:
//                     1. stage the tile's S rows and (if b - a <= 2048) its R
//                        range in shared memory;
//                     2. build an open-addressing hash table of the R range's
//                        distinct keys with shared-memory atomicCAS: slot ->
//                        (first, end) of the key's run of R rows;
//                     3. probe it once per S row -> match count and run start;
//                     4. exclusive scan of the counts inside the CTA, then a
//                        decoupled look-back over all tiles of all jobs gives
//                        the tile's first output index;
//                     5. write the pairs, ordered by key, S position, R
//                        position, if they fit the caller's capacity.
//                   Tiles whose R range exceeds the on-chip capacity (S sparse
//                   against R) binary-search each key in global memory instead.
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

template <typename K>
__device__ __forceinline__ int64_t lower_bound_g(const K* __restrict__ a, int64_t n, K key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

template <typename K>
__device__ __forceinline__ int64_t upper_bound_g(const K* __restrict__ a, int64_t n, K key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (key < a[mid])
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t ht_hash(int32_t k) {
  return ((uint32_t)k * 0x9E3779B9u) >> (32 - 12);
}
__device__ __forceinline__ uint32_t ht_hash(int64_t k) {
  return (uint32_t)(((uint64_t)k * 0x9E3779B97F4A7C15ull) >> (64 - 12));
}
static_assert(kHTSlots == 4096, "ht_hash assumes 4096 slots");
static_assert(kRCap < 0xFFFF, "run bounds are packed in 16 bits");

constexpr uint32_t kHTEmpty = 0xFFFFFFFFu;

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_volatile_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---------------------------------------------------------------------------
template <typename K>
__global__ void k_tile_ranges(const JoinJob<K>* __restrict__ jobs, int num_jobs,
                              int64_t total_tiles, int64_t* __restrict__ ra,
                              int64_t* __restrict__ rb, const int32_t* __restrict__ tile_job) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total_tiles) return;
  const int j = tile_job ? tile_job[t] : find_job_j(jobs, num_jobs, t);
  const JoinJob<K>* J = jobs + j;
  const int64_t row0 = (t - J->tile0) * kJTile;
  const int64_t row1 = min(J->ns, row0 + kJTile);
  const K kf = J->sk[row0];
  const K kl = J->sk[row1 - 1];
  ra[t] = lower_bound_g(J->rk, J->nr, kf);
  rb[t] = upper_bound_g(J->rk, J->nr, kl);
}

// ---------------------------------------------------------------------------
template <typename K>
constexpr size_t join_smem_bytes() {
  return sizeof(K) * kJTile             // S keys of the tile
         + sizeof(K) * kRCap            // R keys of the tile's R range
         + sizeof(uint32_t) * kHTSlots  // hash table: packed (first, end) of a run
         + sizeof(uint64_t) * kJTile    // per-row counts -> exclusive offsets
         + sizeof(uint32_t) * kJTile;   // per-row run start (relative to a)
}

template <typename K>
__global__ void __launch_bounds__(kThreads, 3)
    k_join(const JoinJob<K>* __restrict__ jobs, int num_jobs, int64_t total_tiles,
           const int64_t* __restrict__ ra, const int64_t* __restrict__ rb,
           uint64_t* __restrict__ lookback, uint32_t* __restrict__ tile_counter,
           K* __restrict__ out, int64_t capacity, const int64_t* __restrict__ out_base,
           int64_t* __restrict__ job_out, int64_t* __restrict__ total, int* __restrict__ err,
           const int32_t* __restrict__ tile_job) {
  extern __shared__ __align__(16) unsigned char smem[];
  K* s_sk = reinterpret_cast<K*>(smem);
  K* s_rk = s_sk + kJTile;
  uint32_t* s_ht = reinterpret_cast<uint32_t*>(s_rk + kRCap);
  uint64_t* s_off = reinterpret_cast<uint64_t*>(s_ht + kHTSlots);
  uint32_t* s_rs = reinterpret_cast<uint32_t*>(s_off + kJTile);
  __shared__ uint64_t s_wsum[kWarps];
  __shared__ uint64_t s_base, s_tot;
  __shared__ uint32_t s_t;
  __shared__ int s_maxcnt;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_t = atomicAdd(tile_counter, 1u);
    s_maxcnt = 0;
  }
  __syncthreads();
  const int64_t t = s_t;
  if (t >= total_tiles) return;
  const int j = tile_job ? tile_job[t] : find_job_j(jobs, num_jobs, t);
  const JoinJob<K> J = jobs[j];
  const int64_t a = ra[t];
  const int64_t nrr = rb[t] - a;
  const int64_t lt = t - J.tile0;
  const int64_t row0 = lt * kJTile;
  const int nv = (int)min((int64_t)kJTile, J.ns - row0);
  const K* __restrict__ sk_g = J.sk + row0;
  const K* __restrict__ sv_g = J.sv + row0;
  const K* __restrict__ rk_g = J.rk + a;
  const K* __restrict__ rv_g = J.rv + a;

  // S ids of this thread's rows, loaded now and used only when writing
  constexpr int kRows = kJTile / kThreads;
  K sid[kRows];
#pragma unroll
  for (int u = 0; u < kRows; ++u) {
    const int q = tid + u * kThreads;
    sid[u] = q < nv ? sv_g[q] : K(0);
  }
  for (int q = tid; q < nv; q += kThreads) s_sk[q] = sk_g[q];

  // Probe: match count and run start of every S row of the tile.  The tile's
  // R range is aligned chunk by chunk (kRCap rows each, up to kMaxChunks)
  // through the on-chip table; a run of equal keys that straddles chunks adds
  // up.  Tiles whose R range is wider (S sparse against R) binary-search R in
  // global memory instead.
  const int64_t nchunks = (nrr + kRCap - 1) / kRCap;
  uint32_t cnt[kRows], start[kRows];
#pragma unroll
  for (int u = 0; u < kRows; ++u) cnt[u] = start[u] = 0u;
  if (nchunks <= kMaxChunks) {
    for (int64_t c = 0; c < nchunks; ++c) {
      const int c0 = (int)(c * kRCap);
      const int nc = (int)min((int64_t)kRCap, nrr - c0);
      __syncthreads();  // the previous chunk's probes are done
      for (int i = tid; i < nc; i += kThreads) s_rk[i] = rk_g[c0 + i];
      for (int i = tid; i < kHTSlots; i += kThreads) s_ht[i] = kHTEmpty;
      __syncthreads();
      // insert the first row of every run of equal keys; keys are distinct, so
      // an occupied slot is never this key and insertion needs no comparison
      for (int i = tid; i < nc; i += kThreads) {
        if (i == 0 || s_rk[i] != s_rk[i - 1]) {
          uint32_t h = ht_hash(s_rk[i]);
          while (atomicCAS(&s_ht[h], kHTEmpty, (uint32_t)i | 0xFFFF0000u) != kHTEmpty)
            h = (h + 1) & (kHTSlots - 1);
        }
      }
      __syncthreads();
      // the last row of every run records the run's end
      for (int i = tid; i < nc; i += kThreads) {
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
      for (int u = 0; u < kRows; ++u) {
        const int q = tid + u * kThreads;
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
  } else {
#pragma unroll
    for (int u = 0; u < kRows; ++u) {
      const int q = tid + u * kThreads;
      if (q >= nv) continue;
      const K key = s_sk[q];
      const int64_t lo = lower_bound_g(rk_g, nrr, key);
      const int64_t hi = upper_bound_g(rk_g, nrr, key);
      start[u] = (uint32_t)lo;
      cnt[u] = (uint32_t)(hi - lo);
    }
  }
  // the R id of each row's first match is gathered right away (used when writing)
  int mymax = 0;
  K rid[kRows];
#pragma unroll
  for (int u = 0; u < kRows; ++u) {
    const int q = tid + u * kThreads;
    rid[u] = K(0);
    if (q >= nv) continue;
    s_off[q] = cnt[u];
    s_rs[q] = start[u];
    if (cnt[u]) rid[u] = rv_g[start[u]];
    mymax = max(mymax, (int)cnt[u]);
  }
  if (mymax > 1) atomicMax(&s_maxcnt, mymax);
  __syncthreads();

  // exclusive scan of the tile's counts: thread tid owns rows [8 tid, 8 tid + 8)
  {
    constexpr int kPer = kJTile / kThreads;
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
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    uint64_t pre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      if (w < warp) pre += s_wsum[w];
      tot += s_wsum[w];
    }
    uint64_t run = pre + x - sum;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int q = tid * kPer + i;
      if (q < nv) s_off[q] = run;
      run += v[i];
    }
    if (tid == 0) s_tot = tot;
  }
  __syncthreads();
  const uint64_t C = s_tot;

  // chained scan over all join tiles (all jobs): this tile's first output index
  if (tid == 0) {
    uint64_t* mine = lookback + t;
    uint64_t prefix = 0;
    if (t == 0) {
      st_volatile_u64(mine, kFlagInc64 | (C & kValMask64));
    } else {
      st_volatile_u64(mine, kFlagAgg64 | (C & kValMask64));
      int64_t k = t - 1;  // newest predecessor not yet summed
      int spins = 0;
      bool done = false;
      while (!done) {
        uint64_t v[kLookWindow];
#pragma unroll
        for (int w = 0; w < kLookWindow; ++w)
          v[w] = (k - w >= 0) ? ld_volatile_u64(lookback + (k - w)) : kFlagInc64;
        int used = 0;
        uint64_t acc = 0;
#pragma unroll
        for (int w = 0; w < kLookWindow; ++w) {
          if (used != w) break;
          const uint64_t f = v[w] & ~kValMask64;
          if (f == 0ull) break;
          acc += v[w] & kValMask64;
          ++used;
          if (f == kFlagInc64) {
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
      st_volatile_u64(mine, kFlagInc64 | ((prefix + C) & kValMask64));
    }
    s_base = prefix;
    if (lt == 0 && job_out) job_out[j] = (int64_t)prefix;
    if (t == total_tiles - 1) *total = (int64_t)(prefix + C);
  }
  __syncthreads();
  // output index of this tile's first pair: the group's base (the partitioned
  // join writes several groups one after another) plus the chained prefix
  const uint64_t E = s_base + (out_base ? (uint64_t)*out_base : 0ull);
  if (E + C > (uint64_t)capacity) return;  // the host reports TJ_ERR_CAPACITY

  K* __restrict__ o = out + 2 * E;
  if (s_maxcnt <= 1) {
    // at most one match per S row (e.g. a foreign-key join): row-wise writes
#pragma unroll
    for (int u = 0; u < kRows; ++u) {
      const int q = tid + u * kThreads;
      if (q >= nv) break;
      const uint64_t off = s_off[q];
      const bool hit = (q + 1 < nv ? s_off[q + 1] : C) > off;
      if (hit) {
        o[2 * off] = rid[u];
        o[2 * off + 1] = sid[u];
      }
    }
  } else {
    // general fan-out: output-wise, each output index finds its S row
    for (uint64_t x = tid; x < C; x += kThreads) {
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
                               int64_t* d_ra, int64_t* d_rb, cudaStream_t st,
                               const int32_t* d_tile_job) {
  if (total_tiles <= 0) return cudaSuccess;
  const int64_t grid = (total_tiles + kThreads - 1) / kThreads;
  k_tile_ranges<K><<<(unsigned)grid, kThreads, 0, st>>>(d_jobs, num_jobs, total_tiles, d_ra, d_rb,
                                                        d_tile_job);
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
cudaError_t launch_join(const JoinJob<K>* d_jobs, int num_jobs, int64_t total_tiles,
                        const int64_t* d_ra, const int64_t* d_rb, uint64_t* d_lookback,
                        uint32_t* d_tile_counter, K* out, int64_t capacity,
                        const int64_t* d_out_base, int64_t* d_job_out, int64_t* d_total,
                        int* d_err, cudaStream_t st, const int32_t* d_tile_job) {
  if (total_tiles <= 0) return cudaSuccess;
  const size_t smem = join_smem_bytes<K>();
  k_join<K><<<(unsigned)total_tiles, kThreads, smem, st>>>(
      d_jobs, num_jobs, total_tiles, d_ra, d_rb, d_lookback, d_tile_counter, out, capacity,
      d_out_base, d_job_out, d_total, d_err, d_tile_job);
  return cudaGetLastError();
}

// base += group total (stream-ordered between the groups of a partitioned join)
__global__ void k_add_base(int64_t* base, int64_t* total) {
  *base += *total;
  *total = 0;
}

cudaError_t launch_add_base(int64_t* d_base, int64_t* d_total, cudaStream_t st) {
  k_add_base<<<1, 1, 0, st>>>(d_base, d_total);
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

cudaError_t join_init_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_join<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)join_smem_bytes<int32_t>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_join<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)join_smem_bytes<int64_t>());
}

#define TJ_INSTANTIATE_JOIN(K)                                                                  \
  template cudaError_t launch_tile_ranges<K>(const JoinJob<K>*, int, int64_t, int64_t*, int64_t*, \
                                             cudaStream_t, const int32_t*);                     \
  template cudaError_t launch_fill_join_tile_job<K>(const JoinJob<K>*, int, int32_t*,            \
                                                    cudaStream_t);                              \
  template cudaError_t launch_join<K>(const JoinJob<K>*, int, int64_t, const int64_t*,           \
                                      const int64_t*, uint64_t*, uint32_t*, K*, int64_t,          \
                                      const int64_t*, int64_t*, int64_t*, int*, cudaStream_t,     \
                                      const int32_t*);                                            \
  template cudaError_t launch_fix_job_out<K>(const JoinJob<K>*, int, int64_t, int64_t*,          \
                                             const int64_t*, cudaStream_t);
TJ_INSTANTIATE_JOIN(int32_t)
TJ_INSTANTIATE_JOIN(int64_t)

}  // namespace tj
