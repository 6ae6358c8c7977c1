// Learned key-range partitioner (no counterpart in the paper; it chooses the
// key-range batches of the partitioned join, the device analogue of the
// relational path's work_mem batches of Sec. 6).
//
//   k_sample_gather : every `stride`-th row of R and of S from seeded offsets,
//                     pooled (a 1% sample for stride 100).
//   k_quantiles     : knots / boundaries at sample quantiles of the sorted
//                     sample, q_i = s[floor(i (m - 1) / G)] (the piecewise-
//                     linear CDF model; its partition boundaries for P | G are
//                     the knots t_{(G/P) p}).
//   MLP kernels     : see tj_mlp.cu.
#include <algorithm>

#include "tj_internal.cuh"

namespace tj {

template <typename K>
__global__ void k_sample_gather(const K* __restrict__ a, int64_t ma, int64_t off_a,
                                const K* __restrict__ b, int64_t mb, int64_t off_b, int stride,
                                K* __restrict__ out_k, K* __restrict__ out_v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ma) {
    out_k[i] = a[off_a + i * stride];
    out_v[i] = (K)i;
  } else if (i < ma + mb) {
    out_k[i] = b[off_b + (i - ma) * stride];
    out_v[i] = (K)i;
  }
}

// out[i] = sorted[floor(i * (m - 1) / G) ] for i in [first, last]
template <typename K>
__global__ void k_quantiles(const K* __restrict__ sorted, int64_t m, int G, int first, int last,
                            int step, K* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = first + i * step;
  if (q > last) return;
  const int64_t idx = ((int64_t)q * (m - 1)) / G;
  out[i] = sorted[idx];
}

// edges[d] = number of sorted sample keys below lo + d * 2^shift, d = 0..nb
// (the balance of equal-width key ranges, judged on the sample)
template <typename K>
__global__ void k_sorted_bucket_edges(const K* __restrict__ sorted, int64_t m, uint64_t lo,
                                      int shift, int nb, int64_t* __restrict__ edges) {
  using U = typename UnsignedOf<K>::type;
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d > nb) return;
  const unsigned long long off = shift >= 64 ? 0ull : ((unsigned long long)d << shift);
  const bool past = d > 0 && (shift >= 64 || (off >> shift) != (unsigned long long)d ||
                              off > (unsigned long long)(U)(~(U)0));
  int64_t a = 0, b = m;  // first index with (key - lo) >= off
  if (past) {
    a = m;
  } else {
    while (a < b) {
      const int64_t mid = (a + b) >> 1;
      if ((unsigned long long)(U)((U)sorted[mid] - (U)lo) < off)
        a = mid + 1;
      else
        b = mid;
    }
  }
  edges[d] = a;
}

// counts[side * kMaxBins + p]: sample rows of each side (sample index < m_r:
// R) whose key lies in batch p (p = number of cuts <= key)
template <typename K>
__global__ void k_sample_route_counts(const K* __restrict__ keys, const K* __restrict__ idx,
                                      int64_t m, int64_t m_r, const K* __restrict__ cuts,
                                      int ncuts, uint32_t* __restrict__ counts) {
  __shared__ uint32_t s_c[2 * kMaxBins];
  for (int i = threadIdx.x; i < 2 * kMaxBins; i += blockDim.x) s_c[i] = 0u;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const K key = keys[i];
    int a = 0, b = ncuts;  // first cut > key
    while (a < b) {
      const int mid = (a + b) >> 1;
      if (cuts[mid] <= key)
        a = mid + 1;
      else
        b = mid;
    }
    const int side = (int64_t)idx[i] < m_r ? 0 : 1;
    atomicAdd(&s_c[side * kMaxBins + a], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * kMaxBins; i += blockDim.x)
    if (s_c[i]) atomicAdd(&counts[i], s_c[i]);
}

template <typename K>
cudaError_t launch_sample_route_counts(const K* keys, const K* idx, int64_t m, int64_t m_r,
                                       const K* cuts, int ncuts, uint32_t* counts,
                                       cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const int64_t grid = std::min<int64_t>((m + kThreads - 1) / kThreads, 152 * 4);
  k_sample_route_counts<K><<<(unsigned)grid, kThreads, 0, st>>>(keys, idx, m, m_r, cuts, ncuts,
                                                                 counts);
  return cudaGetLastError();
}

template <typename K>
cudaError_t launch_sorted_bucket_edges(const K* sorted, int64_t m, uint64_t lo, int shift, int nb,
                                       int64_t* edges, cudaStream_t st) {
  k_sorted_bucket_edges<K><<<(nb + 1 + kThreads - 1) / kThreads, kThreads, 0, st>>>(
      sorted, m, lo, shift, nb, edges);
  return cudaGetLastError();
}

template <typename K>
cudaError_t launch_sample_gather(const K* a, int64_t ma, int64_t off_a, const K* b, int64_t mb,
                                 int64_t off_b, int stride, K* out_k, K* out_v, cudaStream_t st) {
  const int64_t n = ma + mb;
  if (n <= 0) return cudaSuccess;
  k_sample_gather<K><<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(
      a, ma, off_a, b, mb, off_b, stride, out_k, out_v);
  return cudaGetLastError();
}

template <typename K>
cudaError_t launch_quantiles(const K* sorted, int64_t m, int G, int first, int last, int step,
                             K* out, cudaStream_t st) {
  const int n = (last - first) / step + 1;
  if (n <= 0) return cudaSuccess;
  k_quantiles<K><<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(sorted, m, G, first, last,
                                                                      step, out);
  return cudaGetLastError();
}

#define TJ_INSTANTIATE_LEARNED(K)                                                                \
  template cudaError_t launch_sample_gather<K>(const K*, int64_t, int64_t, const K*, int64_t,    \
                                               int64_t, int, K*, K*, cudaStream_t);              \
  template cudaError_t launch_quantiles<K>(const K*, int64_t, int, int, int, int, K*, cudaStream_t); \
  template cudaError_t launch_sorted_bucket_edges<K>(const K*, int64_t, uint64_t, int, int,      \
                                                     int64_t*, cudaStream_t);                   \
  template cudaError_t launch_sample_route_counts<K>(const K*, const K*, int64_t, int64_t,       \
                                                     const K*, int, uint32_t*, cudaStream_t);
TJ_INSTANTIATE_LEARNED(int32_t)
TJ_INSTANTIATE_LEARNED(int64_t)

}  // namespace tj
