// Late materialisation of payload columns (paper Sec. 3.1, Sec. 3.2): the
// join aligns R(A, B, C) and S(B, D, E) on B and yields (r_id, s_id) pairs;
// k_gather_pairs then reads, for every pair, each requested column of R at
// r_id and of S at s_id and writes it to the pair's position of an output
// column.  One pass over the pairs; up to kGatherCols columns per launch.
//
// Work per pair: one 2w-byte pair read (coalesced), and per column one
// element read at a data-dependent row (a 32-byte sector per element unless
// neighbouring pairs share it) and one element written (coalesced).  Each
// thread takes kGatherRows pairs, blockDim apart, and issues all their loads
// of a column before its stores.
#include <algorithm>
#include <type_traits>

#include "tj_internal.cuh"

namespace tj {

constexpr int kGatherThreads = 256;
constexpr int kGatherRows = 4;  // pairs per thread per round

template <typename I>
__device__ __forceinline__ void load_pair(const I* p, int64_t i, I& r, I& s);
template <>
__device__ __forceinline__ void load_pair<int32_t>(const int32_t* p, int64_t i, int32_t& r,
                                                   int32_t& s) {
  const int2 v = __ldg(reinterpret_cast<const int2*>(p) + i);
  r = v.x;
  s = v.y;
}
template <>
__device__ __forceinline__ void load_pair<int64_t>(const int64_t* p, int64_t i, int64_t& r,
                                                   int64_t& s) {
  const longlong2 v = __ldg(reinterpret_cast<const longlong2*>(p) + i);
  r = v.x;
  s = v.y;
}

template <typename E>
__device__ __forceinline__ void gather_col(const GatherCol& c, const int64_t (&row)[kGatherRows],
                                           const int64_t (&at)[kGatherRows]) {
  const E* __restrict__ src = reinterpret_cast<const E*>(c.src);
  E* __restrict__ dst = reinterpret_cast<E*>(c.dst);
  E v[kGatherRows];
#pragma unroll
  for (int u = 0; u < kGatherRows; ++u) v[u] = row[u] >= 0 ? __ldg(src + row[u]) : E(0);
#pragma unroll
  for (int u = 0; u < kGatherRows; ++u)
    if (row[u] >= 0) dst[at[u]] = v[u];
}

// pairs[i] = (r_id, s_id), i < n; an id outside [0, rows of its side) sets
// *err = TJ_ERR_INVALID and its row is not written.
template <typename I>
__global__ void __launch_bounds__(kGatherThreads)
    k_gather_pairs(const I* __restrict__ pairs, int64_t n, int64_t n_r, int64_t n_s,
                   GatherArgs a, int* __restrict__ err) {
  const int64_t per_block = (int64_t)kGatherThreads * kGatherRows;
  for (int64_t b0 = (int64_t)blockIdx.x * per_block; b0 < n; b0 += (int64_t)gridDim.x * per_block) {
    int64_t at[kGatherRows], rr[kGatherRows], sr[kGatherRows];
    bool bad = false;
#pragma unroll
    for (int u = 0; u < kGatherRows; ++u) {
      at[u] = b0 + u * kGatherThreads + threadIdx.x;
      rr[u] = sr[u] = -1;
      if (at[u] < n) {
        I r, s;
        load_pair<I>(pairs, at[u], r, s);
        const bool ok = (int64_t)r >= 0 && (int64_t)r < n_r && (int64_t)s >= 0 && (int64_t)s < n_s;
        if (ok) {
          rr[u] = (int64_t)r;
          sr[u] = (int64_t)s;
        } else {
          bad = true;
        }
      }
    }
    if (bad) atomicCAS(err, 0, (int)TJ_ERR_INVALID);
    for (int c = 0; c < a.n; ++c) {
      const GatherCol& col = a.c[c];
      if (col.bytes == 8) {
        if (col.side)
          gather_col<unsigned long long>(col, sr, at);
        else
          gather_col<unsigned long long>(col, rr, at);
      } else {
        if (col.side)
          gather_col<unsigned int>(col, sr, at);
        else
          gather_col<unsigned int>(col, rr, at);
      }
    }
  }
}

template <typename I>
cudaError_t launch_gather_pairs(const I* pairs, int64_t n, int64_t n_r, int64_t n_s,
                                const GatherArgs& a, int* d_err, int sms, cudaStream_t st) {
  if (n <= 0 || a.n <= 0) return cudaSuccess;
  const int64_t per_block = (int64_t)kGatherThreads * kGatherRows;
  const int64_t want = (n + per_block - 1) / per_block;
  const int64_t grid = std::min<int64_t>(want, (int64_t)std::max(1, sms) * 8);
  k_gather_pairs<I><<<(unsigned)grid, kGatherThreads, 0, st>>>(pairs, n, n_r, n_s, a, d_err);
  return cudaGetLastError();
}

// dst[i] = src[idx[i]], i < n (idx: a permutation of rows, so every index
// is in range); elements of 4 or 8 bytes (T = unsigned int / long long).
template <typename I, typename T>
__global__ void __launch_bounds__(kGatherThreads)
    k_gather_idx(const T* __restrict__ src, const I* __restrict__ idx, T* __restrict__ dst,
                 int64_t n) {
  const int64_t per_block = (int64_t)kGatherThreads * kGatherRows;
  for (int64_t b0 = (int64_t)blockIdx.x * per_block; b0 < n; b0 += (int64_t)gridDim.x * per_block) {
    T v[kGatherRows];
#pragma unroll
    for (int u = 0; u < kGatherRows; ++u) {
      const int64_t i = b0 + u * kGatherThreads + threadIdx.x;
      v[u] = i < n ? __ldg(src + (int64_t)__ldg(idx + i)) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kGatherRows; ++u) {
      const int64_t i = b0 + u * kGatherThreads + threadIdx.x;
      if (i < n) dst[i] = v[u];
    }
  }
}

template <typename I>
__global__ void k_iota(I* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (I)i;
}

template <typename K>
cudaError_t launch_gather_idx(const K* src, const K* idx, K* dst, int64_t n, int sms,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  using T = typename std::conditional<sizeof(K) == 8, unsigned long long, unsigned int>::type;
  const int64_t per_block = (int64_t)kGatherThreads * kGatherRows;
  const int64_t grid = std::min<int64_t>((n + per_block - 1) / per_block,
                                         (int64_t)std::max(1, sms) * 8);
  k_gather_idx<K, T><<<(unsigned)grid, kGatherThreads, 0, st>>>(
      reinterpret_cast<const T*>(src), idx, reinterpret_cast<T*>(dst), n);
  return cudaGetLastError();
}

template <typename K>
cudaError_t launch_iota(K* out, int64_t n, int sms, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t grid = std::min<int64_t>((n + kGatherThreads - 1) / kGatherThreads,
                                         (int64_t)std::max(1, sms) * 8);
  k_iota<K><<<(unsigned)grid, kGatherThreads, 0, st>>>(out, n);
  return cudaGetLastError();
}

template cudaError_t launch_gather_idx<int32_t>(const int32_t*, const int32_t*, int32_t*, int64_t,
                                                int, cudaStream_t);
template cudaError_t launch_gather_idx<int64_t>(const int64_t*, const int64_t*, int64_t*, int64_t,
                                                int, cudaStream_t);
template cudaError_t launch_iota<int32_t>(int32_t*, int64_t, int, cudaStream_t);
template cudaError_t launch_iota<int64_t>(int64_t*, int64_t, int, cudaStream_t);
// Multi-column keys folded into one key when their significant bits fit:
// packed[i] = sum over c of (cols[c][i] - lo[c]) << shift[c] (unsigned
// arithmetic; the first column holds the highest bits), and back:
// cols[c][i] = ((packed[i] >> shift[c]) & mask[c]) + lo[c].
template <typename K>
__global__ void __launch_bounds__(kGatherThreads)
    k_pack(PackArgs<K> a, K* __restrict__ packed, int64_t n) {
  using U = typename std::make_unsigned<K>::type;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    U v = 0;
    for (int c = 0; c < a.n; ++c) v |= ((U)__ldg(a.col[c] + i) - (U)a.lo[c]) << a.shift[c];
    packed[i] = (K)v;
  }
}

template <typename K>
__global__ void __launch_bounds__(kGatherThreads)
    k_unpack(PackArgs<K> a, const K* __restrict__ packed, int64_t n) {
  using U = typename std::make_unsigned<K>::type;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const U v = (U)__ldg(packed + i);
    for (int c = 0; c < a.n; ++c) {
      const U m = a.bits[c] >= (int)(8 * sizeof(K)) ? ~(U)0 : (((U)1 << a.bits[c]) - 1);
      a.col[c][i] = (K)(((v >> a.shift[c]) & m) + (U)a.lo[c]);
    }
  }
}

template <typename K>
cudaError_t launch_pack(const PackArgs<K>& a, K* packed, int64_t n, bool unpack, int sms,
                        cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t grid = std::min<int64_t>((n + kGatherThreads - 1) / kGatherThreads,
                                         (int64_t)std::max(1, sms) * 8);
  if (unpack)
    k_unpack<K><<<(unsigned)grid, kGatherThreads, 0, st>>>(a, packed, n);
  else
    k_pack<K><<<(unsigned)grid, kGatherThreads, 0, st>>>(a, packed, n);
  return cudaGetLastError();
}

template cudaError_t launch_pack<int32_t>(const PackArgs<int32_t>&, int32_t*, int64_t, bool, int,
                                          cudaStream_t);
template cudaError_t launch_pack<int64_t>(const PackArgs<int64_t>&, int64_t*, int64_t, bool, int,
                                          cudaStream_t);
// Small control transfers between device memory and pinned host memory that
// the device maps (tables going in, counts and statistics coming out), done by
// a kernel instead of a copy engine: a transfer queued on an engine behind a
// caller's bulk copy in the same direction would wait for all of it.
__global__ void k_copy_bytes(unsigned char* __restrict__ dst, const unsigned char* __restrict__ src,
                             size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((((uintptr_t)dst | (uintptr_t)src) & 15u) == 0) {
    const size_t n16 = n / 16;
    for (size_t i = t; i < n16; i += stride)
      reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
    for (size_t i = n16 * 16 + t; i < n; i += stride) dst[i] = src[i];
  } else {
    for (size_t i = t; i < n; i += stride) dst[i] = src[i];
  }
}

cudaError_t launch_copy_bytes(void* dst, const void* src, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const size_t per = (size_t)kGatherThreads * 16;
  const unsigned grid = (unsigned)std::min<size_t>((n + per - 1) / per, 1024);
  k_copy_bytes<<<grid, kGatherThreads, 0, st>>>(static_cast<unsigned char*>(dst),
                                                static_cast<const unsigned char*>(src), n);
  return cudaGetLastError();
}

template cudaError_t launch_gather_pairs<int32_t>(const int32_t*, int64_t, int64_t, int64_t,
                                                  const GatherArgs&, int*, int, cudaStream_t);
template cudaError_t launch_gather_pairs<int64_t>(const int64_t*, int64_t, int64_t, int64_t,
                                                  const GatherArgs&, int*, int, cudaStream_t);

}  // namespace tj
