// The MLP key-CDF model of the learned partitioner (no counterpart in the
// paper): a 1 -> 32 -> 32 -> 1 ReLU network on x = log2(1 + k - s_0) /
// log2(1 + s_{m-1} - s_0), fitted to the empirical CDF of a sorted key sample
// (y_j = j / (m - 1)) by mean squared error with Adam, entirely on the device.
//
// Parameters (1153 fp32, flat): [b3 | w1(32) | b1(32) | W2(32x32, row i = from
// hidden-1 unit i) | b2(32) | w3(32)].
//
// One CTA of 512 threads runs the whole training: each step draws a batch of
// 256 sample rows with a counter-based generator (splitmix64 of seed, step,
// row), runs the forward and backward pass one sample per thread with the
// activations kept in shared memory, reduces every parameter's gradient over
// the batch in a fixed order (one parameter per thread), and applies Adam.
// The network is then tabulated on a grid of the normalised axis and made
// monotone by a running maximum; partition boundaries are read off the table.
#include <math.h>

#include "tj_internal.cuh"

namespace tj {

constexpr int kH = 32;
constexpr int kNP = 1 + kH + kH + kH * kH + kH + kH;  // 1153
constexpr int kMB = 256;                               // batch rows per step
constexpr int kMT = 512;                               // threads of the training CTA
// offsets in the flat parameter vector
constexpr int kOB3 = 0, kOW1 = 1, kOB1 = 1 + kH, kOW2 = 1 + 2 * kH, kOB2 = 1 + 2 * kH + kH * kH,
              kOW3 = 1 + 3 * kH + kH * kH;

// per-sample rows padded to 33 words so a warp's rows fall in distinct banks
constexpr int kHP = kH + 1;
struct MlpSmem {
  float th[kNP];
  float g[kNP];
  float x[kMB], y[kMB], dy[kMB];
  float h1[kMB][kHP];
  float h2[kMB][kHP];
  float dz1[kMB][kHP];
  float dz2[kMB][kHP];
};

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Forward + backward of the batch in S.x / S.y (n <= kMB rows) and the batch
// gradient of the mean squared error into S.g.  Reads S.th.
__device__ void mlp_batch_grad(MlpSmem& S, int n) {
  const int tid = threadIdx.x;
  const float inv = 2.0f / (float)n;
  if (tid < n) {
    const float x = S.x[tid];
    float* h1 = S.h1[tid];
    float* h2 = S.h2[tid];
    float* dz1 = S.dz1[tid];
    float* dz2 = S.dz2[tid];
#pragma unroll 8
    for (int i = 0; i < kH; ++i) h1[i] = fmaxf(fmaf(S.th[kOW1 + i], x, S.th[kOB1 + i]), 0.f);
    float out = S.th[kOB3];
    for (int j = 0; j < kH; ++j) {
      float a = S.th[kOB2 + j];
#pragma unroll 8
      for (int i = 0; i < kH; ++i) a = fmaf(h1[i], S.th[kOW2 + i * kH + j], a);
      const float h = fmaxf(a, 0.f);
      h2[j] = h;
      out = fmaf(h, S.th[kOW3 + j], out);
    }
    const float dy = inv * (out - S.y[tid]);
    S.dy[tid] = dy;
#pragma unroll 8
    for (int j = 0; j < kH; ++j) dz2[j] = h2[j] > 0.f ? dy * S.th[kOW3 + j] : 0.f;
    for (int i = 0; i < kH; ++i) {
      float a = 0.f;
#pragma unroll 8
      for (int j = 0; j < kH; ++j) a = fmaf(S.th[kOW2 + i * kH + j], dz2[j], a);
      dz1[i] = h1[i] > 0.f ? a : 0.f;
    }
  }
  __syncthreads();
  // one parameter per thread, batch summed in row order
  for (int p = tid; p < kNP; p += kMT) {
    float a = 0.f;
    if (p == kOB3) {
      for (int b = 0; b < n; ++b) a += S.dy[b];
    } else if (p < kOB1) {
      const int i = p - kOW1;
      for (int b = 0; b < n; ++b) a = fmaf(S.x[b], S.dz1[b][i], a);
    } else if (p < kOW2) {
      const int i = p - kOB1;
      for (int b = 0; b < n; ++b) a += S.dz1[b][i];
    } else if (p < kOB2) {
      const int i = (p - kOW2) / kH, j = (p - kOW2) % kH;
      for (int b = 0; b < n; ++b) a = fmaf(S.h1[b][i], S.dz2[b][j], a);
    } else if (p < kOW3) {
      const int j = p - kOB2;
      for (int b = 0; b < n; ++b) a += S.dz2[b][j];
    } else {
      const int j = p - kOW3;
      for (int b = 0; b < n; ++b) a = fmaf(S.dy[b], S.h2[b][j], a);
    }
    S.g[p] = a;
  }
  __syncthreads();
}

// x of a key on the normalised log axis
template <typename K>
__device__ __forceinline__ float norm_x(K k, K s0, double inv_l) {
  const double d = (double)k - (double)s0;
  return (float)(log2(1.0 + (d > 0 ? d : 0.0)) * inv_l);
}

template <typename K>
__global__ void __launch_bounds__(kMT, 1)
    k_mlp_train(const K* __restrict__ sorted, int64_t m, float* __restrict__ theta_io,
                int steps, float lr, uint64_t seed) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
  __shared__ float s_m[kNP], s_v[kNP];
  const int tid = threadIdx.x;
  const K s0 = sorted[0], s1 = sorted[m - 1];
  const double L = log2(1.0 + ((double)s1 - (double)s0));
  const double inv_l = L > 0 ? 1.0 / L : 0.0;
  for (int p = tid; p < kNP; p += kMT) {
    S.th[p] = theta_io[p];
    s_m[p] = 0.f;
    s_v[p] = 0.f;
  }
  __syncthreads();
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float b1t = 1.f, b2t = 1.f;
  for (int t = 1; t <= steps; ++t) {
    if (tid < kMB) {
      const uint64_t r = splitmix64(seed ^ ((uint64_t)t * kMB + (uint64_t)tid));
      const int64_t idx = (int64_t)(r % (uint64_t)m);
      S.x[tid] = norm_x<K>(sorted[idx], s0, inv_l);
      S.y[tid] = (float)((double)idx / (double)(m > 1 ? m - 1 : 1));
    }
    __syncthreads();
    mlp_batch_grad(S, kMB);
    b1t *= b1;
    b2t *= b2;
    for (int p = tid; p < kNP; p += kMT) {
      const float g = S.g[p];
      const float mm = b1 * s_m[p] + (1.f - b1) * g;
      const float vv = b2 * s_v[p] + (1.f - b2) * g * g;
      s_m[p] = mm;
      s_v[p] = vv;
      const float mh = mm / (1.f - b1t);
      const float vh = vv / (1.f - b2t);
      S.th[p] -= lr * mh / (sqrtf(vh) + eps);
    }
    __syncthreads();
  }
  for (int p = tid; p < kNP; p += kMT) theta_io[p] = S.th[p];
}

// Gradient of one given batch (used to check the backward pass).
__global__ void __launch_bounds__(kMT, 1)
    k_mlp_grad(const float* __restrict__ theta, const float* __restrict__ x,
               const float* __restrict__ y, int n, float* __restrict__ grad) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
  for (int p = threadIdx.x; p < kNP; p += kMT) S.th[p] = theta[p];
  if (threadIdx.x < n) {
    S.x[threadIdx.x] = x[threadIdx.x];
    S.y[threadIdx.x] = y[threadIdx.x];
  }
  __syncthreads();
  mlp_batch_grad(S, n);
  for (int p = threadIdx.x; p < kNP; p += kMT) grad[p] = S.g[p];
}

// One Adam update of a parameter vector (used to check the optimiser step).
__global__ void k_adam(float* theta, float* m, float* v, const float* g, int n, int t, float lr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float mm = b1 * m[p] + (1.f - b1) * g[p];
  const float vv = b2 * v[p] + (1.f - b2) * g[p] * g[p];
  m[p] = mm;
  v[p] = vv;
  const float mh = mm / (1.f - powf(b1, (float)t));
  const float vh = vv / (1.f - powf(b2, (float)t));
  theta[p] -= lr * mh / (sqrtf(vh) + eps);
}

// Monotone tabulation: table[u] = max_{u' <= u} clip(f(u' / T), 0, 1).
__global__ void __launch_bounds__(1024) k_mlp_table(const float* __restrict__ theta, int T,
                                                    float* __restrict__ table) {
  __shared__ float th[kNP];
  __shared__ float s_run[33];
  for (int p = threadIdx.x; p < kNP; p += blockDim.x) th[p] = theta[p];
  __syncthreads();
  float carry = 0.f;
  for (int base = 0; base <= T; base += blockDim.x) {
    const int u = base + threadIdx.x;
    float yv = 0.f;
    if (u <= T) {
      const float x = (float)u / (float)T;
      float h1[kH];
#pragma unroll
      for (int i = 0; i < kH; ++i) h1[i] = fmaxf(fmaf(th[kOW1 + i], x, th[kOB1 + i]), 0.f);
      float out = th[kOB3];
      for (int j = 0; j < kH; ++j) {
        float a = th[kOB2 + j];
#pragma unroll
        for (int i = 0; i < kH; ++i) a = fmaf(h1[i], th[kOW2 + i * kH + j], a);
        out = fmaf(fmaxf(a, 0.f), th[kOW3 + j], out);
      }
      yv = fminf(fmaxf(out, 0.f), 1.f);
    }
    // inclusive running max over the block, then over the blocks
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float x2 = yv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float z = __shfl_up_sync(0xFFFFFFFFu, x2, o);
      if (lane >= o) x2 = fmaxf(x2, z);
    }
    if (lane == 31) s_run[warp] = x2;
    __syncthreads();
    float pre = carry;
    for (int w2 = 0; w2 < warp; ++w2) pre = fmaxf(pre, s_run[w2]);
    const float v = fmaxf(pre, x2);
    if (u <= T) table[u] = v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_run[32] = v;
    __syncthreads();
    carry = s_run[32];
    __syncthreads();
  }
}

// B_p = key of the first grid point whose tabulated CDF reaches p / P.
template <typename K>
__global__ void k_table_boundaries(const float* __restrict__ table, int T, int parts,
                                   const K* __restrict__ sorted, int64_t m, K* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (p >= parts) return;
  const float target = (float)p / (float)parts;
  int lo = 0, hi = T + 1;  // first u with table[u] >= target (T + 1 if none)
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (table[mid] >= target)
      hi = mid;
    else
      lo = mid + 1;
  }
  const K s0 = sorted[0], s1 = sorted[m - 1];
  const double L = log2(1.0 + ((double)s1 - (double)s0));
  const double x = (double)min(lo, T) / (double)T;
  const double k = (double)s0 + (exp2(x * L) - 1.0);
  K key;
  if (k >= (double)s1)
    key = s1;
  else if (k <= (double)s0)
    key = s0;
  else
    key = (K)ceil(k);
  if (key > s1) key = s1;
  out[p - 1] = key;
}

size_t mlp_smem_bytes() { return sizeof(MlpSmem); }

cudaError_t mlp_init_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_mlp_train<int32_t>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(MlpSmem));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_mlp_train<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(MlpSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(MlpSmem));
}

template <typename K>
cudaError_t launch_mlp_train(const K* sorted, int64_t m, float* theta, int steps, float lr,
                             uint64_t seed, cudaStream_t st) {
  k_mlp_train<K><<<1, kMT, sizeof(MlpSmem), st>>>(sorted, m, theta, steps, lr, seed);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float* theta, const float* x, const float* y, int n,
                            float* grad, cudaStream_t st) {
  k_mlp_grad<<<1, kMT, sizeof(MlpSmem), st>>>(theta, x, y, n, grad);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* theta, float* m, float* v, const float* g, int n, int t, float lr,
                        cudaStream_t st) {
  k_adam<<<(n + 255) / 256, 256, 0, st>>>(theta, m, v, g, n, t, lr);
  return cudaGetLastError();
}

template <typename K>
cudaError_t launch_mlp_boundaries(const float* theta, int T, float* table, int parts,
                                  const K* sorted, int64_t m, K* out, cudaStream_t st) {
  k_mlp_table<<<1, 1024, 0, st>>>(theta, T, table);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_table_boundaries<K><<<(parts + 255) / 256, 256, 0, st>>>(table, T, parts, sorted, m, out);
  return cudaGetLastError();
}

#define TJ_INSTANTIATE_MLP(K)                                                                    \
  template cudaError_t launch_mlp_train<K>(const K*, int64_t, float*, int, float, uint64_t,      \
                                           cudaStream_t);                                        \
  template cudaError_t launch_mlp_boundaries<K>(const float*, int, float*, int, const K*, int64_t, \
                                                K*, cudaStream_t);
TJ_INSTANTIATE_MLP(int32_t)
TJ_INSTANTIATE_MLP(int64_t)

}  // namespace tj
