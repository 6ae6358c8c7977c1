// The MLP key-CDF model of the learned partitioner (no counterpart in the
// paper): a 1 -> 32 -> 32 -> 1 ReLU network on x = log2(1 + k - s_0) /
// log2(1 + s_{m-1} - s_0), fitted to the empirical CDF of a sorted key sample
// (y_j = j / (m - 1)) by mean squared error with Adam, entirely on the device.
//
// Parameters (1153 fp32, flat): [b3 | w1(32) | b1(32) | W2(32x32, row i = from
// hidden-1 unit i) | b2(32) | w3(32)].
//
// One CTA of 512 threads runs the whole training.  Each step draws a batch of
// up to 256 sample rows with a counter-based generator (splitmix64 of seed,
// step, row) and runs the forward and backward pass one sample per thread,
// the activations in registers and the weights read from shared memory as
// 16-byte broadcasts.  The activations then go to shared memory feature by
// feature, and every parameter's gradient is summed over the batch in a
// fixed order (the 32 x 32 layer: two weights a thread, four rows per
// 16-byte load); Adam updates the parameters in place.
// The network is then tabulated on a grid of the normalised axis and made
// monotone by a running maximum; partition boundaries are read off the table.
#include <math.h>

#include "tj_internal.cuh"

namespace tj {

constexpr int kH = 32;
constexpr int kNP = 1 + kH + kH + kH * kH + kH + kH;  // 1153
constexpr int kMB = 256;                               // batch rows per step, at most
constexpr int kMT = 512;                               // threads of the training CTA
// offsets in the flat parameter vector (the layout of the C interface)
constexpr int kOB3 = 0, kOW1 = 1, kOB1 = 1 + kH, kOW2 = 1 + 2 * kH, kOB2 = 1 + 2 * kH + kH * kH,
              kOW3 = 1 + 3 * kH + kH * kH;

// The parameters as the kernels keep them: every vector 16-byte aligned.
// Flat index p >= 1 is net index p - 1; b3 (p = 0) is net index kH * kH + 4 kH.
struct __align__(16) Net {
  float w1[kH];
  float b1[kH];
  float W2[kH][kH];  // row i: from hidden-1 unit i
  float b2[kH];
  float w3[kH];
  float b3;
  float pad[3];
};
constexpr int kNetB3 = kH * kH + 4 * kH;  // 1152
static_assert(sizeof(Net) == (kNetB3 + 4) * sizeof(float), "Net is packed");
__device__ __forceinline__ int net_index(int p) { return p == 0 ? kNetB3 : p - 1; }
__device__ __forceinline__ float* net_at(Net& n, int q) { return reinterpret_cast<float*>(&n) + q; }

// per-feature rows of the batch's activations, padded so that the rows of
// eight consecutive features start in distinct 16-byte bank groups
constexpr int kBP = kMB + 4;
struct MlpSmem {
  Net th;  // parameters
  Net g;   // gradient of the batch
  Net m, v;  // Adam moments (training only)
  float x[kMB], y[kMB], dy[kMB];
  float wloss[kMT / 32];  // per warp: the batch's squared errors
  float a1[kH][kBP];  // hidden-1 outputs
  float d1[kH][kBP];  // their gradients (pre-activation)
  float a2[kH][kBP];  // hidden-2 outputs
  float d2[kH][kBP];  // their gradients (pre-activation)
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
  float e2 = 0.f;  // this row's squared error
  if (tid < n) {
    const float x = S.x[tid];
    const float4* w1 = reinterpret_cast<const float4*>(S.th.w1);
    const float4* b1 = reinterpret_cast<const float4*>(S.th.b1);
    const float4* b2 = reinterpret_cast<const float4*>(S.th.b2);
    const float4* w3 = reinterpret_cast<const float4*>(S.th.w3);
    float h1[kH], a[kH];
#pragma unroll
    for (int q = 0; q < kH / 4; ++q) {
      const float4 w = w1[q], b = b1[q], c = b2[q];
      h1[4 * q + 0] = fmaxf(fmaf(w.x, x, b.x), 0.f);
      h1[4 * q + 1] = fmaxf(fmaf(w.y, x, b.y), 0.f);
      h1[4 * q + 2] = fmaxf(fmaf(w.z, x, b.z), 0.f);
      h1[4 * q + 3] = fmaxf(fmaf(w.w, x, b.w), 0.f);
      a[4 * q + 0] = c.x;
      a[4 * q + 1] = c.y;
      a[4 * q + 2] = c.z;
      a[4 * q + 3] = c.w;
    }
    // hidden 2: a_j = b2_j + Sum_i h1_i W2[i][j], row i read as 8 broadcasts
#pragma unroll
    for (int i = 0; i < kH; ++i) {
      const float4* row = reinterpret_cast<const float4*>(S.th.W2[i]);
      const float hi = h1[i];
#pragma unroll
      for (int q = 0; q < kH / 4; ++q) {
        const float4 w = row[q];
        a[4 * q + 0] = fmaf(hi, w.x, a[4 * q + 0]);
        a[4 * q + 1] = fmaf(hi, w.y, a[4 * q + 1]);
        a[4 * q + 2] = fmaf(hi, w.z, a[4 * q + 2]);
        a[4 * q + 3] = fmaf(hi, w.w, a[4 * q + 3]);
      }
    }
    float out = S.th.b3;
#pragma unroll
    for (int q = 0; q < kH / 4; ++q) {
      const float4 w = w3[q];
      a[4 * q + 0] = fmaxf(a[4 * q + 0], 0.f);
      a[4 * q + 1] = fmaxf(a[4 * q + 1], 0.f);
      a[4 * q + 2] = fmaxf(a[4 * q + 2], 0.f);
      a[4 * q + 3] = fmaxf(a[4 * q + 3], 0.f);
      out = fmaf(a[4 * q + 0], w.x, out);
      out = fmaf(a[4 * q + 1], w.y, out);
      out = fmaf(a[4 * q + 2], w.z, out);
      out = fmaf(a[4 * q + 3], w.w, out);
    }
    const float err = out - S.y[tid];
    const float dy = inv * err;
    S.dy[tid] = dy;
    e2 = err * err;
    // hidden 2 outputs, then their gradients in place
#pragma unroll
    for (int q = 0; q < kH / 4; ++q) {
      const float4 w = w3[q];
      const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = 4 * q + e;
        S.a2[j][tid] = a[j];
        a[j] = a[j] > 0.f ? dy * wv[e] : 0.f;
        S.d2[j][tid] = a[j];
      }
    }
    // hidden 1 gradients: Sum_j W2[i][j] dz2_j where h1_i > 0 (W2 is read
    // again, not kept in registers from the forward pass)
    asm volatile("" ::: "memory");
#pragma unroll
    for (int i = 0; i < kH; ++i) {
      const float4* row = reinterpret_cast<const float4*>(S.th.W2[i]);
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < kH / 4; ++q) {
        const float4 w = row[q];
        acc = fmaf(w.x, a[4 * q + 0], acc);
        acc = fmaf(w.y, a[4 * q + 1], acc);
        acc = fmaf(w.z, a[4 * q + 2], acc);
        acc = fmaf(w.w, a[4 * q + 3], acc);
      }
      S.a1[i][tid] = h1[i];
      S.d1[i][tid] = h1[i] > 0.f ? acc : 0.f;
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) e2 += __shfl_xor_sync(0xFFFFFFFFu, e2, o);
  if ((tid & 31) == 0) S.wloss[tid >> 5] = e2;
  __syncthreads();
  // Sums over the batch, rows in order.  Thread (i0 = warp, j = lane): W2
  // gradients [i0][j] and [i0 + 16][j]; besides, warp 0 sums b2[j], warp 1
  // w3[j], warp 2 w1[j] and b1[j], warp 3 (lane 0) b3.
  {
    const int j = tid & 31, i0 = tid >> 5;
    const float4* D2 = reinterpret_cast<const float4*>(S.d2[j]);
    const float4* A0 = reinterpret_cast<const float4*>(S.a1[i0]);
    const float4* A1 = reinterpret_cast<const float4*>(S.a1[i0 + 16]);
    const float4* A2 = reinterpret_cast<const float4*>(S.a2[j]);
    const float4* D1 = reinterpret_cast<const float4*>(S.d1[j]);
    const float4* X = reinterpret_cast<const float4*>(S.x);
    const float4* DY = reinterpret_cast<const float4*>(S.dy);
    float g0 = 0.f, g1 = 0.f, e0 = 0.f, e1 = 0.f;
    const int n4 = n >> 2;
    for (int c = 0; c < n4; ++c) {
      const float4 d = D2[c], p = A0[c], q = A1[c];
      g0 = fmaf(p.x, d.x, g0);
      g0 = fmaf(p.y, d.y, g0);
      g0 = fmaf(p.z, d.z, g0);
      g0 = fmaf(p.w, d.w, g0);
      g1 = fmaf(q.x, d.x, g1);
      g1 = fmaf(q.y, d.y, g1);
      g1 = fmaf(q.z, d.z, g1);
      g1 = fmaf(q.w, d.w, g1);
      if (i0 == 0) {
        e0 += d.x;
        e0 += d.y;
        e0 += d.z;
        e0 += d.w;
      } else if (i0 == 1) {
        const float4 h = A2[c], t = DY[c];
        e0 = fmaf(t.x, h.x, e0);
        e0 = fmaf(t.y, h.y, e0);
        e0 = fmaf(t.z, h.z, e0);
        e0 = fmaf(t.w, h.w, e0);
      } else if (i0 == 2) {
        const float4 h = D1[c], t = X[c];
        e0 = fmaf(t.x, h.x, e0);
        e0 = fmaf(t.y, h.y, e0);
        e0 = fmaf(t.z, h.z, e0);
        e0 = fmaf(t.w, h.w, e0);
        e1 += h.x;
        e1 += h.y;
        e1 += h.z;
        e1 += h.w;
      } else if (i0 == 3 && j == 0) {
        const float4 t = DY[c];
        e0 += t.x;
        e0 += t.y;
        e0 += t.z;
        e0 += t.w;
      }
    }
    for (int b = 4 * n4; b < n; ++b) {
      const float d = S.d2[j][b];
      g0 = fmaf(S.a1[i0][b], d, g0);
      g1 = fmaf(S.a1[i0 + 16][b], d, g1);
      if (i0 == 0) {
        e0 += d;
      } else if (i0 == 1) {
        e0 = fmaf(S.dy[b], S.a2[j][b], e0);
      } else if (i0 == 2) {
        e0 = fmaf(S.x[b], S.d1[j][b], e0);
        e1 += S.d1[j][b];
      } else if (i0 == 3 && j == 0) {
        e0 += S.dy[b];
      }
    }
    S.g.W2[i0][j] = g0;
    S.g.W2[i0 + 16][j] = g1;
    if (i0 == 0) S.g.b2[j] = e0;
    if (i0 == 1) S.g.w3[j] = e0;
    if (i0 == 2) {
      S.g.w1[j] = e0;
      S.g.b1[j] = e1;
    }
    if (i0 == 3 && j == 0) S.g.b3 = e0;
  }
  __syncthreads();
}

// x of a key on the normalised log axis
template <typename K>
__device__ __forceinline__ float norm_x(K k, K s0, double inv_l) {
  const double d = (double)k - (double)s0;
  return (float)(log2(1.0 + (d > 0 ? d : 0.0)) * inv_l);
}

// Training stops early once the loss has levelled off: an exponential moving
// average of the batches' mean squared error (weight 1/10 per step), compared
// every kCheck steps with its value 2 kCheck steps before; less than
// kMinGain relative improvement ends the training (not before 3 kCheck
// steps).  Every thread computes the same average, so all stop together.
constexpr int kCheck = 50;
constexpr float kMinGain = 0.02f;

template <typename K>
__global__ void __launch_bounds__(kMT, 1)
    k_mlp_train(const K* __restrict__ sorted, int64_t m, float* __restrict__ theta_io,
                int steps, int batch, float lr, uint64_t seed, int* __restrict__ steps_run) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const K s0 = sorted[0], s1 = sorted[m - 1];
  const double L = log2(1.0 + ((double)s1 - (double)s0));
  const double inv_l = L > 0 ? 1.0 / L : 0.0;
  for (int p = tid; p < kNP; p += kMT) {
    const int q = net_index(p);
    *net_at(S.th, q) = theta_io[p];
    *net_at(S.m, q) = 0.f;
    *net_at(S.v, q) = 0.f;
  }
  __syncthreads();
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float b1t = 1.f, b2t = 1.f;
  float ema = 0.f, ema1 = 0.f, ema2 = 0.f;  // now, kCheck and 2 kCheck steps ago
  int t = 1;
  for (; t <= steps; ++t) {
    if (tid < batch) {
      const uint64_t r = splitmix64(seed ^ ((uint64_t)t * kMB + (uint64_t)tid));
      const int64_t idx = (int64_t)(r % (uint64_t)m);
      S.x[tid] = norm_x<K>(sorted[idx], s0, inv_l);
      S.y[tid] = (float)((double)idx / (double)(m > 1 ? m - 1 : 1));
    }
    __syncthreads();
    mlp_batch_grad(S, batch);
    {
      float l = 0.f;
#pragma unroll
      for (int w = 0; w < kMT / 32; ++w) l += S.wloss[w];
      l /= (float)batch;
      ema = t == 1 ? l : 0.9f * ema + 0.1f * l;
    }
    b1t *= b1;
    b2t *= b2;
    for (int q = tid; q < kNP; q += kMT) {
      const float g = *net_at(S.g, q);
      const float mm = b1 * *net_at(S.m, q) + (1.f - b1) * g;
      const float vv = b2 * *net_at(S.v, q) + (1.f - b2) * g * g;
      *net_at(S.m, q) = mm;
      *net_at(S.v, q) = vv;
      const float mh = mm / (1.f - b1t);
      const float vh = vv / (1.f - b2t);
      *net_at(S.th, q) -= lr * mh / (sqrtf(vh) + eps);
    }
    __syncthreads();
    if (t % kCheck == 0) {
      if (t >= 3 * kCheck && ema > (1.f - kMinGain) * ema2) {
        ++t;
        break;
      }
      ema2 = ema1;
      ema1 = ema;
    }
  }
  for (int p = tid; p < kNP; p += kMT) theta_io[p] = *net_at(S.th, net_index(p));
  if (tid == 0 && steps_run) *steps_run = t - 1;
}

// Gradient of one given batch (used to check the backward pass).
__global__ void __launch_bounds__(kMT, 1)
    k_mlp_grad(const float* __restrict__ theta, const float* __restrict__ x,
               const float* __restrict__ y, int n, float* __restrict__ grad) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
  for (int p = threadIdx.x; p < kNP; p += kMT) *net_at(S.th, net_index(p)) = theta[p];
  if (threadIdx.x < n) {
    S.x[threadIdx.x] = x[threadIdx.x];
    S.y[threadIdx.x] = y[threadIdx.x];
  }
  __syncthreads();
  mlp_batch_grad(S, n);
  for (int p = threadIdx.x; p < kNP; p += kMT) grad[p] = *net_at(S.g, net_index(p));
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
cudaError_t launch_mlp_train(const K* sorted, int64_t m, float* theta, int steps, int batch,
                             float lr, uint64_t seed, int* steps_run, cudaStream_t st) {
  if (batch < 1 || batch > kMB) return cudaErrorInvalidValue;
  k_mlp_train<K><<<1, kMT, sizeof(MlpSmem), st>>>(sorted, m, theta, steps, batch, lr, seed,
                                                   steps_run);
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
  template cudaError_t launch_mlp_train<K>(const K*, int64_t, float*, int, int, float, uint64_t, \
                                           int*, cudaStream_t);                                  \
  template cudaError_t launch_mlp_boundaries<K>(const float*, int, float*, int, const K*, int64_t, \
                                                K*, cudaStream_t);
TJ_INSTANTIATE_MLP(int32_t)
TJ_INSTANTIATE_MLP(int64_t)

}  // namespace tj
