// Learned per-vertex work model: a 4 -> 32 -> 32 -> 1 multilayer perceptron
// (ReLU, FP32) predicting log2 of the cycles the per-root pass spends on a
// root, from log2(1 + x) of four per-vertex features: DAG out-degree d+(u),
// neighbour degree sum sum_{v in N(u)} d(v) (the wedges rooted at u), sum
// over out-neighbours of their out-degree, and T(u).  Its
// prediction orders the persistent root queue (largest first); the counts
// themselves never depend on it.  The paper has no such model: it schedules
// nothing.
//
// Parameter vector (1249 floats): W1[32][4], b1[32], W2[32][32], b2[32],
// W3[32], b3.  Loss: mean squared error over the samples of a batch.
#include "evoke_internal.cuh"

namespace {

constexpr int kIn = 4, kH = 32;
constexpr int kOW1 = 0, kOB1 = kOW1 + kH * kIn, kOW2 = kOB1 + kH, kOB2 = kOW2 + kH * kH,
              kOW3 = kOB2 + kH, kOB3 = kOW3 + kH, kNP = kOB3 + 1;
static_assert(kNP == 1249, "parameter count");
constexpr int kFwdThreads = 256;
constexpr int kGradThreads = 64;  // keeps the staged activations under 48 KB

__device__ __forceinline__ float lg(float x) { return log2f(1.0f + x); }

// features of every vertex (needs T(u), i.e. after the triangle passes)
__global__ void features_kernel(Graph g, const u64* __restrict__ acc, float* __restrict__ X) {
  const u32 u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= g.n) return;
  const u32 b = g.dag_ptr[u], e = g.dag_ptr[u + 1];
  u64 s = 0;
  for (u32 p = b; p < e; ++p) {
    const u32 v = g.dag_col[p];
    s += g.dag_ptr[v + 1] - g.dag_ptr[v];
  }
  X[(u64)u * 4 + 0] = lg((float)(e - b));
  X[(u64)u * 4 + 1] = lg((float)acc[(u64)A_WORK * g.n + u]);
  X[(u64)u * 4 + 2] = lg((float)s);
  X[(u64)u * 4 + 3] = lg((float)acc[(u64)A_T * g.n + u]);
}

__device__ __forceinline__ float mlp_one(const float* p, const float* x, float* h1, float* h2) {
#pragma unroll
  for (int i = 0; i < kH; ++i) {
    float z = p[kOB1 + i];
#pragma unroll
    for (int j = 0; j < kIn; ++j) z = fmaf(p[kOW1 + i * kIn + j], x[j], z);
    h1[i] = fmaxf(z, 0.0f);
  }
#pragma unroll 4
  for (int i = 0; i < kH; ++i) {
    float z = p[kOB2 + i];
#pragma unroll
    for (int j = 0; j < kH; ++j) z = fmaf(p[kOW2 + i * kH + j], h1[j], z);
    h2[i] = fmaxf(z, 0.0f);
  }
  float y = p[kOB3];
#pragma unroll
  for (int j = 0; j < kH; ++j) y = fmaf(p[kOW3 + j], h2[j], y);
  return y;
}

__global__ void __launch_bounds__(kFwdThreads)
forward_kernel(const float* __restrict__ X, u32 N, const float* __restrict__ params,
               float* __restrict__ y) {
  __shared__ float p[kNP];
  for (int i = threadIdx.x; i < kNP; i += blockDim.x) p[i] = params[i];
  __syncthreads();
  const u32 k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  float x[kIn], h1[kH], h2[kH];
#pragma unroll
  for (int j = 0; j < kIn; ++j) x[j] = X[(u64)k * kIn + j];
  y[k] = mlp_one(p, x, h1, h2);
}

// Gradient of the mean squared error over samples [lo, lo+cnt) (indices into
// X, y through `idx` if given).  Each block stages its samples' activations
// and back-propagated errors in shared memory and forms the weight gradients
// as sums over its samples; one atomic add per parameter per block.
__global__ void __launch_bounds__(kGradThreads)
grad_kernel(const float* __restrict__ X, const float* __restrict__ T, const u32* __restrict__ idx,
            u32 lo, u32 cnt, const float* __restrict__ params, float* __restrict__ grad,
            float* __restrict__ loss) {
  __shared__ float p[kNP];
  __shared__ float sx[kGradThreads][kIn];
  __shared__ float sh1[kGradThreads][kH + 1];
  __shared__ float sh2[kGradThreads][kH + 1];
  __shared__ float sd2[kGradThreads][kH + 1];
  __shared__ float sd1[kGradThreads][kH + 1];
  __shared__ float sdy[kGradThreads];
  for (int i = threadIdx.x; i < kNP; i += blockDim.x) p[i] = params[i];
  __syncthreads();
  const u32 r = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = r < cnt;
  const float inv = 1.0f / (float)cnt;
  float x[kIn], h1[kH], h2[kH];
  float dy = 0.0f;
  if (valid) {
    const u32 k = idx ? idx[lo + r] : lo + r;
#pragma unroll
    for (int j = 0; j < kIn; ++j) x[j] = X[(u64)k * kIn + j];
    const float yv = mlp_one(p, x, h1, h2);
    const float e = yv - T[k];
    dy = 2.0f * e * inv;
    atomicAdd(loss, e * e * inv);
  } else {
#pragma unroll
    for (int j = 0; j < kIn; ++j) x[j] = 0.0f;
#pragma unroll
    for (int j = 0; j < kH; ++j) h1[j] = h2[j] = 0.0f;
  }
  // back-propagate through the two hidden layers
  float d2[kH], d1[kH];
#pragma unroll
  for (int j = 0; j < kH; ++j) d2[j] = (h2[j] > 0.0f) ? dy * p[kOW3 + j] : 0.0f;
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kH; ++i) s = fmaf(p[kOW2 + i * kH + j], d2[i], s);
    d1[j] = (h1[j] > 0.0f) ? s : 0.0f;
  }
  const int t = threadIdx.x;
#pragma unroll
  for (int j = 0; j < kIn; ++j) sx[t][j] = x[j];
#pragma unroll
  for (int j = 0; j < kH; ++j) {
    sh1[t][j] = h1[j];
    sh2[t][j] = h2[j];
    sd2[t][j] = d2[j];
    sd1[t][j] = d1[j];
  }
  sdy[t] = dy;
  __syncthreads();
  const int B = kGradThreads;
  // W2 (32 x 32): dW2[i][j] = sum_s d2[s][i] h1[s][j]
  for (int q = t; q < kH * kH; q += B) {
    const int i = q / kH, j = q % kH;
    float s = 0.0f;
    for (int k = 0; k < B; ++k) s = fmaf(sd2[k][i], sh1[k][j], s);
    if (s != 0.0f) atomicAdd(&grad[kOW2 + q], s);
  }
  // W1 (32 x 4), b1, b2, W3, b3
  for (int q = t; q < kH * kIn + 3 * kH + 1; q += B) {
    float s = 0.0f;
    if (q < kH * kIn) {
      const int i = q / kIn, j = q % kIn;
      for (int k = 0; k < B; ++k) s = fmaf(sd1[k][i], sx[k][j], s);
      if (s != 0.0f) atomicAdd(&grad[kOW1 + q], s);
    } else if (q < kH * kIn + kH) {
      const int i = q - kH * kIn;
      for (int k = 0; k < B; ++k) s += sd1[k][i];
      if (s != 0.0f) atomicAdd(&grad[kOB1 + i], s);
    } else if (q < kH * kIn + 2 * kH) {
      const int i = q - kH * kIn - kH;
      for (int k = 0; k < B; ++k) s += sd2[k][i];
      if (s != 0.0f) atomicAdd(&grad[kOB2 + i], s);
    } else if (q < kH * kIn + 3 * kH) {
      const int j = q - kH * kIn - 2 * kH;
      for (int k = 0; k < B; ++k) s = fmaf(sdy[k], sh2[k][j], s);
      if (s != 0.0f) atomicAdd(&grad[kOW3 + j], s);
    } else {
      for (int k = 0; k < B; ++k) s += sdy[k];
      if (s != 0.0f) atomicAdd(&grad[kOB3], s);
    }
  }
}

// Adam (Kingma & Ba) with bias correction; state = [m(1249), v(1249)]
__global__ void adam_kernel(float* __restrict__ params, const float* __restrict__ grad,
                            float* __restrict__ state, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNP) return;
  const float gi = grad[i];
  float m = state[i] = b1 * state[i] + (1.0f - b1) * gi;
  float v = state[kNP + i] = b2 * state[kNP + i] + (1.0f - b2) * gi * gi;
  const float mh = m / c1, vh = v / c2;
  params[i] -= lr * mh / (sqrtf(vh) + eps);
}

// priorities -> the persistent queue order: 256 buckets over log2 cycles,
// largest predicted cost first
__device__ __forceinline__ u32 prio_bucket(float y) {
  float b = y * 8.0f;
  b = fminf(fmaxf(b, 0.0f), 255.0f);
  return 255u - (u32)b;
}
__global__ void prio_hist_kernel(const float* __restrict__ y, u32 n, u32* cnt) {
  const u32 u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) atomicAdd(&cnt[prio_bucket(y[u])], 1u);
}
__global__ void prio_scan_kernel(u32* cnt, u32* head) {
  u32 run = 0;
  for (int b = 0; b < 256; ++b) {
    const u32 c = cnt[b];
    cnt[b] = run;
    run += c;
  }
  *head = 0;
}
__global__ void prio_scatter_kernel(const float* __restrict__ y, u32 n, u32* cursor, u32* order) {
  const u32 u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) order[atomicAdd(&cursor[prio_bucket(y[u])], 1u)] = u;
}

}  // namespace

int mlp_param_count() { return kNP; }

void launch_features(const Graph& g, const u64* acc, float* X, cudaStream_t st) {
  if (g.n) features_kernel<<<(g.n + 255) / 256, 256, 0, st>>>(g, acc, X);
}

void launch_mlp_forward(const float* X, u32 N, const float* params, float* y, cudaStream_t st) {
  if (N) forward_kernel<<<(N + kFwdThreads - 1) / kFwdThreads, kFwdThreads, 0, st>>>(X, N, params, y);
}

void launch_mlp_grad(const float* X, const float* T, const u32* idx, u32 lo, u32 cnt,
                     const float* params, float* grad, float* loss, cudaStream_t st) {
  cudaMemsetAsync(grad, 0, sizeof(float) * kNP, st);
  if (cnt)
    grad_kernel<<<(cnt + kGradThreads - 1) / kGradThreads, kGradThreads, 0, st>>>(
        X, T, idx, lo, cnt, params, grad, loss);
}

void launch_adam(float* params, const float* grad, float* state, float lr, int step,
                 cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float c1 = 1.0f, c2 = 1.0f;
  for (int i = 0; i < step; ++i) {
    c1 *= b1;
    c2 *= b2;
  }
  adam_kernel<<<(kNP + 255) / 256, 256, 0, st>>>(params, grad, state, lr, b1, b2, eps, 1.0f - c1,
                                                 1.0f - c2);
}

void launch_priority_schedule(const float* y, u32 n, u32* bucket_cnt /*256*/, u32* head,
                              u32* order, cudaStream_t st) {
  if (!n) return;
  cudaMemsetAsync(bucket_cnt, 0, 256 * sizeof(u32), st);
  prio_hist_kernel<<<(n + 255) / 256, 256, 0, st>>>(y, n, bucket_cnt);
  prio_scan_kernel<<<1, 1, 0, st>>>(bucket_cnt, head);
  prio_scatter_kernel<<<(n + 255) / 256, 256, 0, st>>>(y, n, bucket_cnt, order);
}
