// Cost-model training kernels: a multilayer perceptron d_in -> h1 -> h2 -> V
// with ReLU hidden layers, a masked mean-squared-error loss and Adam, in FP32
// on CUDA cores (the matrices are a few thousand rows by at most a few
// hundred columns; the work is latency-bound, not a tensor-core contraction).
//
// The model predicts one log-time per kernel variant from the features of a
// call; the autotuner's measurements are its training data (the paper's
// empirical exploration of split sizes and vector widths, Sec. 6.2, and its
// model-guided search, Sec. 6.3).
//
// Parameter buffer (one contiguous fp32 array, row-major matrices):
//   W1 [d_in][h1] | b1 [h1] | W2 [h1][h2] | b2 [h2] | W3 [h2][V] | b3 [V]
// Work buffer per batch of B rows:
//   Z1 [B][h1] | H1 [B][h1] | Z2 [B][h2] | H2 [B][h2] | D0 [B][hm] | D1 [B][hm]
// with hm = max(h1, h2).
#include "lift_internal.cuh"

namespace lift {
namespace {

constexpr int kTile = 32;

// C[M][N] = op(A)[M][K] . op(B)[K][N] + bias[N] (optional), with an
// epilogue: 0 store; 1 store Z in C and relu(Z) in C2; 2 multiply by
// [gate > 0] (ReLU backward).  op(A) = A [M][K] or A^T with A [K][M].
template <bool TA, bool TB>
__global__ void __launch_bounds__(kTile * 8)
    gemm_small(int M, int N, int K, const float* __restrict__ A, const float* __restrict__ B,
               float* __restrict__ C, const float* __restrict__ bias, float* __restrict__ C2,
               const float* __restrict__ gate, int epilogue) {
  __shared__ float As[kTile][kTile + 1];
  __shared__ float Bs[kTile][kTile + 1];
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;  // 32 x 8
  const int row0 = blockIdx.y * kTile, col0 = blockIdx.x * kTile;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += kTile) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = ty + 8 * i;  // tile row
      const int gm = row0 + r, gk = k0 + tx;
      float a = 0.f;
      if (gm < M && gk < K) a = TA ? A[(size_t)gk * M + gm] : A[(size_t)gm * K + gk];
      As[r][tx] = a;
      const int bk = k0 + r, bn = col0 + tx;
      float b = 0.f;
      if (bk < K && bn < N) b = TB ? B[(size_t)bn * K + bk] : B[(size_t)bk * N + bn];
      Bs[r][tx] = b;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kTile; ++kk) {
      const float b = Bs[kk][tx];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = fmaf(As[ty + 8 * i][kk], b, acc[i]);
    }
    __syncthreads();
  }
  const int n = col0 + tx;
  if (n >= N) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = row0 + ty + 8 * i;
    if (m >= M) continue;
    float z = acc[i] + (bias ? bias[n] : 0.f);
    const size_t o = (size_t)m * N + n;
    if (epilogue == 2) z = gate[o] > 0.f ? z : 0.f;
    C[o] = z;
    if (epilogue == 1) C2[o] = z > 0.f ? z : 0.f;
  }
}

// db[j] = sum_b D[b][j]
__global__ void col_sum(int B, int N, const float* __restrict__ D, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += D[(size_t)b * N + j];
  out[j] = s;
}

// loss = sum(mask * (P - T)^2) * inv;  dP = 2 * mask * (P - T) * inv
__global__ void __launch_bounds__(1024)
    masked_mse(const float* __restrict__ P, const float* __restrict__ T, const float* __restrict__ Mk,
               int64_t count, float inv, float* __restrict__ dP, float* __restrict__ loss) {
  __shared__ float red[kWarp];
  float s = 0.f;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {
    const float d = Mk[i] > 0.f ? P[i] - T[i] : 0.f;
    dP[i] = 2.f * d * inv;
    s = fmaf(d, d, s);
  }
  s = warp_tree(s);
  const int lane = threadIdx.x & 31, w = threadIdx.x / 32;
  if (lane == 0) red[w] = s;
  __syncthreads();
  if (w == 0) {
    s = lane < (int)(blockDim.x / 32) ? red[lane] : 0.f;
    s = warp_tree(s);
    if (lane == 0) *loss = s * inv;
  }
}

__global__ void adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                     float* __restrict__ v, int64_t count, float lr, float b1, float b2, float eps,
                     float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

struct Layout {
  int64_t W1, b1, W2, b2, W3, b3, total;
  Layout(int d, int h1, int h2, int V) {
    W1 = 0;
    b1 = W1 + (int64_t)d * h1;
    W2 = b1 + h1;
    b2 = W2 + (int64_t)h1 * h2;
    W3 = b2 + h2;
    b3 = W3 + (int64_t)h2 * V;
    total = b3 + V;
  }
};

template <bool TA, bool TB>
lift_status gemm(int M, int N, int K, const float* A, const float* B, float* C, const float* bias,
                 float* C2, const float* gate, int epi, cudaStream_t s) {
  dim3 grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
  gemm_small<TA, TB><<<grid, kTile * 8, 0, s>>>(M, N, K, A, B, C, bias, C2, gate, epi);
  return cuda_check(cudaGetLastError(), "mlp gemm launch");
}

bool bad_shape(int d, int h1, int h2, int V) { return d < 1 || h1 < 1 || h2 < 1 || V < 1; }

}  // namespace
}  // namespace lift

using namespace lift;

extern "C" {

int64_t lift_mlp_param_count(int d_in, int h1, int h2, int V) {
  if (bad_shape(d_in, h1, h2, V)) return -1;
  return Layout(d_in, h1, h2, V).total;
}

int64_t lift_mlp_work_count(int64_t B, int h1, int h2) {
  if (B < 0 || h1 < 1 || h2 < 1) return -1;
  const int64_t hm = h1 > h2 ? h1 : h2;
  return B * (2 * (int64_t)h1 + 2 * (int64_t)h2 + 2 * hm);
}

lift_status lift_mlp_forward(int d_in, int h1, int h2, int V, const float* params, const float* X,
                             int64_t B, float* work, float* P, void* stream) {
  if (bad_shape(d_in, h1, h2, V) || B < 1 || !params || !X || !work || !P || B > (1 << 30))
    return set_error(LIFT_ERR_INVALID_ARG, "mlp_forward arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Layout L(d_in, h1, h2, V);
  float* Z1 = work;
  float* H1 = Z1 + B * h1;
  float* Z2 = H1 + B * h1;
  float* H2 = Z2 + B * h2;
  const int b = (int)B;
  lift_status rc = gemm<false, false>(b, h1, d_in, X, params + L.W1, Z1, params + L.b1, H1, nullptr, 1, s);
  if (rc == LIFT_OK)
    rc = gemm<false, false>(b, h2, h1, H1, params + L.W2, Z2, params + L.b2, H2, nullptr, 1, s);
  if (rc == LIFT_OK)
    rc = gemm<false, false>(b, V, h2, H2, params + L.W3, P, params + L.b3, nullptr, nullptr, 0, s);
  return rc;
}

lift_status lift_mlp_loss(const float* P, const float* T, const float* mask, int64_t count,
                          float inv_measured, float* dP, float* loss, void* stream) {
  if (count < 1 || !P || !T || !mask || !dP || !loss)
    return set_error(LIFT_ERR_INVALID_ARG, "mlp_loss arguments");
  masked_mse<<<1, 1024, 0, static_cast<cudaStream_t>(stream)>>>(P, T, mask, count, inv_measured,
                                                                 dP, loss);
  return cuda_check(cudaGetLastError(), "mlp_loss launch");
}

lift_status lift_mlp_backward(int d_in, int h1, int h2, int V, const float* params, const float* X,
                              int64_t B, float* work, const float* dP, float* grads, void* stream) {
  if (bad_shape(d_in, h1, h2, V) || B < 1 || !params || !X || !work || !dP || !grads ||
      B > (1 << 30))
    return set_error(LIFT_ERR_INVALID_ARG, "mlp_backward arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Layout L(d_in, h1, h2, V);
  const int64_t hm = h1 > h2 ? h1 : h2;
  float* Z1 = work;
  float* H1 = Z1 + B * h1;
  float* Z2 = H1 + B * h1;
  float* H2 = Z2 + B * h2;
  float* D0 = H2 + B * h2;
  float* D1 = D0 + B * hm;
  const int b = (int)B;
  // layer 3: dW3 = H2^T dP, db3 = colsum(dP), dZ2 = (dP W3^T) * [Z2 > 0]
  lift_status rc = gemm<true, false>(h2, V, b, H2, dP, grads + L.W3, nullptr, nullptr, nullptr, 0, s);
  if (rc != LIFT_OK) return rc;
  col_sum<<<(V + 127) / 128, 128, 0, s>>>(b, V, dP, grads + L.b3);
  rc = gemm<false, true>(b, h2, V, dP, params + L.W3, D0, nullptr, nullptr, Z2, 2, s);
  if (rc != LIFT_OK) return rc;
  // layer 2: dW2 = H1^T dZ2, db2 = colsum(dZ2), dZ1 = (dZ2 W2^T) * [Z1 > 0]
  rc = gemm<true, false>(h1, h2, b, H1, D0, grads + L.W2, nullptr, nullptr, nullptr, 0, s);
  if (rc != LIFT_OK) return rc;
  col_sum<<<(h2 + 127) / 128, 128, 0, s>>>(b, h2, D0, grads + L.b2);
  rc = gemm<false, true>(b, h1, h2, D0, params + L.W2, D1, nullptr, nullptr, Z1, 2, s);
  if (rc != LIFT_OK) return rc;
  // layer 1: dW1 = X^T dZ1, db1 = colsum(dZ1)
  rc = gemm<true, false>(d_in, h1, b, X, D1, grads + L.W1, nullptr, nullptr, nullptr, 0, s);
  if (rc != LIFT_OK) return rc;
  col_sum<<<(h1 + 127) / 128, 128, 0, s>>>(b, h1, D1, grads + L.b1);
  return cuda_check(cudaGetLastError(), "mlp_backward launch");
}

lift_status lift_mlp_adam(float* params, const float* grads, float* m, float* v, int64_t count, int t,
                          float lr, float beta1, float beta2, float eps, void* stream) {
  if (count < 1 || t < 1 || !params || !grads || !m || !v)
    return set_error(LIFT_ERR_INVALID_ARG, "mlp_adam arguments");
  const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
  int blocks = (int)((count + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  adam<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, grads, m, v, count, lr, beta1,
                                                               beta2, eps, c1, c2);
  return cuda_check(cudaGetLastError(), "mlp_adam launch");
}

}  // extern "C"
