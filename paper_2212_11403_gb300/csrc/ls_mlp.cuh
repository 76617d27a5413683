// ls_mlp.cuh -- training kernels of the donor-proposal MLP (FP32 master weights).
//
// Network: 8 inputs (7 window match fractions, one zero slot) -> 256 -> 256 -> 1, ReLU between
// layers.  Loss: half mean squared error between the score and the label.  The kernels are plain
// FP32: a tiled GEMM with optional transposes and accumulation, bias/activation epilogues, column
// sums and the Adam update.  Inference uses the BF16 MMA kernel of ls_propose.cuh.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lsk {

constexpr int kMlpIn = 8;
// packed parameter vector (host and device FP32): W1 [8][256] (input x unit), b1 [256],
// W2 [256][256], b2 [256], w3 [256], b3
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpIn * 256;
constexpr int kOffW2 = kOffB1 + 256;
constexpr int kOffB2 = kOffW2 + 256 * 256;
constexpr int kOffW3 = kOffB2 + 256;
constexpr int kOffB3 = kOffW3 + 256;
constexpr int kMlpParams = kOffB3 + 1;

// C[M][N] = beta * C + sum_k A(m, k) B(k, n), A(m, k) = ta ? A[k*lda + m] : A[m*lda + k],
// B(k, n) = tb ? B[n*ldb + k] : B[k*ldb + n].  16 x 16 tiles, 256 threads.
__global__ void gemm_f32_kernel(int M, int N, int K, const float* __restrict__ A, int lda, int ta,
                                const float* __restrict__ B, int ldb, int tb, float* __restrict__ Cm, int ldc,
                                float beta) {
  __shared__ float As[16][17], Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m = blockIdx.y * 16 + ty, n = blockIdx.x * 16 + tx;
  float acc = 0.0f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    {
      const int mm = blockIdx.y * 16 + ty, kk = k0 + tx;
      As[ty][tx] = (mm < M && kk < K) ? (ta ? A[(size_t)kk * lda + mm] : A[(size_t)mm * lda + kk]) : 0.0f;
      const int kb = k0 + ty, nn = blockIdx.x * 16 + tx;
      Bs[ty][tx] = (kb < K && nn < N) ? (tb ? B[(size_t)nn * ldb + kb] : B[(size_t)kb * ldb + nn]) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fmaf(As[ty][k], Bs[k][tx], acc);
    __syncthreads();
  }
  if (m < M && n < N) {
    float* c = Cm + (size_t)m * ldc + n;
    *c = beta == 0.0f ? acc : fmaf(beta, *c, acc);
  }
}

// Z[r][c] += b[c]; H = relu(Z) (H may alias nothing; Z keeps the pre-activation)
__global__ void bias_relu_kernel(float* __restrict__ Z, const float* __restrict__ b, int rows, int cols,
                                 float* __restrict__ H) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const float z = Z[e] + b[e % cols];
  Z[e] = z;
  if (H) H[e] = fmaxf(z, 0.0f);
}

// dZ = dH * (Z > 0), in place on dH
__global__ void relu_back_kernel(float* __restrict__ dH, const float* __restrict__ Z, long long n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n && !(Z[e] > 0.0f)) dH[e] = 0.0f;
}

// s = H2 w3 + b3 per row; ds = (s - y) / n; loss terms (s - y)^2 / 2 summed into loss (FP64 atomics
// are avoided: one partial per block)
__global__ void head_kernel(const float* __restrict__ H2, const float* __restrict__ w3, const float* __restrict__ b3,
                            const float* __restrict__ y, int n, float* __restrict__ ds, double* __restrict__ part) {
  __shared__ double red[256];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (r < n) {
    float s = b3[0];
    for (int c = 0; c < 256; ++c) s = fmaf(H2[(size_t)r * 256 + c], w3[c], s);
    const float d = s - y[r];
    ds[r] = d / (float)n;
    l = 0.5 * (double)d * (double)d;
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// dH2[r][c] = ds[r] w3[c]
__global__ void outer_kernel(const float* __restrict__ ds, const float* __restrict__ w3, int n, float* __restrict__ dH) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (long long)n * 256) dH[e] = ds[e / 256] * w3[e % 256];
}

// out[c] = sum_r X[r][c] (column sums, fixed order per column), one thread per column
__global__ void colsum_kernel(const float* __restrict__ X, int rows, int cols, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0;
  for (int r = 0; r < rows; ++r) s += X[(size_t)r * cols + c];
  out[c] = (float)s;
}

// Adam: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr * mhat / (sqrt(vhat) + eps)
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float c1, float c2, float eps) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.0f - b1) * gi;
  const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// gather a minibatch: rows sel[r] of X ([n][8]) and y
__global__ void gather_rows_kernel(const float* __restrict__ X, const float* __restrict__ y, const int* __restrict__ sel,
                                   int B, float* __restrict__ Xb, float* __restrict__ yb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * kMlpIn) return;
  const int r = e / kMlpIn, c = e % kMlpIn;
  Xb[e] = X[(size_t)sel[r] * kMlpIn + c];
  if (c == 0) yb[r] = y[sel[r]];
}

}  // namespace lsk
