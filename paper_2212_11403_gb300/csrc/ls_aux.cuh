// ls_aux.cuh -- auxiliary kernels: haplotype bit packing, posterior/half-distance from tables and
// the in-place symmetrisation of the distance matrix.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "ls_prop.cuh"

namespace lsk {

// Validation and fingerprint of a prior matrix (Sec. 2.1: Pi, recipient-major rows that sum to one
// with a zero diagonal), one CTA of 256 threads per row.  bad[i]: bit 0 a negative or non-finite
// entry, bit 1 a non-zero diagonal; sums[i]: the row sum in FP64 (thread-strided partial sums,
// added in thread order); hashes[i]: FNV-1a of each thread's entries' bytes in column order, the
// 256 thread hashes folded in thread order.  Deterministic for a given matrix.
__global__ void prior_check_kernel(const float* __restrict__ Pi, int N, int* __restrict__ bad,
                                   double* __restrict__ sums, unsigned long long* __restrict__ hashes) {
  __shared__ double ps[256];
  __shared__ unsigned long long ph[256];
  __shared__ int pb;
  const int i = blockIdx.x, tid = threadIdx.x;
  const float* row = Pi + (size_t)i * N;
  if (tid == 0) pb = 0;
  __syncthreads();
  int b = 0;
  double s = 0.0;
  unsigned long long h = 1469598103934665603ull;
  for (int j = tid; j < N; j += 256) {
    const float v = row[j];
    if (!(v >= 0.0f) || !isfinite(v)) b |= 1;
    s += (double)v;
    const uint32_t u = __float_as_uint(v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      h ^= (u >> (8 * k)) & 0xffu;
      h *= 1099511628211ull;
    }
  }
  if (tid == 0 && row[i] != 0.0f) b |= 2;
  if (b) atomicOr(&pb, b);
  ps[tid] = s;
  ph[tid] = h;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    unsigned long long g = 1469598103934665603ull;
    for (int k = 0; k < 256; ++k) {
      t += ps[k];
      for (int q = 0; q < 8; ++q) {
        g ^= (ph[k] >> (8 * q)) & 0xffull;
        g *= 1099511628211ull;
      }
    }
    bad[i] = pb;
    sums[i] = t;
    hashes[i] = g;
  }
}

// The BF16 prior format: every entry rounded to the nearest bfloat16 (ties to even), in place.
__global__ void prior_bf16_kernel(float* __restrict__ Pi, long long n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) Pi[e] = __bfloat162float(__float2bfloat16_rn(Pi[e]));
}

// Doubled rows for the propagation kernel: out[l][q] holds bits [32q, 32q+32) of the cyclic string
// b -> h[l][b mod N] for b < 2N (zero beyond), so every rotated slice is one contiguous run.
__global__ void double_rows_kernel(const uint32_t* __restrict__ bits, int rw, int N, int L, uint32_t* __restrict__ out,
                                   int rw2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)L * rw2) return;
  const int l = (int)(i / rw2), q = (int)(i % rw2);
  const uint32_t* row = bits + (size_t)l * rw;
  const long long p0 = 32ll * q;
  uint32_t v = 0;
  if (p0 < 2ll * N) {
    const int g = (int)(p0 < N ? p0 : p0 - N);
    v = N >= 32 ? cyclic32(row, N, g) : cyclic32_slow(row, N, g);
    const long long rem = 2ll * N - p0;
    if (rem < 32) v &= (1u << rem) - 1u;
  }
  out[i] = v;
}


// Pack uint8 [L][N] 0/1 haplotypes into variant-major rows of 32 haplotypes per word, haplotype i
// in bit i%32 of word i/32 (Sec. 4.1.1).  One warp per output word: a coalesced 32-byte read and a
// ballot.  Padding words must be zeroed beforehand.
__global__ void pack_kernel(const uint8_t* __restrict__ h, int N, int L, int row_words, uint32_t* __restrict__ out) {
  const int nw = (N + 31) / 32;
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (long long)nw * L) return;
  const int l = (int)(wid / nw), w = (int)(wid % nw);
  const int i = 32 * w + lane;
  const bool bit = i < N && h[(size_t)l * N + i] != 0;
  const uint32_t word = __ballot_sync(0xffffffffu, bit);
  if (lane == 0) out[(size_t)l * row_words + w] = word;
}

// Eq. postprob from a forward table (alpha) and a backward table (beta) at the same locus, one
// CTA per target row: p_j = alpha_j beta_j / sum_k alpha_k beta_k (eps for all j if the sum is 0),
// p_ii = 0.  mode 0 writes p; mode 1 writes -log(max(p, eps))/2 (the half distance of Eq. distmat).
__global__ void posterior_kernel(const float* __restrict__ alpha, const float* __restrict__ beta, int N, int t0,
                                 int mode, float* __restrict__ out) {
  constexpr float eps = 2.220446049250313e-16f;
  const int r = blockIdx.x, i = t0 + r;
  const float* a = alpha + (size_t)r * N;
  const float* b = beta + (size_t)r * N;
  float s = 0.0f;
  for (int j = threadIdx.x; j < N; j += blockDim.x)
    if (j != i) s += a[j] * (b[j] * kProdScale);
  __shared__ float red[32];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const float Z = red[0];
  const float invZ = Z > 0.0f ? 1.0f / Z : 0.0f;
  float* o = out + (size_t)r * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    float p = j == i ? 0.0f : (Z > 0.0f ? a[j] * (b[j] * kProdScale) * invZ : eps);
    if (mode == 1) p = j == i ? 0.0f : -0.5f * logf(fmaxf(p, eps));
    o[j] = p;
  }
}

// Decode loci of the D slots of a fused pipeline (at most kMaxStore), passed by value.
struct DecodeLoci {
  int l[kMaxStore];
};

// Normalise the products that the backward pass left at D decode loci ([D][N][N], row i = recipient
// i) into half distances -log(max(p, eps))/2 with p of Eq. postprob, in place.  A product is
// alpha^l t^l (times a power of two), t = theta beta the backward tile after its update at l, so
// each entry is first divided by its emission theta^l_ij (1 - mu where donor j carries the target's
// allele at l, mu elsewhere, read from the packed row; a zero theta means alpha = 0 too, and the
// entry is 0).  A zero normaliser gives p = eps for every donor (Sec. 2.2).  Grid (N, D), one CTA
// per row.
__global__ void decode_kernel(float* __restrict__ prod, int N, const uint32_t* __restrict__ bits, int row_words,
                              const float* __restrict__ thm, const float* __restrict__ thx, const DecodeLoci dl) {
  constexpr float eps = 2.220446049250313e-16f;
  const int r = blockIdx.x;
  const int l = dl.l[blockIdx.y];
  const uint32_t* row = bits + (size_t)l * row_words;
  const uint32_t ai = (row[r >> 5] >> (r & 31)) & 1u;
  const float tm = thm[l], tx = thx[l];
  const float im = tm > 0.0f ? 1.0f / tm : 0.0f, ix = tx > 0.0f ? 1.0f / tx : 0.0f;
  float* a = prod + ((size_t)blockIdx.y * N + r) * N;
  auto q = [&](int j) { return a[j] * ((((row[j >> 5] >> (j & 31)) & 1u) == ai) ? im : ix); };
  float s = 0.0f;
  for (int j = threadIdx.x; j < N; j += blockDim.x)
    if (j != r) s += q(j);
  __shared__ float red[32];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const float Z = red[0];
  const float invZ = Z > 0.0f ? 1.0f / Z : 0.0f;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const float p = Z > 0.0f ? q(j) * invZ : eps;
    a[j] = j == r ? 0.0f : -0.5f * logf(fmaxf(p, eps));
  }
}

// In-place symmetrisation of D stacked N x N matrices of half distances h: d = h + h^T with a zero
// diagonal (Eq. distmat).  Block (bx, by) with bx <= by owns the tile pair (bx, by)/(by, bx): it
// reads both 32x32 tiles into shared memory before writing either, so no element is read after
// another block wrote it.  Reads and writes are 128-byte rows.
__global__ void symmetrize_kernel(float* __restrict__ d, int N) {
  const int bx = blockIdx.x, by = blockIdx.y;
  if (bx > by) return;
  float* m = d + (size_t)blockIdx.z * N * N;
  __shared__ float A[32][33], B[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int ra = bx * 32 + k, ca = by * 32 + tx;  // tile (bx, by)
    const int rb = by * 32 + k, cb = bx * 32 + tx;  // tile (by, bx)
    A[k][tx] = (ra < N && ca < N) ? m[(size_t)ra * N + ca] : 0.0f;
    B[k][tx] = (rb < N && cb < N) ? m[(size_t)rb * N + cb] : 0.0f;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int ra = bx * 32 + k, ca = by * 32 + tx;
    if (ra < N && ca < N) m[(size_t)ra * N + ca] = ra == ca ? 0.0f : A[k][tx] + B[tx][k];
    if (bx != by) {
      const int rb = by * 32 + k, cb = bx * 32 + tx;
      if (rb < N && cb < N) m[(size_t)rb * N + cb] = B[k][tx] + A[tx][k];
    }
  }
}

// Binary16 checkpoint of one forward state row per block: scale = max_j alpha_j (NaN when the row
// holds a non-finite value), q_j = alpha_j / scale rounded to nearest binary16 (0 for a zero row).
__global__ void ckpt_encode_f16_kernel(const float* __restrict__ alpha, int N, __half* __restrict__ q,
                                       float* __restrict__ scale) {
  __shared__ float wmax[32];
  __shared__ int wbad[32];
  const size_t row = blockIdx.x;
  const float* x = alpha + row * (size_t)N;
  float m = 0.0f;
  int bad = 0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const float v = x[j];
    if (!(v <= 3.40282347e+38f)) bad = 1;
    m = fmaxf(m, v);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    bad |= __shfl_xor_sync(0xffffffffu, bad, off);
  }
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    wmax[warp] = m;
    wbad[warp] = bad;
  }
  __syncthreads();
  m = 0.0f;
  bad = 0;
  for (int w = 0; w < nw; ++w) {
    m = fmaxf(m, wmax[w]);
    bad |= wbad[w];
  }
  const float sc = bad ? __int_as_float(0x7fc00000) : m;
  if (threadIdx.x == 0) scale[row] = sc;
  __half* qr = q + row * (size_t)N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) qr[j] = __float2half_rn(sc > 0.0f ? x[j] / sc : 0.0f);
}

// Inverse of ckpt_encode_f16_kernel: alpha_j = q_j * scale, one row per block.
__global__ void ckpt_decode_f16_kernel(const __half* __restrict__ q, const float* __restrict__ scale, int N,
                                       float* __restrict__ alpha) {
  const size_t row = blockIdx.x;
  const float sc = scale[row];
  const __half* qr = q + row * (size_t)N;
  float* x = alpha + row * (size_t)N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) x[j] = __half2float(qr[j]) * sc;
}

// Adjoint: per (group g, target t) the posterior expectation of a statistic at the group's end
// locus, sum_j w_j beta_j / sum_j alpha_j beta_j, from the stored alpha, w and beta rows.  FP32
// products, FP64 sums.  grid (T, G), 256 threads.
__global__ void grad_dot_kernel(const float* __restrict__ A, const float* __restrict__ Wst, const float* __restrict__ B,
                                int N, int T, double* __restrict__ out) {
  __shared__ double sa[256], sw[256];
  const size_t row = (size_t)blockIdx.y * T + blockIdx.x;
  const float* a = A + row * N;
  const float* w = Wst + row * N;
  const float* b = B + row * N;
  double da = 0.0, dw = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const float bj = b[j];
    da += (double)(a[j] * bj);
    dw += (double)(w[j] * bj);
  }
  sa[threadIdx.x] = da;
  sw[threadIdx.x] = dw;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      sa[threadIdx.x] += sa[threadIdx.x + h];
      sw[threadIdx.x] += sw[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[row] = sw[0] / sa[0];
}

// Fixed-order FP64 sums of `rows` vectors of length n (one block of 256 threads per row).
__global__ void sum_rows_kernel(const double* __restrict__ v, int n, double* __restrict__ out) {
  __shared__ double s[256];
  const double* r = v + (size_t)blockIdx.x * n;
  double acc = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) acc += r[j];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

}  // namespace lsk
