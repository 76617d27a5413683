// ls_mlp_tc.cuh -- the proposal network's scorer on the fifth-generation tensor cores (tcgen05).
//
// scores[r] = w3 . relu(W2^T relu(W1^T x_r + b1) + b2) + b3 for n rows of BF16 features, in tiles
// of 128 rows, 256 threads.  Layer 1 (7 inputs -> 256) runs on the FP32 pipe, two threads per row
// (128 hidden units each), and writes the BF16-rounded hidden row into shared memory; layer 2
// (256 x 256) is one 128 x 256 x 256 product on the tensor cores: sixteen tcgen05.mma (M = 128,
// N = 256, K = 16, BF16 inputs, FP32 accumulation) issued by one thread, the accumulator in tensor
// memory (256 columns x 128 lanes); layer 3 reads the accumulator back with tcgen05.ld (warp w its
// 32 lanes 32 (w % 4).. = rows and the columns of half w / 4), takes bias, ReLU and the dot product
// with w3 in FP32, and adds the two halves' partial sums through shared memory.
//
// Operand layout (shared memory, K-major, 128-byte swizzle): a matrix of R rows x 256 BF16 columns
// is four 64-column atoms of R rows x 128 bytes, row r of an atom at byte 128 r, its 16-byte chunk c
// stored at chunk c ^ (r % 8).  The atoms start on 1024-byte boundaries, so the hardware's swizzle
// (address bits 4-6 XOR bits 7-9) matches.  The k-th slice of 16 columns is the atom k / 4 shifted
// by 32 (k % 4) bytes; consecutive 8-row groups are 1024 bytes apart (the stride field).
//
// The network's parameters are staged once per CTA (persistent CTAs, one per SM).  Every wait has a
// time limit; on a timeout the CTA records it in *err, stops and frees its tensor memory.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace lsk {

constexpr int kTcThreads = 256;
constexpr int kTcRows = 128;                       // rows per tile (M)
constexpr int kTcCols = 256;                       // hidden units (N = K of layer 2)
constexpr int kTcB = 0;                            // W2^T as the B operand: 4 atoms x 256 rows x 128 B
constexpr int kTcA = kTcB + 4 * kTcCols * 128;     // hidden tile as the A operand: 4 atoms x 128 rows x 128 B
constexpr int kTcW1 = kTcA + 4 * kTcRows * 128;    // W1 as FP32 [8][256]
constexpr int kTcBias = kTcW1 + 8 * kTcCols * 4;   // b1, b2, w3 as FP32 [3][256]
constexpr int kTcPart = kTcBias + 3 * kTcCols * 4;  // partial scores of the second column half [128]
constexpr int kTcBar = kTcPart + kTcRows * 4;       // mbarrier (8 B), tensor-memory address (4 B)
constexpr int kTcBytes = kTcBar + 16;
constexpr int kTcSmem = kTcBytes + 1024;           // + alignment of the base to 1024 bytes

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t tc_pack_bf16(float lo, float hi) {  // round to nearest even
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading-dimension offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride-dimension offset
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // swizzle: 128 bytes
  return d;
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, N = 256, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcCols >> 3) << 17) |
                              ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ bool tc_mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t tc_now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// 32 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// byte offset of element (row, col) of a K-major, 128-byte-swizzled operand with R rows
__device__ __forceinline__ uint32_t tc_off(int R, int row, int col) {
  const int atom = col >> 6, chunk = (col >> 3) & 7;
  return (uint32_t)(atom * R * 128 + row * 128 + ((chunk ^ (row & 7)) << 4) + ((col & 7) << 1));
}

struct MlpTcDev {
  const __nv_bfloat16* w1t;  // [256][16]  w1t[n][k] = W1[k][n]
  const float* b1;           // [256]
  const __nv_bfloat16* w2t;  // [256][256] w2t[n][k] = W2[k][n]
  const float* b2;           // [256]
  const float* w3;           // [256]
  float b3;
  int* err;                  // set to 1 when a wait ran out of time
};

__global__ void __launch_bounds__(kTcThreads, 1) mlp_score_tc_kernel(MlpTcDev m, const __nv_bfloat16* __restrict__ X,
                                                                     long long n, float* __restrict__ scores) {
  extern __shared__ unsigned char tc_raw[];
  const uint32_t raw = tc_smem_u32(tc_raw);
  unsigned char* sm = tc_raw + (((raw + 1023u) & ~1023u) - raw);  // 1024-byte aligned base
  const uint32_t base = tc_smem_u32(sm);
  float* W1f = reinterpret_cast<float*>(sm + kTcW1);    // [8][256]
  float* bias = reinterpret_cast<float*>(sm + kTcBias);  // b1 [256], b2 [256], w3 [256]
  const uint32_t bar = base + kTcBar;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kTcBar + 8);
  const int tid = threadIdx.x, warp = tid >> 5;

  // stage W2^T in the swizzled layout (16-byte chunks), W1, biases
  for (int e = tid; e < kTcCols * kTcCols / 8; e += kTcThreads) {
    const int row = e >> 5, c8 = (e & 31) << 3;  // row n of W2^T, first of 8 columns k
    const uint4 v = *reinterpret_cast<const uint4*>(m.w2t + (size_t)row * kTcCols + c8);
    *reinterpret_cast<uint4*>(sm + kTcB + tc_off(kTcCols, row, c8)) = v;
  }
  for (int e = tid; e < 8 * kTcCols; e += kTcThreads) {
    const int k = e >> 8, u = e & 255;
    W1f[e] = k < 7 ? __bfloat162float(m.w1t[u * 16 + k]) : 0.0f;
  }
  for (int e = tid; e < kTcCols; e += kTcThreads) {
    bias[e] = m.b1[e];
    bias[kTcCols + e] = m.b2[e];
    bias[2 * kTcCols + e] = m.w3[e];
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // 256 columns of tensor memory for the 128 x 256 FP32 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(tslot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // staged W2 -> tensor-core reads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  const long long ntile = (n + kTcRows - 1) / kTcRows;
  uint32_t phase = 0;
  float* part = reinterpret_cast<float*>(sm + kTcPart);
  const int row = tid & (kTcRows - 1), half = tid >> 7;  // layer 1: row and half of the hidden units
  for (long long t = blockIdx.x; t < ntile; t += gridDim.x) {
    const long long r = t * kTcRows + row;
    // layer 1 on the FP32 pipe; the hidden row rounded to BF16 into the A operand
    float x[7];
    {
      const __nv_bfloat16* xr = X + (size_t)(r < n ? r : 0) * 16;
#pragma unroll
      for (int k = 0; k < 7; ++k) x[k] = r < n ? __bfloat162float(xr[k]) : 0.0f;
    }
#pragma unroll 2
    for (int c8 = 128 * half; c8 < 128 * half + 128; c8 += 8) {
      float h[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) h[u] = bias[c8 + u];
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const float4 w0 = *reinterpret_cast<const float4*>(W1f + k * kTcCols + c8);
        const float4 w1 = *reinterpret_cast<const float4*>(W1f + k * kTcCols + c8 + 4);
        h[0] = fmaf(x[k], w0.x, h[0]);
        h[1] = fmaf(x[k], w0.y, h[1]);
        h[2] = fmaf(x[k], w0.z, h[2]);
        h[3] = fmaf(x[k], w0.w, h[3]);
        h[4] = fmaf(x[k], w1.x, h[4]);
        h[5] = fmaf(x[k], w1.y, h[5]);
        h[6] = fmaf(x[k], w1.z, h[6]);
        h[7] = fmaf(x[k], w1.w, h[7]);
      }
      uint4 pk;
      pk.x = tc_pack_bf16(fmaxf(h[0], 0.f), fmaxf(h[1], 0.f));
      pk.y = tc_pack_bf16(fmaxf(h[2], 0.f), fmaxf(h[3], 0.f));
      pk.z = tc_pack_bf16(fmaxf(h[4], 0.f), fmaxf(h[5], 0.f));
      pk.w = tc_pack_bf16(fmaxf(h[6], 0.f), fmaxf(h[7], 0.f));
      *reinterpret_cast<uint4*>(sm + kTcA + tc_off(kTcRows, row, c8)) = pk;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // hidden tile -> tensor-core reads
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
#pragma unroll
      for (int k = 0; k < kTcCols / 16; ++k) {
        const uint32_t koff = (uint32_t)((k & 3) * 32);  // 16 columns = 32 bytes within the atom
        tc_mma(tmem, tc_desc(base + kTcA + (k >> 2) * kTcRows * 128 + koff),
               tc_desc(base + kTcB + (k >> 2) * kTcCols * 128 + koff), k > 0 ? 1u : 0u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
    }
    // wait for the products (at most ~2 s), the same decision in every thread
    bool ok = tc_mbar_test(bar, phase);
    if (!ok) {
      const uint64_t t0 = tc_now_ns();
      while (!(ok = tc_mbar_test(bar, phase)) && tc_now_ns() - t0 < 2000000000ull) __nanosleep(32);
    }
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(m.err, 1);
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // layer 3: bias, ReLU and the dot product with w3 over this thread's row and column half of
    // the accumulator; the second half's partial sums meet the first's in shared memory
    const int erow = 32 * (warp & 3) + (tid & 31), ecol = 128 * (warp >> 2);
    float s = 0.0f;
#pragma unroll 1
    for (int c0 = ecol; c0 < ecol + 128; c0 += 32) {
      float v[32];
      tc_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int k = 0; k < 32; ++k) s = fmaf(fmaxf(v[k] + bias[kTcCols + c0 + k], 0.0f), bias[2 * kTcCols + c0 + k], s);
    }
    if (warp >= 4) part[erow] = s;
    __syncthreads();
    const long long er = t * kTcRows + erow;
    if (warp < 4 && er < n) scores[er] = (s + part[erow]) + m.b3;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // the accumulator and the hidden tile are rewritten by the next tile
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

}  // namespace lsk
