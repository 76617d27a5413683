// ls_mlp_tc.cuh -- the proposal network's scorer on the fifth-generation tensor cores (tcgen05).
//
// scores[r] = w3 . relu(W2^T relu(W1^T x_r + b1) + b2) + b3 for n rows of BF16 features, in tiles
// of 128 rows, one persistent CTA of 256 threads per SM.  Both products run on the tensor cores,
// issued by one thread, FP32 accumulators in tensor memory:
//   layer 1: one tcgen05.mma (M = 128, N = 256, K = 16: the 7 features zero-padded) of the feature
//            tile by W1;
//   layer 2: sixteen tcgen05.mma (M = 128, N = 256, K = 16 each) of the BF16 hidden tile by W2.
// The CUDA cores only move data between them: epilogue 1 reads the layer-1 accumulator back with
// tcgen05.ld, adds b1, applies ReLU while rounding to BF16 (one cvt.rn.relu.bf16x2 per pair) and
// writes the hidden tile into shared memory; epilogue 2 reads the layer-2 accumulator, adds b2,
// applies ReLU and takes the dot product with w3 in FP32 (warp w: TMEM lanes 32 (w % 4).. = rows,
// columns of half w / 4; the halves meet through shared memory).
//
// Pipeline: two 256-column accumulators in tensor memory (512 columns).  Tile t uses buffer t % 2
// for both of its layers; while the tensor cores run tile t's layer 2, the CUDA cores drain tile
// t-1's layer-2 accumulator from the other buffer, and tile t+1's layer 1 goes into that buffer as
// soon as it has been read.
//
// Operand layouts (shared memory, K-major).  W2^T and the hidden tile: 128-byte swizzle, a matrix of
// R rows x 256 BF16 columns is four 64-column atoms of R rows x 128 bytes, row r of an atom at byte
// 128 r, its 16-byte chunk c stored at chunk c ^ (r % 8), atoms on 1024-byte boundaries (the
// hardware's swizzle XORs address bits 4-6 with bits 7-9); the k-th 16-column slice is atom k / 4
// shifted by 32 (k % 4) bytes, 8-row groups 1024 bytes apart.  W1^T and the feature tile (16
// columns): no swizzle, 8-row x 16-byte core matrices, the two along K 128 bytes apart and
// consecutive 8-row groups 256 bytes apart.
//
// The network's parameters are staged once per CTA.  Every wait has a time limit; on a timeout the
// CTA records it in *err, stops and frees its tensor memory.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace lsk {

constexpr int kTcThreads = 256;
constexpr int kTcRows = 128;                       // rows per tile (M)
constexpr int kTcCols = 256;                       // hidden units (N of both layers, K of layer 2)
constexpr int kTcB = 0;                            // W2^T as the B operand: 4 atoms x 256 rows x 128 B
constexpr int kTcA = kTcB + 4 * kTcCols * 128;     // hidden tile as the A operand: 4 atoms x 128 rows x 128 B
constexpr int kTcW1 = kTcA + 4 * kTcRows * 128;    // W1^T as the B operand of layer 1: 256 rows x 32 B
constexpr int kTcX = kTcW1 + kTcCols * 32;         // feature tile as the A operand of layer 1: 128 rows x 32 B
constexpr int kTcBias = kTcX + kTcRows * 32;       // b1, b2, w3 as FP32 [3][256]
constexpr int kTcPart = kTcBias + 3 * kTcCols * 4;  // partial scores of the second column half [128]
constexpr int kTcBar = kTcPart + kTcRows * 4;       // two mbarriers (16 B), tensor-memory address (4 B)
constexpr int kTcBytes = kTcBar + 32;
constexpr int kTcSmem = kTcBytes + 1024;           // + alignment of the base to 1024 bytes
constexpr int kTcTmemCols = 2 * kTcCols;           // two accumulators

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

// shared-memory matrix descriptor: K-major, no swizzle, 8-row x 16-byte core matrices, the next
// core matrix along K 128 bytes on, the next 8-row group 256 bytes on (a 16-column operand)
__device__ __forceinline__ uint64_t tc_desc_k16(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)(128 >> 4) << 16;           // leading-dimension (K) offset
  d |= (uint64_t)(256 >> 4) << 32;           // stride-dimension (M/N) offset
  d |= (uint64_t)1 << 46;                    // descriptor version; swizzle field 0: none
  return d;
}
// byte offset of the 16-byte chunk c (columns 8c..8c+7) of row r in that layout
__device__ __forceinline__ uint32_t tc_off_k16(int r, int c) {
  return (uint32_t)((r >> 3) * 256 + c * 128 + (r & 7) * 16);
}

// (relu(lo), relu(hi)) rounded to BF16, lo in the low half
__device__ __forceinline__ uint32_t tc_relu_bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
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

// 32 consecutive accumulator columns of this thread's lane (the wait carries the registers, so
// nothing reads them before the load has landed)
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
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
                 "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                 "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
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

// wait for phase `parity` of an mbarrier for at most ~2 s; the same answer in every thread
__device__ __forceinline__ bool tc_wait_all(uint32_t bar, uint32_t parity) {
  bool ok = tc_mbar_test(bar, parity);
  if (!ok) {
    const uint64_t t0 = tc_now_ns();
    while (!(ok = tc_mbar_test(bar, parity)) && tc_now_ns() - t0 < 2000000000ull) __nanosleep(32);
  }
  return !__syncthreads_or(!ok);
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// every thread's tensor-memory accesses and shared-memory writes before this point are ordered before
// the tensor-core operations the issuing thread starts after it
__device__ __forceinline__ void tc_sync_for_mma() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__global__ void __launch_bounds__(kTcThreads, 1) mlp_score_tc_kernel(MlpTcDev m, const __nv_bfloat16* __restrict__ X,
                                                                     long long n, float* __restrict__ scores) {
  extern __shared__ unsigned char tc_raw[];
  const uint32_t raw = tc_smem_u32(tc_raw);
  unsigned char* sm = tc_raw + (((raw + 1023u) & ~1023u) - raw);  // 1024-byte aligned base
  const uint32_t base = tc_smem_u32(sm);
  const float* b1s = reinterpret_cast<const float*>(sm + kTcBias);
  const float* b2s = b1s + kTcCols;
  const float* w3s = b2s + kTcCols;
  float* part = reinterpret_cast<float*>(sm + kTcPart);
  const uint32_t bar1 = base + kTcBar, bar2 = base + kTcBar + 8;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kTcBar + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // stage W2^T (swizzled), W1^T (16 columns, no swizzle) and the FP32 vectors
  for (int e = tid; e < kTcCols * kTcCols / 8; e += kTcThreads) {
    const int row = e >> 5, c8 = (e & 31) << 3;  // row n of W2^T, first of 8 columns k
    const uint4 v = *reinterpret_cast<const uint4*>(m.w2t + (size_t)row * kTcCols + c8);
    *reinterpret_cast<uint4*>(sm + kTcB + tc_off(kTcCols, row, c8)) = v;
  }
  for (int e = tid; e < kTcCols * 2; e += kTcThreads) {
    const int row = e >> 1, c = e & 1;
    *reinterpret_cast<uint4*>(sm + kTcW1 + tc_off_k16(row, c)) = *reinterpret_cast<const uint4*>(m.w1t + row * 16 + 8 * c);
  }
  for (int e = tid; e < kTcCols; e += kTcThreads) {
    float* bias = reinterpret_cast<float*>(sm + kTcBias);
    bias[e] = m.b1[e];
    bias[kTcCols + e] = m.b2[e];
    bias[2 * kTcCols + e] = m.w3[e];
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar2) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // two 256-column accumulators (128 lanes x FP32)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(tslot)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }

  // the feature tile of tile t: thread -> (row, 16-byte half of the row); rows beyond n read as
  // zero.  fetch_x loads this thread's part into registers, store_x puts it into the A operand.
  auto fetch_x = [&](long long t) -> uint4 {
    const long long r = t * kTcRows + (tid >> 1);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (r < n) v = *reinterpret_cast<const uint4*>(X + (size_t)r * 16 + 8 * (tid & 1));
    return v;
  };
  auto store_x = [&](uint4 v) { *reinterpret_cast<uint4*>(sm + kTcX + tc_off_k16(tid >> 1, tid & 1)) = v; };
  // tensor-core issue (one thread): layer 1 of a tile into accumulator `buf`, layer 2 likewise
  auto mma1 = [&](uint32_t d) { tc_mma(d, tc_desc_k16(base + kTcX), tc_desc_k16(base + kTcW1), 0u); };
  auto mma2 = [&](uint32_t d) {
#pragma unroll
    for (int k = 0; k < kTcCols / 16; ++k) {
      const uint32_t koff = (uint32_t)((k & 3) * 32);  // 16 columns = 32 bytes within the atom
      tc_mma(d, tc_desc(base + kTcA + (k >> 2) * kTcRows * 128 + koff), tc_desc(base + kTcB + (k >> 2) * kTcCols * 128 + koff),
             k > 0 ? 1u : 0u);
    }
  };
  // this thread's accumulator lane (= row of the tile) and column half
  const int erow = 32 * (warp & 3) + lane, ecol = 128 * (warp >> 2);
  const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
  // epilogue 1: b1, ReLU, BF16 into the hidden tile (the A operand of layer 2)
  auto epi1 = [&](uint32_t d) {
#pragma unroll 1
    for (int c0 = ecol; c0 < ecol + 128; c0 += 32) {
      float v[32];
      tc_ld32(d + lane_off + (uint32_t)c0, v);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 ba = *reinterpret_cast<const float4*>(b1s + c0 + 8 * q);
        const float4 bb = *reinterpret_cast<const float4*>(b1s + c0 + 8 * q + 4);
        uint4 pk;
        pk.x = tc_relu_bf16x2(v[8 * q + 0] + ba.x, v[8 * q + 1] + ba.y);
        pk.y = tc_relu_bf16x2(v[8 * q + 2] + ba.z, v[8 * q + 3] + ba.w);
        pk.z = tc_relu_bf16x2(v[8 * q + 4] + bb.x, v[8 * q + 5] + bb.y);
        pk.w = tc_relu_bf16x2(v[8 * q + 6] + bb.z, v[8 * q + 7] + bb.w);
        *reinterpret_cast<uint4*>(sm + kTcA + tc_off(kTcRows, erow, c0 + 8 * q)) = pk;
      }
    }
  };
  // epilogue 2: b2, ReLU and the dot product with w3; the column halves meet in shared memory
  auto epi2 = [&](uint32_t d, long long t) {
    float2 acc[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll 1
    for (int c0 = ecol; c0 < ecol + 128; c0 += 32) {
      float v[32];
      tc_ld32(d + lane_off + (uint32_t)c0, v);
#pragma unroll
      for (int k = 0; k < 32; k += 4) {
        const float4 bv = *reinterpret_cast<const float4*>(b2s + c0 + k);
        const float4 wv = *reinterpret_cast<const float4*>(w3s + c0 + k);
        const float2 h01 = __fadd2_rn(make_float2(v[k], v[k + 1]), make_float2(bv.x, bv.y));
        const float2 h23 = __fadd2_rn(make_float2(v[k + 2], v[k + 3]), make_float2(bv.z, bv.w));
        acc[(k >> 2) & 1] = __ffma2_rn(make_float2(fmaxf(h01.x, 0.f), fmaxf(h01.y, 0.f)), make_float2(wv.x, wv.y),
                                       acc[(k >> 2) & 1]);
        acc[2 + ((k >> 2) & 1)] = __ffma2_rn(make_float2(fmaxf(h23.x, 0.f), fmaxf(h23.y, 0.f)),
                                             make_float2(wv.z, wv.w), acc[2 + ((k >> 2) & 1)]);
      }
    }
    const float s = ((acc[0].x + acc[0].y) + (acc[1].x + acc[1].y)) + ((acc[2].x + acc[2].y) + (acc[3].x + acc[3].y));
    if (warp >= 4) part[erow] = s;
    __syncthreads();
    const long long er = t * kTcRows + erow;
    if (warp < 4 && er < n) scores[er] = (s + part[erow]) + m.b3;
  };

  const long long ntile = (n + kTcRows - 1) / kTcRows;
  const long long G = gridDim.x;
  long long t = blockIdx.x;
  store_x(fetch_x(t));
  tc_sync_for_mma();  // also publishes the staged weights, the barriers and the tensor-memory address
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    mma1(tmem);
    tc_commit(bar1);
  }
  uint32_t ph1 = 0;
  int i = 0;
  bool ok = true;
  for (; t < ntile; t += G, ++i) {
    const uint32_t d = tmem + (uint32_t)((i & 1) * kTcCols), d_prev = tmem + (uint32_t)(((i + 1) & 1) * kTcCols);
    // the next tile's features are requested now and land while this tile's epilogue runs
    const uint4 xn = t + G < ntile ? fetch_x(t + G) : make_uint4(0u, 0u, 0u, 0u);
    // tile t's layer 1 is done, and with it (same issuing thread, in order) tile t - G's layer 2
    if (!(ok = tc_wait_all(bar1, ph1))) break;
    ph1 ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    epi1(d);
    if (t + G < ntile) store_x(xn);  // layer 1 of tile t has read the feature tile
    tc_sync_for_mma();
    if (tid == 0) mma2(d);
    if (i > 0) epi2(d_prev, t - G);  // overlaps tile t's layer 2
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // d_prev has been read: it takes the next tile's layer 1
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0 && t + G < ntile) {
      mma1(d_prev);
      tc_commit(bar1);
    }
  }
  if (ok && i > 0) {  // layer 2 of this CTA's last tile
    if (tid == 0) tc_commit(bar2);
    if ((ok = tc_wait_all(bar2, 0u))) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      epi2(tmem + (uint32_t)(((i - 1) & 1) * kTcCols), t - G);
    }
  }
  if (!ok && tid == 0) atomicExch(m.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
}

}  // namespace lsk
