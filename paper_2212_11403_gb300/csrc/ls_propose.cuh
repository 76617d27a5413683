// ls_propose.cuh -- donor proposal for the sparse recursions: window match-count features, a
// first-stage pre-filter and top-K (the MLP scorer on the tensor cores is in ls_mlp_tc.cuh).
//
// Windows hold 256 consecutive loci.  For haplotypes i, j and window w the feature is the match
// count m_ij^w = n_w - popcount(h_i^w XOR h_j^w) (n_w = loci in the window).  Stage 1 keeps, for
// target i and window w, the C donors with the smallest mismatch sum over windows w-1..w+1 (ties
// to the lower donor id, never i itself).  Stage 2 scores each candidate with the MLP on the
// match fractions m^{w+d}/n_{w+d}, d = -3..3 (windows clamped to the range), and keeps the K best
// (ties to the lower id).  Sets are written in ascending donor order.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace lsk {

constexpr int kPropWS = 256;       // loci per window
constexpr int kFeat = 16;          // feature slots per candidate (7 used, zero padded to one MMA k-step)
constexpr int kFeatUsed = 7;
constexpr int kHidden = 256;

// Haplotype-major window bits: hw[(w*N + i)*8 + k] bit b = allele of haplotype i at locus
// w*256 + 32k + b (0 beyond L).  grid (ceil(N/32), 8, Wn), one warp: a 32 x 32 bit transpose by
// ballots.
__global__ void hapmajor_kernel(const uint32_t* __restrict__ bits, int row_words, int N, int L,
                                uint32_t* __restrict__ hw) {
  const int g = blockIdx.x, k = blockIdx.y, w = blockIdx.z, lane = threadIdx.x;
  const int l = w * kPropWS + 32 * k + lane;
  const uint32_t word = l < L ? bits[(size_t)l * row_words + g] : 0u;
  uint32_t mine = 0u;
#pragma unroll
  for (int h = 0; h < 32; ++h) {
    const uint32_t b = __ballot_sync(0xffffffffu, (word >> h) & 1u);
    if (lane == h) mine = b;
  }
  const int i = 32 * g + lane;
  if (i < N) hw[((size_t)w * N + i) * 8 + k] = mine;
}

// Mismatch counts of one window, min(popcount, 255) as bytes: M[i*Np + j].  64 x 64 pairs per
// block of 256 threads; thread t handles row t/4 and 16 consecutive columns (one 16-byte store).
__global__ void mismatch_kernel(const uint32_t* __restrict__ hw, int N, int Np, uint8_t* __restrict__ M) {
  __shared__ uint32_t A[64][9], B[64][9];
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  for (int e = threadIdx.x; e < 64 * 8; e += 256) {
    const int r = e >> 3, k = e & 7;
    A[r][k] = i0 + r < N ? hw[(size_t)(i0 + r) * 8 + k] : 0u;
    B[r][k] = j0 + r < N ? hw[(size_t)(j0 + r) * 8 + k] : 0u;
  }
  __syncthreads();
  const int r = threadIdx.x >> 2, c0 = (threadIdx.x & 3) * 16;
  uint32_t a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = A[r][k];
  uint32_t packed[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    int m = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) m += __popc(a[k] ^ B[c0 + c][k]);
    packed[c >> 2] |= (uint32_t)min(m, 255) << (8 * (c & 3));
  }
  if (i0 + r < N && j0 + c0 < Np)
    *reinterpret_cast<uint4*>(M + (size_t)(i0 + r) * Np + j0 + c0) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
}

// Stage 1 for one window, one block (256 threads) per target i: the C donors with the smallest
// mismatch sum over the available windows among w-1..w+1 (score <= 765), ties to the lower id,
// written in ascending id order together with their features (match fractions of windows
// w-3..w+3, clamped).  Ms[d] = count matrix of window w+d-3 (clamped), nv[d] its locus count.
struct Stage1Args {
  const uint8_t* Ms[7];
  float inv_nv[7];
  int use[3];  // whether windows w-1, w, w+1 exist
};

__global__ void __launch_bounds__(256) stage1_kernel(Stage1Args a, int N, int Np, int C, int32_t* __restrict__ cand,
                                                     __nv_bfloat16* __restrict__ feat, float* __restrict__ feat32) {
  constexpr int NB = 768, NT = 256, V = 16;  // score bins, threads, donors per thread per pass step
  __shared__ int hist[8][NB];                // one histogram per warp (fewer colliding atomics)
  __shared__ int scan_s[8];
  __shared__ int thr_s, need_eq_s;
  const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the three windows' rows of target i (16-byte aligned: Np is a multiple of 64)
  const uint8_t* r0 = a.use[0] ? a.Ms[2] + (size_t)i * Np : nullptr;
  const uint8_t* r1 = a.use[1] ? a.Ms[3] + (size_t)i * Np : nullptr;
  const uint8_t* r2 = a.use[2] ? a.Ms[4] + (size_t)i * Np : nullptr;
  auto load16 = [](const uint8_t* r, int j0) -> uint4 {
    return r ? *reinterpret_cast<const uint4*>(r + j0) : make_uint4(0u, 0u, 0u, 0u);
  };
  auto byte_of = [](const uint4& v, int k) -> int {
    const uint32_t w = k < 4 ? v.x : (k < 8 ? v.y : (k < 12 ? v.z : v.w));
    return (int)((w >> (8 * (k & 3))) & 255u);
  };
  // exclusive prefix of v over the block (thread order) and the block total; two barriers
  auto block_scan = [&](int v, int& total) -> int {
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) scan_s[warp] = x;
    __syncthreads();
    int wpre = 0, tot = 0;
#pragma unroll
    for (int w2 = 0; w2 < 8; ++w2) {
      const int s = scan_s[w2];
      wpre += w2 < warp ? s : 0;
      tot += s;
    }
    __syncthreads();
    total = tot;
    return wpre + x - v;
  };

  for (int b = tid; b < 8 * NB; b += NT) (&hist[0][0])[b] = 0;
  if (tid == 0) {
    thr_s = NB - 1;  // fewer than C donors: every donor is below the threshold
    need_eq_s = 0;
  }
  __syncthreads();
  for (int j0 = V * tid; j0 < N; j0 += V * NT) {
    const uint4 a0 = load16(r0, j0), a1 = load16(r1, j0), a2 = load16(r2, j0);
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int j = j0 + k;
      if (j < N && j != i) atomicAdd(&hist[warp][byte_of(a0, k) + byte_of(a1, k) + byte_of(a2, k)], 1);
    }
  }
  __syncthreads();
  // threshold: the smallest T with #{score <= T} >= C; thread t owns bins 3t .. 3t+2
  {
    int c[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      int s = 0;
#pragma unroll
      for (int w2 = 0; w2 < 8; ++w2) s += hist[w2][3 * tid + e];
      c[e] = s;
    }
    int total;
    int acc = block_scan(c[0] + c[1] + c[2], total);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      if (acc < C && acc + c[e] >= C) {
        thr_s = 3 * tid + e;
        need_eq_s = C - acc;
      }
      acc += c[e];
    }
  }
  __syncthreads();
  const int T = thr_s, need_eq = need_eq_s;
  int base_sel = 0, eq_seen = 0;
  for (int jc = 0; jc < N; jc += V * NT) {  // the same trip count in every thread (block scans inside)
    const int j0 = jc + V * tid;
    uint32_t ltm = 0u, eqm = 0u;  // donors of this thread's 16 below / at the threshold
    if (j0 < N) {
      const uint4 a0 = load16(r0, j0), a1 = load16(r1, j0), a2 = load16(r2, j0);
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const int j = j0 + k;
        const int sc = (j < N && j != i) ? byte_of(a0, k) + byte_of(a1, k) + byte_of(a2, k) : 1 << 30;
        ltm |= (sc < T ? 1u : 0u) << k;
        eqm |= (sc == T ? 1u : 0u) << k;
      }
    }
    // equal scores are taken in ascending j until need_eq of them are in
    int eq_tot;
    int r = eq_seen + block_scan(__popc(eqm), eq_tot);
    uint32_t selm = ltm;
    for (uint32_t m = eqm; m; m &= m - 1u) {
      if (r < need_eq) selm |= m & (~m + 1u);
      ++r;
    }
    int sel_tot;
    int pos = base_sel + block_scan(__popc(selm), sel_tot);
    for (uint32_t m = selm; m; m &= m - 1u, ++pos) {
      if (pos >= C) break;
      const int j = j0 + __ffs(m) - 1;
      cand[(size_t)i * C + pos] = j;
      float f[kFeatUsed];
#pragma unroll
      for (int d = 0; d < kFeatUsed; ++d) f[d] = 1.0f - (float)a.Ms[d][(size_t)i * Np + j] * a.inv_nv[d];
      if (feat) {
        __nv_bfloat16* fo = feat + ((size_t)i * C + pos) * kFeat;
#pragma unroll
        for (int d = 0; d < kFeat; ++d) fo[d] = __float2bfloat16_rn(d < kFeatUsed ? f[d] : 0.0f);
      }
      if (feat32) {
        float* fo = feat32 + ((size_t)i * C + pos) * 8;
#pragma unroll
        for (int d = 0; d < 8; ++d) fo[d] = d < kFeatUsed ? f[d] : 0.0f;
      }
    }
    base_sel += sel_tot;
    eq_seen += eq_tot;
  }
  // fewer than C donors (C >= N): pad with -1
  for (int q = base_sel + tid; q < C; q += NT) cand[(size_t)i * C + q] = -1;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Stage 2, one block (256 threads) per target: the K best of C candidates by score (higher first,
// ties to the lower id; -1 entries last), written to idx[(i*Wn + w)*K ...] in ascending id order.
// Bitonic sorts in shared memory over P = next power of two >= C (<= 2048).
__global__ void topk_kernel(const int32_t* __restrict__ cand, const float* __restrict__ scores, int C, int K, int P,
                            int Wn, int w, int32_t* __restrict__ idx) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* key = reinterpret_cast<float*>(smem);
  int* val = reinterpret_cast<int*>(key + P);
  const int i = blockIdx.x;
  for (int q = threadIdx.x; q < P; q += blockDim.x) {
    const int j = q < C ? cand[(size_t)i * C + q] : -1;
    val[q] = j;
    key[q] = (j >= 0 && scores) ? scores[(size_t)i * C + q] : -3.0e38f;
  }
  __syncthreads();
  // order: higher key first, then lower id (ids >= 0 before -1)
  auto before = [&](int a, int b) -> bool {
    if (key[a] != key[b]) return key[a] > key[b];
    const unsigned ua = (unsigned)val[a], ub = (unsigned)val[b];
    return ua < ub;
  };
  for (int size = 2; size <= P; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int q = threadIdx.x; q < P; q += blockDim.x) {
        const int o = q ^ stride;
        if (o > q) {
          const bool up = (q & size) == 0;
          if (before(o, q) == up) {
            const float tk = key[q];
            key[q] = key[o];
            key[o] = tk;
            const int tv = val[q];
            val[q] = val[o];
            val[o] = tv;
          }
        }
      }
      __syncthreads();
    }
  // the first K by ascending id: sort ids of positions < K (others become +inf)
  for (int q = threadIdx.x; q < P; q += blockDim.x) {
    const int j = q < K ? val[q] : -1;
    val[q] = j;
  }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int q = threadIdx.x; q < P; q += blockDim.x) {
        const int o = q ^ stride;
        if (o > q) {
          const bool up = (q & size) == 0;
          const unsigned a = (unsigned)val[q], b = (unsigned)val[o];
          if ((a > b) == up) {
            val[q] = (int)b;
            val[o] = (int)a;
          }
        }
      }
      __syncthreads();
    }
  for (int q = threadIdx.x; q < K; q += blockDim.x) idx[((size_t)i * Wn + w) * K + q] = val[q];
}

// Training labels of the stage-1 candidates of one window, one thread per (target, candidate):
// y = 1 + log10(max(p_ij, floor)) / 12 with p_ij the dense posterior of candidate j for target i
// (row-major P [N][N]); 0 for padding (-1) and NaN for an id outside [0, N).
__global__ void label_kernel(const float* __restrict__ P, const int32_t* __restrict__ cand, int N, int C, float floor,
                             float* __restrict__ y) {
  const long long n = (long long)N * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int j = cand[e];
    float v = 0.0f;
    if (j >= N) v = __int_as_float(0x7fc00000);
    else if (j >= 0) v = 1.0f + log10f(fmaxf(P[(size_t)(e / C) * N + j], floor)) * (1.0f / 12.0f);
    y[e] = v;
  }
}

}  // namespace lsk
