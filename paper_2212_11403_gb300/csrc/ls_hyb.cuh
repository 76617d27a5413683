// ls_hyb.cuh -- dense propagation for large N: one target per CTA of 512 threads, the target's
// state split between registers and shared memory.
//
// Thread t owns donor positions [B t, B (t+1)), B = 4 (QR + QS): its first QR quads of 4 cells stay
// in registers for all loci, the other QS quads sit in shared memory in quad-major order
// ([QS][512] float4, so a warp's 16-byte accesses are contiguous).  With QR = 12 the registers hold
// 24576 positions per target and shared memory up to 16 x 8 KB more (N <= 57344).  Per locus a
// thread reads the packed bits of its positions from the (L2-resident) packed row one locus ahead,
// XORs them with the target's allele and takes the emission per cell by a bit test (no emission table,
// so shared-memory traffic is the state of the QS quads only: 8 bytes per cell there, none in the
// register part), and updates x <- theta (c x + r) as (c b) x + r b with b = max(1-mu, mu), followed
// by a predicated multiply by min(1-mu, mu) / b on the cells whose emission is the smaller value
// (FFMA2, FMUL, FADD2).  Positions beyond N and the target's own position always take the smaller
// factor: they all start at 0 and see the same operations, so they hold one common value xs,
// replicated in every thread, and the row sum subtracts n_junk * xs (the register-tile kernel's
// treatment).  The row
// sum is a shuffle tree, one CTA barrier and a 16-entry sum; FP64 log scales are accumulated by
// thread 0.
//
// Cluster variant (CL = 2, N up to 2 x 57344): a target's positions are split between the two CTAs
// of a thread-block cluster on two SMs, CTA rank r holding positions [r NP, (r+1) NP).  Per locus
// every warp writes its partial sum into both CTAs' shared memory (distributed shared memory), one
// cluster barrier publishes them, and both CTAs add the 32 partials in the same fixed order, so they
// hold bit-identical normalisers.
//
// Prior matrix (PIM = 1, Sec. 2.1 copying prior Pi): the target's prior row stays on chip for all
// loci as bfloat16, four values per 8 bytes in the same quad-major order ([Q][512] in shared
// memory, 8 bytes per position quad), which is why these variants need the BF16 prior format (the
// context rounds Pi once, so the conversion here is exact).  The forward adds rho * pi_j per cell
// (one more multiply), the backward normaliser is sum_j pi_j t_j (an FMA in place of the add);
// padding and the target's own position have pi = 0, so no junk correction is needed.  The
// register quads are staged through no shared memory: at stores every thread writes its own
// positions.
#pragma once

#include <cuda_bf16.h>

#include "ls_prop.cuh"

namespace lsk {

constexpr int kHybThreads = 512;
constexpr int kHybQR = 12;  // register quads per thread

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// all threads of every CTA of the cluster; release/acquire order shared-memory writes (local and
// remote) before the barrier with reads after it
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// store v at the same shared-memory offset as `local` in CTA `rank` of the cluster
__device__ __forceinline__ void st_cluster(float* local, uint32_t rank, float v) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_u32(local)), "r"(rank));
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v) : "memory");
}

constexpr int kHybPimMaxN1 = kHybThreads * 4 * (kHybQR + 14);  // largest N of one CTA with a prior matrix

template <int QS, int PIM = 0>
struct HybCfg {
  static constexpr int Q = kHybQR + QS;       // quads per thread
  static constexpr int B = 4 * Q;             // positions per thread
  static constexpr int NP = kHybThreads * B;  // positions per target (N <= NP)
  static constexpr int NWA = (B + 31) / 32;   // aligned match words per thread
  static constexpr int NW = NWA + 1;          // row words read per thread (funnel shift)
  // dynamic shared memory: the QS shared quads [QS][512] (float4 each); with a prior matrix the
  // prior quads [Q][512] (4 x bf16 each), else the staging of the register quads at store loci
  // [QR][512] (float4 each); two buffers of 32 warp partials
  static constexpr int XS_OFF = 0;
  static constexpr int PS_OFF = XS_OFF + QS * kHybThreads * 16;
  static constexpr int STG_OFF = PS_OFF + (PIM ? Q * kHybThreads * 8 : 0);
  static constexpr int PART_OFF = STG_OFF + (PIM ? 0 : kHybQR * kHybThreads * 16);
  static constexpr int BYTES = PART_OFF + 2 * 32 * 4;
  __host__ __device__ static int smem_bytes() { return BYTES; }
  // beyond the register-tile kernels' range (N <= 20480); with CL CTAs per target, beyond the
  // one-CTA range (N <= 57344; with a prior matrix N <= 53248)
  __host__ __device__ static bool serves(int N, int CL = 1) {
    return CL == 1 ? (N > 20480 && N <= NP) : (N > (PIM ? kHybPimMaxN1 : 57344) && N <= CL * NP);
  }
};

template <int DIR, int QS, int CL, int PIM = 0>
__global__ void __launch_bounds__(kHybThreads, 1) ls_hyb_kernel(const PropParams p) {
  static_assert(CL == 1 || CL == 2, "one CTA or a cluster of two per target");
  using C = HybCfg<QS, PIM>;
  constexpr int QR = kHybQR, Q = C::Q, B = C::B, NWA = C::NWA, NW = C::NW, T = kHybThreads;
  constexpr int step_dir = DIR == 0 ? 1 : -1;
  extern __shared__ __align__(128) unsigned char smem[];
  float4* Xs = reinterpret_cast<float4*>(smem + C::XS_OFF);    // [QS][T] shared quads
  float4* Stg = reinterpret_cast<float4*>(smem + C::STG_OFF);  // [QR][T] register quads at stores
  uint2* Ps = reinterpret_cast<uint2*>(smem + C::PS_OFF);      // [Q][T] prior quads (PIM)
  float* part = reinterpret_cast<float*>(smem + C::PART_OFF);  // [2][32]
  const int N = p.N, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rank = CL == 2 ? (int)cluster_rank() : 0;
  const int cta_t = p.t_begin + blockIdx.x / CL;  // one target per CTA or cluster (or its list position)
  const int tgt = p.tlist ? p.tlist[cta_t] : cta_t;
  const int row = cta_t - p.tab_t0;
  const int pos0 = rank * C::NP;  // first position of this CTA
  const int d0 = pos0 + B * tid;  // first position of this thread
  const int w0 = d0 >> 5;
  const uint32_t sh = (uint32_t)(d0 & 31);
  const float n_junk = (float)(CL * C::NP - (N - 1));
  if (CL == 2) cluster_sync();  // both CTAs are running before any remote shared-memory store

  // valid positions of the aligned match words: position d0 + 32 k + b is a donor iff it is < N
  // and not the target (bits beyond the thread's B positions are cleared too)
  uint32_t vm[NWA];
#pragma unroll
  for (int k = 0; k < NWA; ++k) {
    uint32_t m = 0u;
    for (int b = 0; b < 32; ++b) {
      const int o = 32 * k + b, pos = d0 + o;
      if (o < B && pos < N && pos != tgt) m |= 1u << b;
    }
    vm[k] = m;
  }
  if (PIM) {  // this thread's prior values as bfloat16 pairs (0 on padding and on the target)
    const float* prow = p.Pi + (size_t)tgt * N;
    for (int q = 0; q < Q; ++q) {
      uint32_t hb[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int pos = d0 + 4 * q + e;
        hb[e] = __bfloat16_as_ushort(__float2bfloat16_rn((pos < N && pos != tgt) ? prow[pos] : 0.0f));
      }
      Ps[q * T + tid] = make_uint2(hb[0] | (hb[1] << 16), hb[2] | (hb[3] << 16));
    }
  }

  // element e of quad q of thread t: shared or staged location (quad-major)
  auto elem = [&](int q, int t, int e) -> float* {
    float4* base = q < QR ? Stg + q * T + t : Xs + (q - QR) * T + t;
    return reinterpret_cast<float*>(base) + e;
  };

  f2 x[QR][2];
#pragma unroll
  for (int q = 0; q < QR; ++q) x[q][0] = x[q][1] = make_float2(0.f, 0.f);
  if (p.load_state && PIM) {  // every thread reads its own positions
    auto ld = [&](int pos) -> float { return (pos < N && pos != tgt) ? p.state[(size_t)row * N + pos] : 0.0f; };
#pragma unroll
    for (int q = 0; q < QR; ++q) {
      x[q][0] = make_float2(ld(d0 + 4 * q), ld(d0 + 4 * q + 1));
      x[q][1] = make_float2(ld(d0 + 4 * q + 2), ld(d0 + 4 * q + 3));
    }
    for (int q = QR; q < Q; ++q) {
      const int b4 = d0 + 4 * q;
      Xs[(q - QR) * T + tid] = make_float4(ld(b4), ld(b4 + 1), ld(b4 + 2), ld(b4 + 3));
    }
    __syncthreads();
  } else if (p.load_state) {
    for (int i = tid; i < C::NP; i += T) {
      const int t = i / B, o = i - t * B, g = pos0 + i;
      *elem(o >> 2, t, o & 3) = (g < N && g != tgt) ? p.state[(size_t)row * N + g] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < QR; ++q) {
      const float4 v = Stg[q * T + tid];
      x[q][0] = make_float2(v.x, v.y);
      x[q][1] = make_float2(v.z, v.w);
    }
    __syncthreads();
  } else {
    for (int i = tid; i < QS * T; i += T) Xs[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }

  auto reduce = [&](float v, int buf) -> float {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (CL == 1) {
      if (lane == 0) part[buf * 32 + warp] = v;
      __syncthreads();
      float t = part[buf * 32 + (lane & 15)];  // both half-warps sum the 16 partials
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      return t;
    }
    // partial of warp w of CTA r at slot 16 r + w, in both CTAs; every lane sums the 32 slots
    if (lane == 0) {
      float* slot = part + buf * 32 + 16 * rank + warp;
      *slot = v;
      st_cluster(slot, (uint32_t)(rank ^ 1), v);
    }
    cluster_sync();
    float t = part[buf * 32 + lane];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    return t;
  };
  // store the row (x, or c x + r when affine) to w1 / multiply m1 by it / w2 (any may be null)
  auto store_state = [&](float* w1, float* m1, float* w2, bool affine, float c, float r) {
    if (PIM && m1 && !w1 && !w2) {  // decode products: a quad's four loads ahead of its stores
      auto put4 = [&](int pos, float x0, float x1, float x2, float x3) {
        const float xv[4] = {x0, x1, x2, x3};
        float gv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          gv[e] = (pos + e < N && pos + e != tgt) ? m1[(size_t)row * N + pos + e] : 0.0f;
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (pos + e < N) {
            const float v = pos + e == tgt ? 0.0f : (affine ? fmaf(c, xv[e], r) : xv[e]);
            m1[(size_t)row * N + pos + e] = pos + e == tgt ? 0.0f : gv[e] * (v * kProdScale);
          }
      };
#pragma unroll
      for (int q = 0; q < QR; ++q) put4(d0 + 4 * q, x[q][0].x, x[q][0].y, x[q][1].x, x[q][1].y);
      for (int q = QR; q < Q; ++q) {
        const float4 v = Xs[(q - QR) * T + tid];
        put4(d0 + 4 * q, v.x, v.y, v.z, v.w);
      }
      return;
    }
    if (PIM) {  // every thread writes its own positions
      auto put = [&](int pos, float xv) {
        if (pos >= N) return;
        const float v = pos == tgt ? 0.0f : (affine ? fmaf(c, xv, r) : xv);
        const size_t ro = (size_t)row * N + pos;
        if (w1) w1[ro] = v;
        if (m1) m1[ro] = pos == tgt ? 0.0f : m1[ro] * (v * kProdScale);
        if (w2) w2[ro] = v;
      };
#pragma unroll
      for (int q = 0; q < QR; ++q) {
        put(d0 + 4 * q, x[q][0].x);
        put(d0 + 4 * q + 1, x[q][0].y);
        put(d0 + 4 * q + 2, x[q][1].x);
        put(d0 + 4 * q + 3, x[q][1].y);
      }
      for (int q = QR; q < Q; ++q) {
        const float4 v = Xs[(q - QR) * T + tid];
        put(d0 + 4 * q, v.x);
        put(d0 + 4 * q + 1, v.y);
        put(d0 + 4 * q + 2, v.z);
        put(d0 + 4 * q + 3, v.w);
      }
      return;
    }
#pragma unroll
    for (int q = 0; q < QR; ++q) Stg[q * T + tid] = make_float4(x[q][0].x, x[q][0].y, x[q][1].x, x[q][1].y);
    __syncthreads();
    const int iend = min(C::NP, N - pos0);
    if (m1 && !w1 && !w2) {
      // decode products: a thread's loads of kXB elements go out ahead of their stores (the
      // compiler cannot tell a store from later loads, so each load would otherwise wait for the
      // previous element's store)
      constexpr int kXB = 8;
      for (int i0 = tid; i0 < iend; i0 += T * kXB) {
        float gv[kXB];
#pragma unroll
        for (int b = 0; b < kXB; ++b) {
          const int i = i0 + b * T, g = pos0 + i;
          gv[b] = (i < iend && g != tgt) ? m1[(size_t)row * N + g] : 0.0f;
        }
#pragma unroll
        for (int b = 0; b < kXB; ++b) {
          const int i = i0 + b * T;
          if (i < iend) {
            const int t = i / B, o = i - t * B, g = pos0 + i;
            const float xv = *elem(o >> 2, t, o & 3);
            const float v = g == tgt ? 0.0f : (affine ? fmaf(c, xv, r) : xv);
            m1[(size_t)row * N + g] = g == tgt ? 0.0f : gv[b] * (v * kProdScale);
          }
        }
      }
      __syncthreads();
      return;
    }
    for (int i = tid; i < iend; i += T) {
      const int t = i / B, o = i - t * B, g = pos0 + i;
      const float xv = *elem(o >> 2, t, o & 3);
      const float v = g == tgt ? 0.0f : (affine ? fmaf(c, xv, r) : xv);
      const size_t ro = (size_t)row * N + g;
      if (w1) w1[ro] = v;
      if (m1) m1[ro] = g == tgt ? 0.0f : m1[ro] * (v * kProdScale);
      if (w2) w2[ro] = v;
    }
    __syncthreads();
  };

  float sig_prev = 1.0f, xs = 0.0f;
  if (p.load_state && DIR == 0) {
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < QR; ++q) s += (x[q][0].x + x[q][0].y) + (x[q][1].x + x[q][1].y);
#pragma unroll
    for (int q = 0; q < QS; ++q) {
      const float4 v = Xs[q * T + tid];
      s += (v.x + v.y) + (v.z + v.w);
    }
    sig_prev = reduce(s, 1);
    __syncthreads();
  }
  double lgs = (tid == 0 && p.logs && !p.init) ? p.logs[row] : 0.0;
  float lsum = 0.0f, lerr = 0.0f;  // logs of the normalisers since the last fold into lgs
  float u_base = 1.0f, u_ratio = 0.0f;  // emission base and ratio (per locus only with a per-locus mu)
  uint32_t sts = 0u;
  int store_next = 0;
  int next_store_l = p.n_store > 0 ? p.store_loci[0] : -1;
  int pend_slot = -1;
  bool pend_save = false;

  // the row words holding this thread's bits, the target's bit and the locus' emission values,
  // loaded one locus ahead
  uint32_t wd[NW], tb;
  float nthm, nthx;
  auto load_locus = [&](int l, bool with_mu) {  // with_mu: also the locus' emission values
    const uint32_t* r = p.bits2 + (size_t)l * p.rw2;
#pragma unroll
    for (int k = 0; k < NW; ++k) wd[k] = (w0 + k < p.rw2) ? r[w0 + k] : 0u;
    tb = (r[tgt >> 5] >> (tgt & 31)) & 1u;
    if (with_mu) {
      nthm = p.thm[l];
      nthx = p.thx[l];
    }
  };
  load_locus(p.l_first, true);
  // One locus.  EV (compile-time) marks the steps with an event (the first step, a store locus, the
  // step after it, the last step): the other steps run a copy without those branches.  MUV
  // (compile-time): mu varies per locus (otherwise the first locus' emission values serve all).
  auto body = [&](const int step, auto evc, auto muvc) {
    constexpr bool EV = decltype(evc)::value;
    constexpr bool MUV = decltype(muvc)::value;
    const int l = p.l_first + step_dir * step;
    uint32_t cw[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) cw[k] = wd[k];
    const uint32_t ctb = tb;
    const float thm = nthm, thx = nthx;
    if (step + 1 < p.n_steps) load_locus(l + step_dir, MUV);
    float c, r;
    bool add_log_prev = false;
    const int mi = DIR == 0 ? l - 1 : l;
    if (EV && step == 0 && p.init) {
      c = 0.0f;
      r = (DIR == 0 && !PIM) ? p.pi_u : 1.0f;  // alpha^0 = theta pi ; beta^{L-1} = 1
    } else if (EV && step == 0 && DIR == 1) {
      c = 1.0f;  // backward resume: x = theta^l beta^l from the stored beta
      r = 0.0f;
    } else {
      c = __fdividef(p.omr[mi], sig_prev);
      r = p.rr[mi];
      add_log_prev = DIR == 1;
    }
    const bool is_store = EV && l == next_store_l;
    const bool save_here = EV && p.save_state && step == p.n_steps - 1;
    if (EV && DIR == 0 && pend_slot >= 0) {  // alpha of the previous locus
      store_state(p.store + (size_t)pend_slot * p.state_rows * N, nullptr, nullptr, false, 0.f, 0.f);
      pend_slot = -1;
    }
    if (EV && DIR == 1 && pend_slot >= 0) {  // decode product of the previous locus: alpha^l t^l, t = theta beta
      store_state(nullptr, p.alpha_dec + (size_t)pend_slot * p.state_rows * N, nullptr, false, 0.f, 0.f);
      pend_slot = -1;
    }
    if (EV && DIR == 1 && ((is_store && p.store) || save_here)) {
      // beta^l = c t^{l+1} + rho (tables and stored rows)
      const size_t so = (size_t)(is_store ? p.store_slot[store_next] : 0) * p.state_rows * N;
      store_state((is_store && p.store) ? p.store + so : nullptr, nullptr, save_here ? p.state : nullptr, true, c, r);
    }

    // Emission as base x f, base = max(1-mu, mu), f in {1, ratio}: a cell is (c base) x + r base,
    // then multiplied by ratio where f = ratio (a predicated multiply, no select).  The "small" bits
    // (f = ratio) are the mismatches, or the matches when mu > 1/2; junk positions have bit 0.
    if (MUV || (EV && step == 0)) {
      u_base = fmaxf(thm, thx);
      u_ratio = u_base > 0.0f ? __fdiv_rn(fminf(thm, thx), u_base) : 0.0f;
    }
    // match bits of the thread's positions (bit o of aw[o >> 5] <-> position d0 + o)
    const uint32_t inv = (ctb ? 0u : 0xffffffffu) ^ (thm < thx ? 0xffffffffu : 0u);
    uint32_t aw[NWA];
#pragma unroll
    for (int k = 0; k < NWA; ++k) aw[k] = (funnel(cw[k], cw[k + 1], sh) ^ inv) & vm[k];
    const float cu = c * u_base, ru = r * u_base;
    const f2 C2 = make_float2(cu, cu), R2 = make_float2(ru, ru);
    f2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    auto emit = [&](f2 u01, f2 u23, uint32_t w, int b, f2& o01, f2& o23) {
      float a0 = u01.x, a1 = u01.y, a2 = u23.x, a3 = u23.y;
      if (!((w >> b) & 1u)) a0 = __fmul_rn(a0, u_ratio);
      if (!((w >> (b + 1)) & 1u)) a1 = __fmul_rn(a1, u_ratio);
      if (!((w >> (b + 2)) & 1u)) a2 = __fmul_rn(a2, u_ratio);
      if (!((w >> (b + 3)) & 1u)) a3 = __fmul_rn(a3, u_ratio);
      o01 = make_float2(a0, a1);
      o23 = make_float2(a2, a3);
    };
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const uint32_t w = aw[(4 * q) >> 5];
      const int b = (4 * q) & 31;
      f2 p01 = make_float2(0.f, 0.f), p23 = make_float2(0.f, 0.f);
      if (PIM) {  // the prior quad, bfloat16 -> FP32 (exact)
        const uint2 pb = Ps[q * T + tid];
        p01 = make_float2(__uint_as_float(pb.x << 16), __uint_as_float(pb.x & 0xffff0000u));
        p23 = make_float2(__uint_as_float(pb.y << 16), __uint_as_float(pb.y & 0xffff0000u));
      }
      // u = c x + r (forward with a prior matrix: c x + r pi_j)
      auto pre = [&](f2 xv, f2 pv) -> f2 {
        return (PIM && DIR == 0) ? __ffma2_rn(C2, xv, __fmul2_rn(R2, pv)) : __ffma2_rn(C2, xv, R2);
      };
      // the normaliser: sum_j x_j (backward with a prior matrix: sum_j pi_j t_j)
      auto add = [&](f2 a, f2 y, f2 pv) -> f2 { return (PIM && DIR == 1) ? __ffma2_rn(y, pv, a) : __fadd2_rn(a, y); };
      if (q < QR) {
        const int qr = q < QR ? q : 0;
        emit(pre(x[qr][0], p01), pre(x[qr][1], p23), w, b, x[qr][0], x[qr][1]);
        acc0 = add(acc0, x[qr][0], p01);
        acc1 = add(acc1, x[qr][1], p23);
      } else {
        float4* sp = Xs + (q - QR) * T + tid;
        const float4 v = *sp;
        f2 y01, y23;
        emit(pre(make_float2(v.x, v.y), p01), pre(make_float2(v.z, v.w), p23), w, b, y01, y23);
        *sp = make_float4(y01.x, y01.y, y23.x, y23.y);
        acc0 = add(acc0, y01, p01);
        acc1 = add(acc1, y23, p23);
      }
    }
    xs = __fmul_rn(u_ratio, __fmaf_rn(cu, xs, ru));  // junk positions: always the "small" factor

    if (DIR == 0) {  // alpha^l is stored at the top of the next step (or after the loop)
      pend_slot = is_store && p.store ? p.store_slot[store_next] : -1;
      pend_save = save_here;
    } else {  // decoding: alpha^l times t^l at the top of the next step (decode_kernel divides by theta)
      pend_slot = is_store && p.alpha_dec ? p.store_slot[store_next] : -1;
    }
    if (is_store) {
      ++store_next;
      next_store_l = store_next < p.n_store ? p.store_loci[store_next] : -1;
    }
    float sig = reduce((acc0.x + acc0.y) + (acc1.x + acc1.y), step & 1) - (PIM ? 0.0f : n_junk * xs);
    if (DIR == 1 && !PIM) sig *= p.pi_u;
    if (tid == 0) {
      const float sg = DIR == 0 ? sig : (add_log_prev ? sig_prev : 1.0f);
      if (sg < 1.17549435e-38f) sts |= 1u;      // LS_STATUS_UNDERFLOW
      if (!(sg <= 3.40282347e+38f)) sts |= 2u;  // LS_STATUS_OVERFLOW
      // FP32 sum with an exact error term per addition (two-sum), taken into the FP64 log scale
      // every 32 loci
      const float lv = logf(sg);
      const float s2 = __fadd_rn(lsum, lv);
      const float bb = __fsub_rn(s2, lsum);
      lerr = __fadd_rn(lerr, __fadd_rn(__fsub_rn(lsum, __fsub_rn(s2, bb)), __fsub_rn(lv, bb)));
      lsum = s2;
      if ((step & 31) == 31 || step == p.n_steps - 1) {
        lgs += (double)lsum + (double)lerr;
        lsum = 0.0f;
        lerr = 0.0f;
      }
    }
    sig_prev = sig;
  };
  auto run_steps = [&](auto muvc) {
    for (int step = 0; step < p.n_steps;) {
      // the next event step: the first and the last step, now if a store is pending, else the next
      // store locus
      int ev = step == 0 ? 0 : p.n_steps - 1;
      if (pend_slot >= 0) ev = step;
      else if (next_store_l >= 0) ev = min(ev, (next_store_l - p.l_first) * step_dir);
      for (; step < ev; ++step) body(step, std::false_type{}, muvc);
      if (step < p.n_steps) body(step++, std::true_type{}, muvc);
    }
  };
  if (p.mu_vec) run_steps(std::true_type{});
  else run_steps(std::false_type{});
  if (DIR == 1 && pend_slot >= 0)  // decode product of the last locus
    store_state(nullptr, p.alpha_dec + (size_t)pend_slot * p.state_rows * N, nullptr, false, 0.f, 0.f);
  if (DIR == 0 && (pend_slot >= 0 || pend_save))
    store_state(pend_slot >= 0 ? p.store + (size_t)pend_slot * p.state_rows * N : nullptr, nullptr,
                pend_save ? p.state : nullptr, false, 0.f, 0.f);
  if (tid == 0 && rank == 0 && cta_t < p.t_begin + p.t_count) {
    if (p.logs) p.logs[row] = lgs;
    if (p.status && sts) atomicOr(p.status + row, sts);
  }
  if (CL == 2) cluster_sync();  // no CTA leaves while its peer may still address its shared memory
}

}  // namespace lsk
