// ls_warp.cuh -- one-warp-per-target propagation kernel (N <= 32 * 4KQ, uniform prior).
//
// Same recursions, emission table, junk-cell handling and doubled rows as ls_prop_kernel, but
// every target lives in one warp: lane q holds slice q of the N donor positions (rotated by the
// CTA's first target o, so target o+w's own cell sits at slot w of lane 0).  The row sum of a
// locus is then five shuffles, with no shared memory and no CTA barrier, and the warps of an SM
// drift freely so that one warp's reduction latency is covered by the others' arithmetic.
//
// The four warps of a CTA (targets o..o+3) share the TMA ring of packed rows.  A slot is refilled
// by whichever warp is the last to finish the block it held (a shared counter per slot); the
// other warps never wait for it, and consumers wait on the slot's mbarrier with a time bound.
#pragma once

#include "ls_prop.cuh"

namespace lsk {

constexpr int kWarpTargets = 4;  // targets (warps) per CTA

template <int KQ>
struct WarpCfg {
  static constexpr int J = 4 * KQ;
  static constexpr int NWORD = (J + 31) / 32;
  static constexpr int BAR_OFF = 0;
  static constexpr int CNT_OFF = kSlots * 8;
  static constexpr int FLAG_OFF = CNT_OFF + kSlots * 4;
  static constexpr int NCHUNK = (KQ + 7) / 8;   // 32-slot chunks staged through shared memory
  static constexpr int STG = 36;                // floats per lane in a warp's staging chunk
  static constexpr int STG_OFF = 128;
  static constexpr int RING_OFF = STG_OFF + kWarpTargets * 32 * STG * 4;
  __host__ __device__ static int smem_bytes(int rw2) { return RING_OFF + kSlots * kRB * rw2 * 4; }
  // a lane's slice must fit its slots, only its last word may be partial, and slice 0 must hold
  // the four diagonal positions
  __host__ __device__ static bool serves(int N) {
    const int Jr = (N + 31) / 32;
    return N >= 8 && Jr >= kWarpTargets && Jr <= J && (NWORD == 1 || Jr - 1 >= 32 * (NWORD - 1));
  }
};

template <int DIR, int KQ>
__global__ void __launch_bounds__(kWarpTargets * 32, 2) ls_warp_kernel(const PropParams p) {
  using C = WarpCfg<KQ>;
  constexpr int NWORD = C::NWORD;
  constexpr int step_dir = DIR == 0 ? 1 : -1;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::BAR_OFF);
  int* cnt = reinterpret_cast<int*>(smem + C::CNT_OFF);
  volatile int* flag = reinterpret_cast<volatile int*>(smem + C::FLAG_OFF);
  uint32_t* ring = reinterpret_cast<uint32_t*>(smem + C::RING_OFF);
  float* stg = reinterpret_cast<float*>(smem + C::STG_OFF) + (threadIdx.x >> 5) * 32 * C::STG;
  // per-warp emission tables, two 256-byte buffers each (this locus and the next when mu varies)
  __shared__ __align__(256) float s_lut[kWarpTargets][2][64];

  const int N = p.N, rw2 = p.rw2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int o = p.t_begin + blockIdx.x * kWarpTargets;  // first target of the CTA
  const int tgt = o + warp;                              // this warp's target
  const int t_end = p.t_begin + p.t_count;
  const bool active = tgt < t_end;
  const int row = tgt - p.tab_t0;
  int start, len;
  slice_of(lane, 32, N, start, len);
  const int b0 = start + o;
  const int wb = b0 >> 5;
  const uint32_t wsh = (uint32_t)(b0 & 31);
  const int abit = tgt;
  const float n_junk = (float)(32 * C::J - (N - 1));
  const uint32_t dclear = lane == 0 ? ~(1u << warp) : 0xffffffffu;  // own cell = slot `warp` of lane 0
  const int vl = len - 32 * (NWORD - 1);
  const uint32_t vmask_last = vl >= 32 ? 0xffffffffu : (vl <= 0 ? 0u : ((1u << vl) - 1u));
  float* lutw = &s_lut[warp][0][0];

  auto blk_rows = [&](int B, int& base, int& nrows) {
    nrows = min(kRB, p.n_steps - kRB * B);
    base = DIR == 0 ? p.l_first + kRB * B : p.l_first - kRB * B - (nrows - 1);
  };
  auto issue = [&](int B) {
    int base, nrows;
    blk_rows(B, base, nrows);
    tma_row(ring + (B % kSlots) * kRB * rw2, p.bits2 + (size_t)base * rw2, (uint32_t)(nrows * rw2 * 4), &bars[B % kSlots]);
  };
  const int nblk = (p.n_steps + kRB - 1) / kRB;
  if (tid == 0) {
    *flag = 0;
    for (int s = 0; s < kSlots; ++s) {
      mbar_init(&bars[s], 1);
      cnt[s] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (lane < 16) {  // emission table of the first locus (for scalar mu: of every locus)
    const int e = lane;
    const float tm = p.thm[p.l_first], tx = p.thx[p.l_first];
    *reinterpret_cast<float4*>(lutw + 4 * e) =
        make_float4((e & 1) ? tm : tx, (e & 2) ? tm : tx, (e & 4) ? tm : tx, (e & 8) ? tm : tx);
  }
  __syncthreads();
  if (tid == 0)
    for (int B = 0; B < kSlots && B < nblk; ++B) issue(B);

  // transfers between the register tile and a table row (store loci and resumes only), one 32-slot
  // chunk at a time through the warp's staging area: slot s of lane q <-> donor (start_q + s + o)
  // mod N, so the 32 lanes write 32 consecutive donors of one source lane at a time.  The
  // target's own cell reads and writes 0.
  f2 x[KQ][2];
#pragma unroll
  for (int k = 0; k < KQ; ++k) x[k][0] = x[k][1] = make_float2(0.f, 0.f);
  // out: w1 = value, m1 *= value, w2 = value (any may be null); value = affine ? c x + r : x
  auto store_regs = [&](bool affine, float c, float r, float* w1, float* m1, float* w2) {
    const size_t ro = (size_t)row * N;
#pragma unroll
    for (int cc = 0; cc < C::NCHUNK; ++cc) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = 8 * cc + q;
        if (k < KQ) {
          const f2 a = affine ? __ffma2_rn(make_float2(c, c), x[k][0], make_float2(r, r)) : x[k][0];
          const f2 b = affine ? __ffma2_rn(make_float2(c, c), x[k][1], make_float2(r, r)) : x[k][1];
          *reinterpret_cast<float4*>(stg + lane * C::STG + 4 * q) = make_float4(a.x, a.y, b.x, b.y);
        }
      }
      __syncwarp();
      if (active) {
#pragma unroll 1
        for (int q = 0; q < 32; ++q) {
          int sq, lq;
          slice_of(q, 32, N, sq, lq);
          const int sl = 32 * cc + lane;
          if (sl < lq) {
            int d = sq + sl + o;
            d = d >= N ? d - N : d;
            const bool diag = q == 0 && sl == warp;
            const float v = diag ? 0.0f : stg[q * C::STG + lane];
            if (w1) w1[ro + d] = v;
            if (m1) m1[ro + d] = diag ? 0.0f : m1[ro + d] * v;
            if (w2) w2[ro + d] = v;
          }
        }
      }
      __syncwarp();
    }
  };
  if (p.load_state) {
    const float* g = p.state + (size_t)row * N;
#pragma unroll
    for (int cc = 0; cc < C::NCHUNK; ++cc) {
#pragma unroll 1
      for (int q = 0; q < 32; ++q) {
        int sq, lq;
        slice_of(q, 32, N, sq, lq);
        const int sl = 32 * cc + lane;
        int d = sq + sl + o;
        d = d >= N ? d - N : d;
        stg[q * C::STG + lane] = (active && sl < lq && !(q == 0 && sl == warp)) ? g[d] : 0.0f;
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = 8 * cc + q;
        if (k < KQ) {
          const float4 v = *reinterpret_cast<const float4*>(stg + lane * C::STG + 4 * q);
          x[k][0] = make_float2(v.x, v.y);
          x[k][1] = make_float2(v.z, v.w);
        }
      }
      __syncwarp();
    }
  }
  auto warp_sum = [&](float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
  };

  float sig_prev = 1.0f;
  float xs = 0.0f;  // common value of the junk cells
  if (p.load_state && DIR == 0) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < KQ; ++k) s += (x[k][0].x + x[k][0].y) + (x[k][1].x + x[k][1].y);
    sig_prev = warp_sum(s);
  }
  double lgs = (active && p.logs && !p.init) ? p.logs[row] : 0.0;  // held by every lane, updated alike
  uint32_t sts = 0u;
  float my_sg = 1.0f;  // this lane's entry of the 32-step ring of normalisers

  float nx_omr = 0.f, nx_rr = 0.f, nx_thx = p.thx[p.l_first], nx_thm = p.thm[p.l_first];
  {
    const int li = DIR == 0 ? p.l_first - 1 : p.l_first;
    if (li >= 0 && li < p.L - 1) {
      nx_omr = p.omr[li];
      nx_rr = p.rr[li];
    }
  }
  int store_next = 0;
  int next_store_l = p.n_store > 0 ? p.store_loci[0] : -1;
  int pend_slot = -1;
  bool pend_save = false;
  const uint32_t* slot_rows = ring;
  int blk_base = 0, blk_n = 0, blk = 0;
  for (int step = 0; step < p.n_steps; ++step) {
    const int l = p.l_first + step_dir * step;
    const float cur_omr = nx_omr, cur_rr = nx_rr, cur_thx = nx_thx;
    if (step + 1 < p.n_steps) {
      const int ln = l + step_dir;
      const int li = DIR == 0 ? ln - 1 : ln;
      nx_omr = p.omr[li];
      nx_rr = p.rr[li];
      nx_thx = p.thx[ln];
      nx_thm = p.thm[ln];
    }
    const int j = step & (kRB - 1);
    if (j == 0) {
      blk = step / kRB;
      mbar_wait_bounded(&bars[blk % kSlots], (uint32_t)((blk / kSlots) & 1), flag);
      slot_rows = ring + (blk % kSlots) * kRB * rw2;
      blk_rows(blk, blk_base, blk_n);
    }
    const uint32_t* rw = slot_rows + (l - blk_base) * rw2;

    float c, r;
    bool add_log_prev = false;
    if (step == 0 && p.init) {
      c = 0.0f;
      r = DIR == 0 ? p.pi_u : 1.0f;
    } else if (step == 0 && DIR == 1) {
      c = 1.0f;
      r = 0.0f;
    } else {
      c = __fdividef(cur_omr, sig_prev);
      r = cur_rr;
      add_log_prev = DIR == 1;
    }
    const bool is_store = l == next_store_l;
    const bool save_here = p.save_state && step == p.n_steps - 1;
    if (DIR == 0 && pend_slot >= 0) {
      store_regs(false, 0.f, 0.f, p.store + (size_t)pend_slot * p.state_rows * N, nullptr, nullptr);
      pend_slot = -1;
    }
    if (DIR == 1 && (is_store || save_here)) {
      // beta^l = c t^{l+1} + rho into the store, times alpha in place for decoding, and the state
      const size_t so = (size_t)(is_store ? p.store_slot[store_next] : 0) * p.state_rows * N;
      store_regs(true, c, r, (is_store && p.store) ? p.store + so : nullptr,
                 (is_store && p.alpha_dec) ? p.alpha_dec + so : nullptr, save_here ? p.state : nullptr);
    }

    const uint32_t inv = ((rw[abit >> 5] >> (abit & 31)) & 1u) ? 0u : 0xffffffffu;
    const uint32_t lut_b = (uint32_t)(warp * 512) + (p.mu_vec ? (uint32_t)((step & 1) << 8) : 0u);
    const f2 C2 = make_float2(c, c), R2 = make_float2(r, r);
    f2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    constexpr int kLA = KQ < 4 ? KQ : 4;
    uint32_t hw[2], lw[2];
    float4 th[kLA];
    auto prep_word = [&](int m) {
      uint32_t wd = funnel(rw[wb + m], rw[wb + m + 1], wsh) ^ inv;
      if (m == NWORD - 1) wd &= vmask_last;
      if (m == 0) wd &= dclear;
      hw[m & 1] = wd & 0xf0f0f0f0u;
      lw[m & 1] = (wd << 4) & 0xf0f0f0f0u;
    };
    auto load_th = [&](int kk) -> float4 {
      const int q = kk & 7, m = kk >> 3;
      const uint32_t off = __byte_perm((q & 1) ? hw[m & 1] : lw[m & 1], lut_b, 0x7650u | (uint32_t)(q >> 1));
      return *reinterpret_cast<const float4*>(reinterpret_cast<const unsigned char*>(&s_lut[0][0][0]) + off);
    };
    prep_word(0);
#pragma unroll
    for (int k = 0; k < kLA; ++k) th[k] = load_th(k);
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
      const float4 t = th[k % kLA];
      const int kn = k + kLA;
      if (kn < KQ) {
        if ((kn & 7) == 0) prep_word(kn >> 3);
        th[k % kLA] = load_th(kn);
      }
      const f2 u01 = __ffma2_rn(C2, x[k][0], R2);
      const f2 u23 = __ffma2_rn(C2, x[k][1], R2);
      x[k][0] = __fmul2_rn(make_float2(t.x, t.y), u01);
      x[k][1] = __fmul2_rn(make_float2(t.z, t.w), u23);
      acc0 = __fadd2_rn(acc0, x[k][0]);
      acc1 = __fadd2_rn(acc1, x[k][1]);
    }
    xs = cur_thx * fmaf(c, xs, r);

    // the warp is done with this block's rows: the last of the CTA's warps refills the slot
    if (j == kRB - 1 || step == p.n_steps - 1) {
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        const int done = atomicAdd(&cnt[blk % kSlots], 1);
        if (done == kWarpTargets - 1) {
          cnt[blk % kSlots] = 0;
          __threadfence_block();
          if (blk + kSlots < nblk) issue(blk + kSlots);
        }
      }
    }

    if (DIR == 0) {
      pend_slot = is_store && p.store ? p.store_slot[store_next] : -1;
      pend_save = save_here;
    }
    if (is_store) {
      ++store_next;
      next_store_l = store_next < p.n_store ? p.store_loci[store_next] : -1;
    }
    if (p.mu_vec && lane < 16 && step + 1 < p.n_steps) {  // next locus' table into the other buffer
      const int e = lane;
      *reinterpret_cast<float4*>(lutw + ((step + 1) & 1) * 64 + 4 * e) =
          make_float4((e & 1) ? nx_thm : nx_thx, (e & 2) ? nx_thm : nx_thx, (e & 4) ? nx_thm : nx_thx,
                      (e & 8) ? nx_thm : nx_thx);
    }

    const float tot = warp_sum((acc0.x + acc0.y) + (acc1.x + acc1.y));
    float sig = tot - n_junk * xs;
    if (DIR == 1) sig *= p.pi_u;
    if (lane == (step & 31)) my_sg = DIR == 0 ? sig : (add_log_prev ? sig_prev : 1.0f);
    if ((step & 31) == 31 || step == p.n_steps - 1) {
      const int cnt_l = (step & 31) + 1;
      const float sg = lane < cnt_l ? my_sg : 1.0f;
      uint32_t stb = 0u;
      if (sg < 1.17549435e-38f) stb |= 1u;
      if (!(sg <= 3.40282347e+38f)) stb |= 2u;
      double v = (double)logf(sg);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      lgs += v;
      sts |= __reduce_or_sync(0xffffffffu, stb);
    }
    if (p.mu_vec) __syncwarp();
    sig_prev = sig;
  }

  if (DIR == 0 && (pend_slot >= 0 || pend_save))
    store_regs(false, 0.f, 0.f, pend_slot >= 0 ? p.store + (size_t)pend_slot * p.state_rows * N : nullptr, nullptr,
               pend_save ? p.state : nullptr);
  if (lane == 0 && active) {
    const uint32_t stb = sts | (*flag ? 4u : 0u);
    if (p.logs) p.logs[row] = lgs;
    if (p.status && stb) atomicOr(p.status + row, stb);
    if (*flag && p.err) atomicOr(p.err, 1);
  }
}

}  // namespace lsk
