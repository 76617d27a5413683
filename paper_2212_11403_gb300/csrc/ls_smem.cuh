// ls_smem.cuh -- dense propagation for large N (uniform prior): one target per CTA, its whole
// N-float state in shared memory.
//
// The register-tile kernels stop near N = 20000 (a target's state must fit the registers of one
// CTA).  Here thread t of 1024 owns donors [4 QT t, 4 QT (t+1)) as QT float4 quads in shared memory
// (up to 4 x 1024 x 14 = 57344 donors in 224 KB).  Per locus a thread reads the packed bits of its
// donors straight from the (L2-resident) packed row, one locus ahead, maps 4 match bits to 4
// emission probabilities through the 16-entry table, updates its quads in place
// (x <- theta (c x + r), FFMA + FMUL + FADD per cell) and adds them up; the row sum is a shuffle
// tree, one CTA barrier and a 32-entry sum.  The target's own cell and the padding beyond N are
// multiplied by 0 (a per-quad mask), so no junk correction is needed.  Shared memory bounds it:
// 12 bytes of shared traffic per cell (state load and store, table load).
#pragma once

#include "ls_prop.cuh"

namespace lsk {

constexpr int kSmemThreads = 1024;

template <int QT>
struct SmemCfg {
  static constexpr int NP = kSmemThreads * 4 * QT;  // padded donor count
  static constexpr int BITS = 4 * QT;                // donors (bits) per thread
  // row words a thread may touch: bits sh .. sh + BITS - 1 (sh < 32), and one more for the funnel
  static constexpr int NW = (4 * QT + 30) / 32 + 2;
  __host__ __device__ static int smem_bytes() { return NP * 4 + 2 * 32 * 4 + 64; }
  // only beyond the register-tile kernels' range (N <= 20480), where nothing else serves
  __host__ __device__ static bool serves(int N) { return N > 20480 && N <= NP; }
};

template <int DIR, int QT>
__global__ void __launch_bounds__(kSmemThreads, 1) ls_smem_kernel(const PropParams p) {
  using C = SmemCfg<QT>;
  constexpr int step_dir = DIR == 0 ? 1 : -1;
  extern __shared__ __align__(16) unsigned char smem[];
  float* X = reinterpret_cast<float*>(smem);                     // [NP] state
  float* part = reinterpret_cast<float*>(smem + C::NP * 4);      // [2][32] warp partials
  __shared__ __align__(256) float s_lut[2][64];
  const int N = p.N, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cta_t = p.t_begin + blockIdx.x;        // one target per CTA (or its target-list position)
  const int tgt = p.tlist ? p.tlist[cta_t] : cta_t;
  const int row = cta_t - p.tab_t0;
  const int d0 = C::BITS * tid;            // first donor of this thread
  // quads' validity: donor < N and not the target itself
  uint32_t qmask[QT];
#pragma unroll
  for (int q = 0; q < QT; ++q) {
    uint32_t m = 0u;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int d = d0 + 4 * q + e;
      if (d < N && d != tgt) m |= 1u << e;
    }
    qmask[q] = m;
  }
  auto mask4 = [&](int q) {
    const uint32_t m = qmask[q];
    return make_float4((m & 1u) ? 1.f : 0.f, (m & 2u) ? 1.f : 0.f, (m & 4u) ? 1.f : 0.f, (m & 8u) ? 1.f : 0.f);
  };
  const uint32_t lut_base = smem_u32(&s_lut[0][0]);
  if (tid < 64) {
    const int e = tid >> 2, k = tid & 3;
    s_lut[0][tid] = ((e >> k) & 1) ? p.thm[p.l_first] : p.thx[p.l_first];
  }
  // state
  for (int i = tid; i < C::NP; i += kSmemThreads) {
    float v = 0.0f;
    if (p.load_state && i < N && i != tgt) v = p.state[(size_t)row * N + i];
    X[i] = v;
  }
  __syncthreads();
  auto reduce = [&](float v, int buf) -> float {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) part[buf * 32 + warp] = v;
    __syncthreads();
    float t = part[buf * 32 + lane];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    return t;
  };
  // the words holding this thread's bits of row l, and the target's own bit
  const int w0 = d0 >> 5, sh = d0 & 31;
  auto load_bits = [&](int l, uint32_t (&wd)[C::NW], uint32_t& tb) {
    const uint32_t* r = p.bits2 + (size_t)l * p.rw2;  // packed rows (first N bits of a doubled row)
#pragma unroll
    for (int k = 0; k < C::NW; ++k) wd[k] = (w0 + k < p.rw2) ? r[w0 + k] : 0u;
    tb = (r[tgt >> 5] >> (tgt & 31)) & 1u;
  };
  auto store_state = [&](float* w1, float* m1, float* w2, bool affine, float c, float r) {
    __syncthreads();
    for (int i = tid; i < N; i += kSmemThreads) {
      const float x = X[i];
      const float v = i == tgt ? 0.0f : (affine ? fmaf(c, x, r) : x);
      const size_t o = (size_t)row * N + i;
      if (w1) w1[o] = v;
      if (m1) m1[o] = i == tgt ? 0.0f : m1[o] * v;
      if (w2) w2[o] = v;
    }
    __syncthreads();
  };

  float sig_prev = 1.0f;
  if (p.load_state && DIR == 0) {
    float s = 0.0f;
    for (int i = tid; i < C::NP; i += kSmemThreads) s += X[i];
    sig_prev = reduce(s, 1);
    __syncthreads();
  }
  double lgs = (p.logs && !p.init) ? p.logs[row] : 0.0;
  uint32_t sts = 0u;
  int store_next = 0;
  int next_store_l = p.n_store > 0 ? p.store_loci[0] : -1;
  int pend_slot = -1;
  bool pend_save = false;
  uint32_t wd[C::NW], tb;
  load_bits(p.l_first, wd, tb);
  for (int step = 0; step < p.n_steps; ++step) {
    const int l = p.l_first + step_dir * step;
    uint32_t cw[C::NW], ctb = tb;
#pragma unroll
    for (int k = 0; k < C::NW; ++k) cw[k] = wd[k];
    if (step + 1 < p.n_steps) load_bits(l + step_dir, wd, tb);  // next locus, in flight during this one
    float c, r;
    bool add_log_prev = false;
    const int mi = DIR == 0 ? l - 1 : l;
    if (step == 0 && p.init) {
      c = 0.0f;
      r = DIR == 0 ? p.pi_u : 1.0f;
    } else if (step == 0 && DIR == 1) {
      c = 1.0f;
      r = 0.0f;
    } else {
      c = __fdividef(p.omr[mi], sig_prev);
      r = p.rr[mi];
      add_log_prev = DIR == 1;
    }
    const bool is_store = l == next_store_l;
    const bool save_here = p.save_state && step == p.n_steps - 1;
    if (DIR == 0 && pend_slot >= 0) {
      store_state(p.store + (size_t)pend_slot * p.state_rows * N, nullptr, nullptr, false, 0.f, 0.f);
      pend_slot = -1;
    }
    if (DIR == 1 && (is_store || save_here)) {
      const size_t so = (size_t)(is_store ? p.store_slot[store_next] : 0) * p.state_rows * N;
      store_state((is_store && p.store) ? p.store + so : nullptr, (is_store && p.alpha_dec) ? p.alpha_dec + so : nullptr,
                  save_here ? p.state : nullptr, true, c, r);
    }
    // emission table of this locus (per-locus mu): rebuilt into the buffer of this step's parity
    uint32_t lb = lut_base + (p.mu_vec ? (uint32_t)((step & 1) << 8) : 0u);
    asm volatile("mov.b32 %0, %0;" : "+r"(lb));  // keeps the table loads after the last barrier
    const uint32_t inv = ctb ? 0u : 0xffffffffu;
    // the thread's bits aligned to bit 0 of aw[0] (static indices below), match bits after the XOR
    uint32_t aw[C::NW - 1];
#pragma unroll
    for (int k = 0; k < C::NW - 1; ++k) aw[k] = funnel(cw[k], cw[k + 1], (uint32_t)sh) ^ inv;
    const f2 C2 = make_float2(c, c), R2 = make_float2(r, r);
    f2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    float4* Xq = reinterpret_cast<float4*>(X) + QT * tid;
#pragma unroll
    for (int q = 0; q < QT; ++q) {
      const uint32_t nib = (aw[(4 * q) >> 5] >> ((4 * q) & 31)) & 15u;
      const float4 t = lds128(lb + 16u * nib);
      const float4 x = Xq[q];
      const f2 u01 = __ffma2_rn(C2, make_float2(x.x, x.y), R2);
      const f2 u23 = __ffma2_rn(C2, make_float2(x.z, x.w), R2);
      f2 y01 = __fmul2_rn(make_float2(t.x, t.y), u01);
      f2 y23 = __fmul2_rn(make_float2(t.z, t.w), u23);
      if (qmask[q] != 15u) {  // the target's own cell or padding
        const float4 m = mask4(q);
        y01 = __fmul2_rn(y01, make_float2(m.x, m.y));
        y23 = __fmul2_rn(y23, make_float2(m.z, m.w));
      }
      Xq[q] = make_float4(y01.x, y01.y, y23.x, y23.y);
      acc0 = __fadd2_rn(acc0, y01);
      acc1 = __fadd2_rn(acc1, y23);
    }
    if (DIR == 0) {
      pend_slot = is_store && p.store ? p.store_slot[store_next] : -1;
      pend_save = save_here;
    }
    if (is_store) {
      ++store_next;
      next_store_l = store_next < p.n_store ? p.store_loci[store_next] : -1;
    }
    if (p.mu_vec && tid < 64 && step + 1 < p.n_steps) {
      const int e = tid >> 2, k = tid & 3, ln = l + step_dir;
      s_lut[(step + 1) & 1][tid] = ((e >> k) & 1) ? p.thm[ln] : p.thx[ln];
    }
    float sig = reduce((acc0.x + acc0.y) + (acc1.x + acc1.y), step & 1);
    if (DIR == 1) sig *= p.pi_u;
    const float sg = DIR == 0 ? sig : (add_log_prev ? sig_prev : 1.0f);
    if (sg < 1.17549435e-38f) sts |= 1u;
    if (!(sg <= 3.40282347e+38f)) sts |= 2u;
    lgs += (double)logf(sg);
    sig_prev = sig;
  }
  if (DIR == 0 && (pend_slot >= 0 || pend_save))
    store_state(pend_slot >= 0 ? p.store + (size_t)pend_slot * p.state_rows * N : nullptr, nullptr,
                pend_save ? p.state : nullptr, false, 0.f, 0.f);
  if (tid == 0 && cta_t < p.t_begin + p.t_count) {
    if (p.logs) p.logs[row] = lgs;
    if (p.status && sts) atomicOr(p.status + row, sts);
  }
}

}  // namespace lsk
