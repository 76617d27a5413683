// ls_prop.cuh -- propagation kernel of the LS all-vs-all recursions on sm_103a.
//
// One kernel serves both directions, because the rescaled recursions have the same shape:
//   forward  (Eq. fwd1):  x_j <- theta_j (c x_j + r),  x = alpha,  c = (1-rho)/sum_j x_j,  r = rho pi
//   backward (Eq. bck1, carried as t = beta*theta):
//                         x_j <- theta_j (c x_j + r),  x = t,      c = (1-rho)/(pi sum_j x_j), r = rho
// (the backward's beta is the pre-emission value c x + r, which is what the table keeps).
//
// Work decomposition.  A CTA owns TPW consecutive targets o..o+TPW-1 and all N donors.  Lane
// (tl, sl) of warp w holds target tl and a slice of J = 4*KQ donor slots; the CTA's W*32/TPW
// slices partition the donors.  Donor positions are rotated by o (position p <-> donor
// (p + o) mod N) so that every target's own diagonal cell sits at position tl, i.e. slot tl of
// slice 0.  The whole tile (TPW x N floats) stays in registers across loci (Sec. 4.2: each column
// is carried to the target locus before moving on).
//
// Emission.  Per locus the lane turns its donors' bits into "match" bits (XOR with its target's
// allele); a 16-entry shared-memory table maps 4 match bits to 4 emission factors, one 16-byte
// load per 4 cells; every other quad of 4 cells instead takes them from a bit test (predicates,
// the integer pipe), which splits the emission fetch between the shared-memory and integer pipes.
// With the uniform prior theta (1-mu on a match, mu on a mismatch, App. A.3) is b f with
// b = max(1-mu, mu) folded into the affine step and f in {1, min(1-mu, mu)/b}: the table holds f
// and the bit-test quads multiply by the ratio under a predicate.  A cell costs three FP32
// operations (FFMA, FMUL, FADD, mostly as packed f32x2 pairs).
//
// Padding and diagonal.  Slots beyond the slice and the diagonal slot are forced to "mismatch".
// Those junk cells all start at 0 and see the same c, r and theta = mu, so they hold one common
// value xs, which every lane replicates with the same FP32 operations; the exact junk total
// n_junk * xs is subtracted from the reduced sum, and junk cells are never written out.
//
// Staging.  Each locus row is kept in HBM twice back to back (2N bits: bit b = h[b mod N]), so the
// bits of any slice under any rotation are one contiguous run.  TMA bulk copies move blocks of 4
// consecutive rows into a 3-slot shared-memory ring (mbarrier completion, time-bounded waits);
// each lane funnel-shifts its 32-bit words straight out of the staged rows.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace lsk {

constexpr int kSlots = 3;        // TMA ring slots
constexpr int kRB = 4;           // consecutive rows per TMA block
constexpr int kMaxStore = 64;    // store loci per launch
// every kAluMod-th quad of a lane's slice takes theta by a bit test and select instead of the table
// (0: none); half of the quads measured fastest on GB300 (the table loads and the selects then
// share the load between the shared-memory and integer pipes)
#ifndef LS_X_ALUMOD
#define LS_X_ALUMOD 2
#endif
#ifndef LS_X_UNI
#define LS_X_UNI 1
#endif
#ifndef LS_X_NACC
#define LS_X_NACC 4
#endif
#ifndef LS_X_RED4
#define LS_X_RED4 0
#endif
constexpr int kAluMod = LS_X_ALUMOD;
constexpr float kEps = 2.220446049250313e-16f;  // DBL_EPSILON = 2^-52, exact in FP32 (Eq. distmat)
// alpha * beta products for the posterior (Eq. postprob) are formed as alpha * (beta * 2^100): the
// power of two is exact and cancels in the normalisation, and it lifts products that FP32 would
// flush to zero (rho = 0 leaves the copied donor's alpha and beta each far below the row maxima)
// while staying below overflow (alpha <= 1 and beta <= N, so the scaled product is < 2^100 N).
constexpr float kProdScale = 0x1p100f;

struct PropParams {
  const uint32_t* bits2;  // doubled packed rows [L][rw2]: bit b of row l = h[l][b mod N], b < 2N
  int rw2;
  int N, L;
  int dir;                // 0 forward, 1 backward (selects the instantiation on the host)
  int t_begin, t_count;   // targets handled by this launch (absolute ids, or positions in tlist)
  int tab_t0;             // table row r <-> target tab_t0 + r (with tlist: list position tab_t0 + r)
  const int* tlist;       // optional target list (one target per CTA variants): CTA b takes target
                          // tlist[t_begin + b]
  int l_first;            // locus of step 0
  int n_steps;            // steps (loci) processed
  int init;               // 1: step 0 is the initial locus (fwd 0 / bwd L-1), no prior state
  const float* omr;       // [L-1] 1 - rho
  const float* rr;        // [L-1] forward: rho * pi;  backward: rho
  const float* thm;       // [L] 1 - mu (match)
  const float* thx;       // [L] mu (mismatch)
  int mu_vec;             // 1: mu differs between loci (the emission table is rebuilt every locus)
  float pi_u;             // uniform prior 1/(N-1)
  const float* Pi;        // prior matrix [N][N] recipient-major (matrix-prior variants only)
  float* state;           // [state_rows][N] table state (alpha or beta)
  double* logs;           // [state_rows] log F / log G (may be null)
  uint32_t* status;       // [state_rows] status bits (may be null)
  int state_rows;
  int load_state;         // 1: start from the table state
  int save_state;         // 1: write the final state back
  int n_store;
  int store_loci[kMaxStore];  // in processing order
  int store_slot[kMaxStore];  // output slot of each store locus
  float* store;           // [slots][state_rows][N] alpha (fwd) / beta (bwd) at store loci
  float* alpha_dec;       // backward decode: alpha at the same loci, same layout (may be null);
                          // multiplied in place by t = theta beta (times 2^100): decode_kernel
                          // divides by theta and normalises
  // forward statistic passes (ST > 0): w_j = alpha_j E[S | Z = j, h_0..l] for an additive S
  const float* gam;       // [L-1] weight of a recombination at interval m (ST 1)
  const uint8_t* reset;   // [L-1] 1: interval m opens a new group, w restarts from 0 (ST 1)
  float eta;              // weight of a mismatch emission, eta = 1/(1-mu) (ST 2, scalar mu)
  const float* eta_vec;   // [L] per-locus eta (ST 2, mu varying per locus)
  float* wstore;          // [slots][state_rows][N] w at the store loci (ST 1), may be null
  float* wstate;          // [state_rows][N] w carried between launches
  double* stat_out;       // [state_rows] sum w / sum alpha after the last step (ST 2)
  int* err;               // device error word (timeouts), may be null
};

typedef unsigned long long u64;
typedef float2 f2;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// 16-byte shared load from a 32-bit shared address.  Not volatile and no memory clobber, so the
// compiler may schedule it like an arithmetic instruction; callers order it after the barrier that
// publishes the emission table through a data dependency on the address.
__device__ __forceinline__ float4 lds128(uint32_t addr) {
  float4 v;
  asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
  return v;
}
__device__ __forceinline__ uint32_t funnel(uint32_t lo, uint32_t hi, uint32_t s) {
  return __funnelshift_r(lo, hi, s);  // (hi:lo) >> s, s in [0, 31]
}

// ---- mbarrier / TMA bulk copy ----------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of a ring slot, for at most ~2 s.  On timeout the CTA-wide flag is set
// and every later wait returns at once; the kernel then runs to completion on stale data and the
// host reports LS_ERR_DEVICE.  No thread leaves early, so CTA barriers stay consistent.
__device__ __forceinline__ void mbar_wait_bounded(uint64_t* bar, uint32_t parity, volatile int* flag) {
  if (*flag) return;
  if (mbar_test(bar, parity)) return;
  const uint64_t t0 = gtimer_ns();
  while (!mbar_test(bar, parity)) {
    if (*flag) return;
    if (gtimer_ns() - t0 > 2000000000ull) {
      *flag = 1;
      return;
    }
    __nanosleep(64);
  }
}
__device__ __forceinline__ void tma_row(uint32_t* dst, const uint32_t* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_arrive_tx(bar, bytes);
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// 32 bits of the cyclic bit string b -> h[(g + b) mod N] of a packed row (N >= 32, 0 <= g < N).
__device__ __forceinline__ uint32_t cyclic32(const uint32_t* raw, int N, int g) {
  const int w = g >> 5, s = g & 31;
  uint32_t v = funnel(raw[w], raw[w + 1], (uint32_t)s);
  const int n1 = N - g;
  if (n1 < 32) v = (v & ((1u << n1) - 1u)) | (raw[0] << n1);
  return v;
}
// Same for any N >= 1 (bit by bit); used when N < 32.
__device__ __forceinline__ uint32_t cyclic32_slow(const uint32_t* raw, int N, int g) {
  uint32_t v = 0;
  for (int b = 0; b < 32; ++b) {
    int d = (g + b) % N;
    v |= ((raw[d >> 5] >> (d & 31)) & 1u) << b;
  }
  return v;
}



struct SmemLayout {
  int ring_off;  // byte offsets of the regions
  int stg_off;
  int pi_off;    // prior values of each lane's slots (matrix prior only)
  int total;
};

__host__ __device__ inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

template <int TPW, int W, int KQ>
struct PropCfg {
  static constexpr int SPW = 32 / TPW;     // slices per warp
  static constexpr int S = W * SPW;        // slices per CTA
  static constexpr int J = 4 * KQ;         // slots per lane
  static constexpr int NWORD = (J + 31) / 32;
  static constexpr int NCHUNK = (KQ + 7) / 8;  // 8-quad chunks staged through shared memory
  static constexpr int THREADS = W * 32;
  static constexpr int STG_STRIDE = 36;    // floats per thread in the staging chunk (16-B aligned)
  // dynamic shared memory: mbarriers, partial sums, log ring, per-target log scale and status,
  // timeout flag, TMA ring, store/load staging (the emission tables are static shared memory)
  static constexpr int BAR_OFF = 0;
  static constexpr int PART_OFF = ((BAR_OFF + kSlots * 8 + 15) / 16) * 16;  // 16-byte aligned partials
  static constexpr int LOGR_OFF = PART_OFF + 2 * TPW * W * 8;  // two buffers of float2 partials
  static constexpr int LOG_OFF = ((LOGR_OFF + TPW * 32 * 4 + 7) / 8) * 8;
  static constexpr int ST_OFF = LOG_OFF + TPW * 8;
  static constexpr int FLAG_OFF = ST_OFF + TPW * 4;
  static constexpr int RING_OFF = ((FLAG_OFF + 16 + 127) / 128) * 128;
  static constexpr int PI_STRIDE = J + 4;  // floats per thread in the prior region (conflict-free 16-B loads)
  // bfloat16 prior (PIM = 2): halves per thread, rows 8 bytes off a 16-byte multiple (conflict-free
  // 8-byte loads)
  static constexpr int PI16_STRIDE = ((J + 7) / 8) * 8 + 4;
  __host__ __device__ static SmemLayout layout(int rw2, int pim) {
    SmemLayout s;
    s.ring_off = RING_OFF;
    s.stg_off = RING_OFF + round_up(kSlots * kRB * rw2 * 4, 128);
    s.pi_off = s.stg_off + THREADS * STG_STRIDE * 4;
    s.total = s.pi_off + (pim == 1 ? THREADS * PI_STRIDE * 4 : pim == 2 ? THREADS * PI16_STRIDE * 2 : 0);
    return s;
  }
  // a variant serves N when a slice fits the slots and only a slice's last word is partial
  __host__ __device__ static bool serves(int N) {
    const int Jr = (N + S - 1) / S;
    return Jr >= TPW && Jr <= J && (NWORD == 1 || Jr - 1 >= 32 * (NWORD - 1));
  }
};

// Slice geometry: S slices over N rotated positions; slice sigma has len positions starting at
// start; the last mshort slices are one shorter.
__host__ __device__ __forceinline__ void slice_of(int sigma, int S, int N, int& start, int& len) {
  const int Jr = (N + S - 1) / S;
  const int mshort = S * Jr - N;
  len = Jr - (sigma >= S - mshort ? 1 : 0);
  start = sigma * Jr - (sigma > S - mshort ? sigma - (S - mshort) : 0);
}

// PIM = 1: prior matrix.  Each lane keeps its slots' prior values pi_j (zero on padding and on
// the diagonal) in shared memory; the forward adds rho * pi_j per cell and the backward sums
// t_j pi_j, so no junk correction is needed.  PIM = 2: the same with the values held as bfloat16
// (the BF16 prior format, whose values are bfloat16 already, so the conversion is exact): half the
// shared-memory bytes per cell, two integer operations per pair of cells to widen them.
//
// ST > 0 (forward, uniform prior): a second register tile w carries w_j = alpha_j tau_j, tau_j the
// filtered expectation of an additive statistic S given copying state j.  With S_{l+1} = S_l +
// gamma_l B_l + eta H_{l+1}(Z_{l+1}) (B_l the recombination event of interval l, H the mismatch
// indicator) the recursion is the forward one plus a source:
//   w_j <- theta_j (c w_j + r (W/s + gamma)) + eta H_j x_j,   W = sum_j w_j, s = sum_j x_j.
// ST 1 takes the recombination term (restarted at every group of intervals), ST 2 the mismatch term.
template <int DIR, int TPW, int W, int KQ, int PIM, int ST>
__global__ void __launch_bounds__(W * 32, ((PIM || ST) && W >= 8) ? 1 : 2) ls_prop_kernel(const PropParams p) {
  static_assert(ST == 0 || (DIR == 0 && PIM == 0), "statistic passes run forward with the uniform prior");
  // UNI (uniform prior, no statistic): theta = base * f with base = max(1-mu, mu) and f in {1, ratio},
  // ratio = min(1-mu, mu) / base; a cell is c' x + r' (c' = c base, r' = r base), then multiplied by
  // ratio where f = ratio -- a predicated multiply on the bit-select quads, f from the table on the
  // others.  "small" bits (f = ratio) are the mismatches (or the matches when mu > 1/2).
  constexpr bool UNI = LS_X_UNI && PIM == 0 && ST == 0;
  constexpr int NACC = UNI ? LS_X_NACC : 2;
  using C = PropCfg<TPW, W, KQ>;
  constexpr int SPW = C::SPW, S = C::S, NWORD = C::NWORD, THREADS = C::THREADS;
  constexpr int step_dir = DIR == 0 ? 1 : -1;
  extern __shared__ __align__(128) unsigned char smem[];
  const int N = p.N;
  const int rw2 = p.rw2;
  const SmemLayout lay = C::layout(rw2, PIM);
  float* part = reinterpret_cast<float*>(smem + C::PART_OFF);
  float* lgr = reinterpret_cast<float*>(smem + C::LOGR_OFF);
  double* lgs = reinterpret_cast<double*>(smem + C::LOG_OFF);
  uint32_t* sts = reinterpret_cast<uint32_t*>(smem + C::ST_OFF);
  volatile int* flag = reinterpret_cast<volatile int*>(smem + C::FLAG_OFF);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::BAR_OFF);
  // emission tables: two 256-byte buffers (this step's and the next one's when mu varies per locus),
  // indexed by 16 x (4 match bits); static so the table's address folds into the load offset
  __shared__ __align__(256) float s_lut[2][64];
  float* lutf = &s_lut[0][0];
  const uint32_t lut_base = smem_u32(&s_lut[0][0]);
  // ST 2: eta H for the same 16 x 4 entries (0 on a match, eta on a mismatch)
  __shared__ __align__(256) float s_hlut[ST == 2 ? 2 : 1][ST == 2 ? 64 : 4];
  const uint32_t hlut_base = smem_u32(&s_hlut[0][0]);
  uint32_t* ring = reinterpret_cast<uint32_t*>(smem + lay.ring_off);
  float* stg = reinterpret_cast<float*>(smem + lay.stg_off);

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tl = lane % TPW;
  const int sl = lane / TPW;
  const int cta_t = p.t_begin + blockIdx.x * TPW;      // first target (or list position) of the CTA
  const int o = p.tlist ? p.tlist[cta_t] : cta_t;       // first target of this CTA (< N)
  const int row0 = cta_t - p.tab_t0;                   // table row of target o
  const int t_end = p.t_begin + p.t_count;
  int start, len;
  slice_of(warp * SPW + sl, S, N, start, len);
  const int b0 = start + o;                     // first bit of this lane's slice in a doubled row
  const int wb = b0 >> 5;
  const uint32_t wsh = (uint32_t)(b0 & 31);
  const int abit = o + tl;                      // bit of the target itself
  const float n_junk = PIM ? 0.0f : (float)(S * C::J - (N - 1));
  const uint32_t dclear = (warp == 0 && sl == 0) ? ~(1u << tl) : 0xffffffffu;  // diagonal = slot tl of slice 0
  const int vl = len - 32 * (NWORD - 1);        // valid slots of the last word
  const uint32_t vmask_last = vl >= 32 ? 0xffffffffu : (vl <= 0 ? 0u : ((1u << vl) - 1u));

  // ---- staged transfers between the register tile and global memory (store loci only) ------
  // element (src thread, slot s of chunk c) <-> donor (start_src + 32c + s + o) mod N of target
  // o + tl_src; consecutive threads take consecutive slots, so global accesses are contiguous.
  // to global: w1 = v, m1 *= v, w2 = v (any may be null); from global: gbase into the staging chunk.
  // The backward of the tiles with up to 255 registers a thread takes a thread's elements in batches
  // of kXB and issues a batch's loads before its stores (the compiler cannot tell the stores from
  // later loads, so the read-modify-write of the decode products would otherwise wait one memory
  // latency per element); the forward, which only reads when it resumes from a table, and the
  // 8-warp tiles (128 registers) keep one element at a time (measured faster, and no spills).
  auto xfer = [&](int c, float* gbase, float* w1, float* m1, float* w2, bool to_global) {
    if constexpr (DIR == 0 || W >= 8) {
      for (int idx = tid; idx < THREADS * 32; idx += THREADS) {
        const int src = idx >> 5, s = idx & 31;
        const int ln = src & 31;
        const int t_s = ln % TPW, sg = (src >> 5) * SPW + ln / TPW;
        int st, ln_s;
        slice_of(sg, S, N, st, ln_s);
        const int gs = 32 * c + s;
        float* sp = stg + src * C::STG_STRIDE + s;
        const bool diag = sg == 0 && gs == t_s;
        const bool ok = gs < ln_s && cta_t + t_s < t_end;
        int d = st + gs + o;
        d = d >= N ? d - N : d;
        d = d >= N ? d - N : d;
        const size_t ro = (size_t)(row0 + t_s) * N + d;
        if (to_global) {
          if (ok) {
            const float v = diag ? 0.0f : *sp;
            if (w1) w1[ro] = v;
            if (m1) m1[ro] = diag ? 0.0f : m1[ro] * (v * kProdScale);
            if (w2) w2[ro] = v;
          }
        } else {
          *sp = (ok && !diag) ? gbase[ro] : 0.0f;
        }
      }
      return;
    }
    constexpr int kXB = 8;
    for (int i0 = tid; i0 < THREADS * 32; i0 += THREADS * kXB) {
      size_t ro[kXB];
      bool ok[kXB], dg[kXB];
      float gv[kXB];
#pragma unroll
      for (int b = 0; b < kXB; ++b) {
        const int idx = i0 + b * THREADS;
        const int src = idx >> 5, s = idx & 31;
        const int ln = src & 31;
        const int t_s = ln % TPW, sg = (src >> 5) * SPW + ln / TPW;
        int st, ln_s;
        slice_of(sg, S, N, st, ln_s);
        const int gs = 32 * c + s;
        dg[b] = sg == 0 && gs == t_s;
        ok[b] = gs < ln_s && cta_t + t_s < t_end;
        int d = st + gs + o;
        d = d >= N ? d - N : d;
        d = d >= N ? d - N : d;
        ro[b] = (size_t)(row0 + t_s) * N + d;
      }
#pragma unroll
      for (int b = 0; b < kXB; ++b) {
        gv[b] = 0.0f;
        if (ok[b] && !dg[b]) {
          if (!to_global) gv[b] = gbase[ro[b]];
          else if (m1) gv[b] = m1[ro[b]];
        }
      }
#pragma unroll
      for (int b = 0; b < kXB; ++b) {
        const int idx = i0 + b * THREADS;
        float* sp = stg + (idx >> 5) * C::STG_STRIDE + (idx & 31);
        if (to_global) {
          if (ok[b]) {
            const float v = dg[b] ? 0.0f : *sp;
            if (w1) w1[ro[b]] = v;
            if (m1) m1[ro[b]] = dg[b] ? 0.0f : gv[b] * (v * kProdScale);
            if (w2) w2[ro[b]] = v;
          }
        } else {
          *sp = gv[b];
        }
      }
    }
  };

  // ---- TMA blocks of kRB consecutive rows ------------------------------------------------------
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
    for (int s = 0; s < kSlots; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // emission table of step 0 (for scalar mu it serves every step)
  if (tid < 64) {
    const int e = tid >> 2, k = tid & 3;
    if (UNI) {
      const float a = p.thm[p.l_first], b = p.thx[p.l_first];
      const float bs = fmaxf(a, b);
      lutf[tid] = ((e >> k) & 1) ? 1.0f : (bs > 0.0f ? __fdiv_rn(fminf(a, b), bs) : 0.0f);
    } else {
      lutf[tid] = ((e >> k) & 1) ? p.thm[p.l_first] : p.thx[p.l_first];
    }
    if (ST == 2) s_hlut[0][tid] = ((e >> k) & 1) ? 0.0f : (p.eta_vec ? p.eta_vec[p.l_first] : p.eta);
  }
  if (tid < TPW) {
    lgs[tid] = (cta_t + tid < t_end && p.logs && !p.init) ? p.logs[row0 + tid] : 0.0;
    sts[tid] = 0u;
  }
  __syncthreads();
  if (tid == 0)
    for (int B = 0; B < kSlots && B < nblk; ++B) issue(B);

  // ---- the register tile ------------------------------------------------------------------
  f2 x[KQ][2];
  f2 wv[ST ? KQ : 1][2];  // statistic tile (ST > 0)
#pragma unroll
  for (int k = 0; k < KQ; ++k) x[k][0] = x[k][1] = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < (ST ? KQ : 1); ++k) wv[k][0] = wv[k][1] = make_float2(0.f, 0.f);
  auto load_tile = [&](f2 (&v)[ST ? KQ : 1][2], f2 (&u)[KQ][2], bool into_w, const float* src) {
#pragma unroll
    for (int c = 0; c < C::NCHUNK; ++c) {
      xfer(c, const_cast<float*>(src), nullptr, nullptr, nullptr, false);
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = 8 * c + q;
        if (k < KQ) {
          const float4 t4 = *reinterpret_cast<const float4*>(stg + tid * C::STG_STRIDE + 4 * q);
          if (into_w) {
            if (ST) {
              v[ST ? k : 0][0] = make_float2(t4.x, t4.y);
              v[ST ? k : 0][1] = make_float2(t4.z, t4.w);
            }
          } else {
            u[k][0] = make_float2(t4.x, t4.y);
            u[k][1] = make_float2(t4.z, t4.w);
          }
        }
      }
      __syncthreads();
    }
  };
  if (p.load_state) {
    load_tile(wv, x, false, p.state);
    if (ST) load_tile(wv, x, true, p.wstate);
  }
  // prior values of this lane's slots (matrix prior): slot s <-> donor (start + s + o) mod N
  const float* pis = reinterpret_cast<const float*>(smem + lay.pi_off) + tid * C::PI_STRIDE;
  const uint16_t* pis16 = reinterpret_cast<const uint16_t*>(smem + lay.pi_off) + tid * C::PI16_STRIDE;
  if (PIM) {
    float* my = reinterpret_cast<float*>(smem + lay.pi_off) + tid * C::PI_STRIDE;
    uint16_t* my16 = reinterpret_cast<uint16_t*>(smem + lay.pi_off) + tid * C::PI16_STRIDE;
    int tgt = o + tl;
    tgt = tgt >= N ? tgt - N : tgt;
    const float* prow = p.Pi + (size_t)tgt * N;
    for (int s2 = 0; s2 < C::J; ++s2) {
      int d = start + s2 + o;
      d = d >= N ? d - N : d;
      d = d >= N ? d - N : d;
      const float v = (s2 < len && d != tgt) ? prow[d] : 0.0f;
      if (PIM == 2) my16[s2] = (uint16_t)(__float_as_uint(v) >> 16);  // bfloat16 already: exact
      else my[s2] = v;
    }
    __syncthreads();
  }

  // store the tile (mode 0: x; 1: c x + r; 2: multiply the destination by c x + r)
  // stage (affine ? c x + r : x) chunk by chunk and write it to w1 / multiply m1 by it / write w2
  auto store_tile = [&](float* w1, float* m1, float* w2, bool affine, float c, float r, bool from_w = false) {
    const f2 C2 = make_float2(c, c), R2 = make_float2(r, r);
#pragma unroll
    for (int cc = 0; cc < C::NCHUNK; ++cc) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = 8 * cc + q;
        if (k < KQ) {
          const f2 xa = (ST && from_w) ? wv[ST ? k : 0][0] : x[k][0];
          const f2 xb = (ST && from_w) ? wv[ST ? k : 0][1] : x[k][1];
          const f2 a = affine ? __ffma2_rn(C2, xa, R2) : xa;
          const f2 b = affine ? __ffma2_rn(C2, xb, R2) : xb;
          *reinterpret_cast<float4*>(stg + tid * C::STG_STRIDE + 4 * q) = make_float4(a.x, a.y, b.x, b.y);
        }
      }
      __syncthreads();
      xfer(cc, nullptr, w1, m1, w2, true);
      __syncthreads();
    }
  };

  float sig_prev = 1.0f;  // previous normaliser (fwd: sum alpha; bwd: S)
  float xs = 0.0f;        // common value of the junk cells

  // reduce one value (or, with ST, a pair) per lane over the layout; CTA totals for target tl
  auto reduce2 = [&](float v, float u, float* buf, float& tu) -> float {
#pragma unroll
    for (int off = TPW; off < 32; off <<= 1) {
      v += __shfl_xor_sync(0xffffffffu, v, off);
      if (ST) u += __shfl_xor_sync(0xffffffffu, u, off);
    }
    if (LS_X_RED4 && !ST && W == 4) {  // the W partials of target tl in one 16-byte load
      if (sl == 0) buf[tl * W + warp] = v;
      __syncthreads();
      const float4 e = *reinterpret_cast<const float4*>(buf + tl * W);
      tu = 0.0f;
      return (e.x + e.y) + (e.z + e.w);
    }
    float2* b2 = reinterpret_cast<float2*>(buf);
    if (sl == 0) b2[tl * W + warp] = make_float2(v, u);
    __syncthreads();
    float t = 0.0f;
    tu = 0.0f;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const float2 e = b2[tl * W + w];
      t += e.x;
      tu += e.y;
    }
    return t;
  };
  auto reduce = [&](float v, float* buf) -> float {
    float dummy;
    return reduce2(v, 0.0f, buf, dummy);
  };
  // fold the log ring into the FP64 log scales and check the normalisers (entries 0..cnt-1).  The
  // ring of target t is written and folded by warp t % W, so the warps share the work and no CTA
  // barrier is needed; the 32 logs are summed in FP32 with an exact error term per addition
  // (two-sum), and one FP64 addition per target takes the compensated sum into the log scale.
  auto flush_logs = [&](int cnt) {
    __syncwarp();
#pragma unroll
    for (int k = 0; k < (TPW + W - 1) / W; ++k) {
      const int t = warp + k * W;
      if (t >= TPW) break;
      const float sg = lane < cnt ? lgr[t * 32 + lane] : 1.0f;
      uint32_t stb = 0u;
      if (sg < 1.17549435e-38f) stb |= 1u;      // LS_STATUS_UNDERFLOW: zero or subnormal normaliser
      if (!(sg <= 3.40282347e+38f)) stb |= 2u;  // LS_STATUS_OVERFLOW: infinite or NaN normaliser
      float v = logf(sg), e = 0.0f;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float vo = __shfl_xor_sync(0xffffffffu, v, off);
        const float eo = __shfl_xor_sync(0xffffffffu, e, off);
        const float s2 = __fadd_rn(v, vo);
        const float bb = __fsub_rn(s2, v);
        const float er = __fadd_rn(__fsub_rn(v, __fsub_rn(s2, bb)), __fsub_rn(vo, bb));  // v + vo - s2, exactly
        v = s2;
        e = __fadd_rn(__fadd_rn(e, eo), er);
      }
      const uint32_t any = __reduce_or_sync(0xffffffffu, stb);
      if (lane == 0) {
        lgs[t] += (double)v + (double)e;
        sts[t] |= any;
      }
    }
    __syncwarp();
  };

  float wsum_prev = 0.0f;  // ST: sum of w over the real donors
  float ws = 0.0f;        // ST: common value of w in the junk cells
  if (p.load_state && DIR == 0) {
    float s = 0.0f, sw = 0.0f;
#pragma unroll
    for (int k = 0; k < KQ; ++k) s += (x[k][0].x + x[k][0].y) + (x[k][1].x + x[k][1].y);
    if (ST) {
#pragma unroll
      for (int k = 0; k < (ST ? KQ : 1); ++k) sw += (wv[k][0].x + wv[k][0].y) + (wv[k][1].x + wv[k][1].y);
    }
    sig_prev = reduce2(s, sw, part + 2 * TPW * W, wsum_prev);
    __syncthreads();
  }

  // per-step scalars, loaded one step ahead
  float nx_omr = 0.f, nx_rr = 0.f, nx_thx = p.thx[p.l_first], nx_thm = p.thm[p.l_first];
  {
    const int li = DIR == 0 ? p.l_first - 1 : p.l_first;
    if (li >= 0 && li < p.L - 1) {
      nx_omr = p.omr[li];
      nx_rr = p.rr[li];
    }
  }
  // UNI: base and ratio of the emission values (recomputed per locus only with a per-locus mu)
  float u_base = fmaxf(nx_thm, nx_thx);
  float u_ratio = u_base > 0.0f ? __fdiv_rn(fminf(nx_thm, nx_thx), u_base) : 0.0f;
  int store_next = 0;
  int next_store_l = p.n_store > 0 ? p.store_loci[0] : -1;  // next locus with a store (-1: none)
  int pend_slot = -1;     // forward: store slot of the previous locus' alpha, written next step
  bool pend_save = false; // forward: save the state after the last step
  const uint32_t* slot_rows = ring;
  int blk_base = 0, blk_n = 0;
  // The steps that open a TMA ring block get their own copy of the step body, except in the
  // backward of the widest one-target-per-CTA tiles, where a third copy of the body spilled
  // registers.
  constexpr bool kRingCopy = !(TPW == 1 && DIR == 1 && KQ >= 32);
  // One locus.  EV (a compile-time flag) marks the steps with an event: the first step, every 32nd
  // (the log scales are folded) and the last, a store locus, the step after it (whose top writes the
  // previous locus' alpha or decode product) and the last step when the state is saved.  The other
  // steps run a copy of the body without those branches, whose register allocation the rare work
  // then does not constrain.
  auto body = [&](const int step, auto evc, auto muvc) {
    // per-locus mu: 0 no, 1 yes (compile-time), 2 decided at run time (the FP32 prior-matrix
    // variants, whose larger body spilled when compiled twice)
    constexpr int MUVK = decltype(muvc)::value;
    const bool MUV = MUVK == 2 ? p.mu_vec != 0 : MUVK == 1;
    constexpr int KIND = decltype(evc)::value;  // 0 plain, 1 plain opening a ring block, 2 event
    constexpr bool EV = KIND == 2;
    constexpr bool RING = KIND >= 1 || !kRingCopy;  // plain steps never open a ring block
    const int l = p.l_first + step_dir * step;
    const float cur_omr = nx_omr, cur_rr = nx_rr, cur_thx = nx_thx, cur_thm = nx_thm;
    // (a plain step is never the last; the forward measured faster without the test there)
    if ((DIR == 0 && !EV) || step + 1 < p.n_steps) {
      const int ln = l + step_dir;
      const int li = DIR == 0 ? ln - 1 : ln;
      nx_omr = p.omr[li];
      nx_rr = p.rr[li];
      if (!UNI || MUV) {  // the emission values change between loci only with a per-locus mu
        nx_thx = p.thx[ln];
        nx_thm = p.thm[ln];
      }
    }
    const int j = step & (kRB - 1);
    if (RING && j == 0) {
      const int B = step / kRB;
      if (tid == 0 && B >= 1 && B + kSlots - 1 < nblk) issue(B + kSlots - 1);  // slot of block B-1 is free
      mbar_wait_bounded(&bars[B % kSlots], (uint32_t)((B / kSlots) & 1), flag);
      slot_rows = ring + (B % kSlots) * kRB * rw2;
      blk_rows(B, blk_base, blk_n);
    }
    const uint32_t* rw = slot_rows + (l - blk_base) * rw2;

    float c, r;
    float cw = 0.0f, rws = 0.0f;  // ST: coefficients of the w recursion
    bool add_log_prev = false;
    if (EV && step == 0 && p.init) {
      c = 0.0f;
      r = (DIR == 0 && !PIM) ? p.pi_u : 1.0f;  // alpha^0 = theta pi ; beta^{L-1} = 1
    } else if (EV && step == 0 && DIR == 1) {
      c = 1.0f;  // backward resume: x = theta^l beta^l from the stored beta
      r = 0.0f;
    } else {
      c = __fdividef(cur_omr, sig_prev);  // interval l-1 (fwd) or l (bwd); 2-ulp reciprocal-multiply
      r = cur_rr;
      add_log_prev = DIR == 1;
      if (ST) {
        const float wbar = __fdividef(wsum_prev, sig_prev);  // W / s = E[S_l | h_0..l]
        if (ST == 1) {
          const bool rs = p.reset[l - 1] != 0;
          cw = rs ? 0.0f : c;
          rws = r * ((rs ? 0.0f : wbar) + p.gam[l - 1]);
        } else {
          cw = c;
          rws = r * wbar;
        }
      }
    }
    const bool is_store = EV && l == next_store_l;
    const bool save_here = EV && p.save_state && step == p.n_steps - 1;
    if (EV && DIR == 0 && pend_slot >= 0) {  // alpha of the previous locus
      store_tile(p.store + (size_t)pend_slot * p.state_rows * N, nullptr, nullptr, false, 0.f, 0.f);
      if (ST && p.wstore)
        store_tile(p.wstore + (size_t)pend_slot * p.state_rows * N, nullptr, nullptr, false, 0.f, 0.f, true);
      pend_slot = -1;
    }

    if (EV && DIR == 1 && pend_slot >= 0) {  // decode product of the previous locus: alpha^l t^l, t = theta beta
      store_tile(nullptr, p.alpha_dec + (size_t)pend_slot * p.state_rows * N, nullptr, false, 0.f, 0.f);
      pend_slot = -1;
    }
    if (EV && DIR == 1 && ((is_store && p.store) || save_here)) {
      // beta^l = c t^{l+1} + rho, the pre-emission value (tables and stored rows)
      const size_t so = (size_t)(is_store ? p.store_slot[store_next] : 0) * p.state_rows * N;
      store_tile((is_store && p.store) ? p.store + so : nullptr, nullptr, save_here ? p.state : nullptr, true, c, r);
    }

    // ---- the hot loop: FFMA2 + FMUL2 + FADD2 per pair of cells -------------------------------
    uint32_t inv = ((rw[abit >> 5] >> (abit & 31)) & 1u) ? 0u : 0xffffffffu;  // target allele
    // UNI: base, ratio and the sense of the "small" bits of this locus
    if (UNI && MUV) {
      u_base = fmaxf(cur_thm, cur_thx);
      u_ratio = u_base > 0.0f ? __fdiv_rn(fminf(cur_thm, cur_thx), u_base) : 0.0f;
    }
    if (UNI && cur_thm < cur_thx) inv = ~inv;  // mu > 1/2: the matches carry the smaller factor
    // shared address of this step's table (256-byte aligned, so a byte permute can put a nibble
    // offset in its low byte and the load needs no further address arithmetic)
    uint32_t lut_b = lut_base + (MUV ? (uint32_t)((step & 1) << 8) : 0u);
    // the loads below are plain asm that the compiler may move; deriving their address from a
    // volatile move here keeps them after the previous locus' barrier (which publishes the table)
    asm volatile("mov.b32 %0, %0;" : "+r"(lut_b));
    const float cu = UNI ? c * u_base : c, ru = UNI ? r * u_base : r;
    const f2 C2 = make_float2(cu, cu), R2 = make_float2(ru, ru);
    const f2 CW2 = make_float2(cw, cw), RW2 = make_float2(rws, rws);
    f2 acc[NACC];
#pragma unroll
    for (int a = 0; a < NACC; ++a) acc[a] = make_float2(0.f, 0.f);
    f2 accw0 = make_float2(0.f, 0.f), accw1 = make_float2(0.f, 0.f);
    // Software pipeline: the emission-table entries are loaded kLA quads ahead of their use from a
    // rotating register buffer; a slice word's nibbles are prepared when the lookahead enters it.
    constexpr int kLA = KQ < 4 ? KQ : 4;
    uint32_t hw[2], lw[2];   // 16 x nibble bytes of the words feeding the lookahead (double-buffered)
    uint32_t mw[2];          // the match words themselves (bit-select quads)
    float4 th[kLA];
    auto prep_word = [&](int m) {
      uint32_t w = funnel(rw[wb + m], rw[wb + m + 1], wsh) ^ inv;  // match bits of 32 slots
      if (m == NWORD - 1) w &= vmask_last;
      if (m == 0) w &= dclear;
      hw[m & 1] = w & 0xf0f0f0f0u;         // 16 x odd nibbles, one per byte
      lw[m & 1] = (w << 4) & 0xf0f0f0f0u;  // 16 x even nibbles
      mw[m & 1] = w;
    };
    // bit-select quads: theta from a bit test and a select instead of a table load (the statistic
    // passes' eta H table is still read through the nibble bytes, which every quad keeps)
    auto sel_quad = [&](int k) -> bool { return kAluMod > 0 && (k % (kAluMod > 0 ? kAluMod : 1)) == kAluMod - 1; };
    auto sel_th = [&](int k) -> float4 {
      const uint32_t w = mw[(k >> 3) & 1];
      const int b = 4 * (k & 7);
      return make_float4((w >> b) & 1u ? cur_thm : cur_thx, (w >> (b + 1)) & 1u ? cur_thm : cur_thx,
                         (w >> (b + 2)) & 1u ? cur_thm : cur_thx, (w >> (b + 3)) & 1u ? cur_thm : cur_thx);
    };
    auto load_th = [&](int kk) -> float4 {
      const int q = kk & 7, m = kk >> 3;
      // PRMT: byte q/2 of the nibble word as the low byte, the table's buffer offset above it
      const uint32_t a = __byte_perm((q & 1) ? hw[m & 1] : lw[m & 1], lut_b, 0x7650u | (uint32_t)(q >> 1));
      return lds128(a);
    };
    prep_word(0);
#pragma unroll
    for (int k = 0; k < kLA; ++k)
      if (!sel_quad(k)) th[k] = load_th(k);
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
      const float4 t = sel_quad(k) ? sel_th(k) : th[k % kLA];
      const int kn = k + kLA;
      if (kn < KQ) {
        if ((kn & 7) == 0) prep_word(kn >> 3);
        if (!sel_quad(kn)) th[k % kLA] = load_th(kn);
      }
      if (PIM) {
        f2 p01, p23;
        if (PIM == 2) {
          const uint2 pb = *reinterpret_cast<const uint2*>(pis16 + 4 * k);
          p01 = make_float2(__uint_as_float(pb.x << 16), __uint_as_float(pb.x & 0xffff0000u));
          p23 = make_float2(__uint_as_float(pb.y << 16), __uint_as_float(pb.y & 0xffff0000u));
        } else {
          const float4 pv = *reinterpret_cast<const float4*>(pis + 4 * k);
          p01 = make_float2(pv.x, pv.y);
          p23 = make_float2(pv.z, pv.w);
        }
        if (DIR == 0) {  // u = c x + rho pi_j
          const f2 u01 = __ffma2_rn(C2, x[k][0], __fmul2_rn(R2, p01));
          const f2 u23 = __ffma2_rn(C2, x[k][1], __fmul2_rn(R2, p23));
          x[k][0] = __fmul2_rn(make_float2(t.x, t.y), u01);
          x[k][1] = __fmul2_rn(make_float2(t.z, t.w), u23);
          acc[0] = __fadd2_rn(acc[0], x[k][0]);
          acc[1] = __fadd2_rn(acc[1], x[k][1]);
        } else {         // S = sum_j t_j pi_j
          const f2 u01 = __ffma2_rn(C2, x[k][0], R2);
          const f2 u23 = __ffma2_rn(C2, x[k][1], R2);
          x[k][0] = __fmul2_rn(make_float2(t.x, t.y), u01);
          x[k][1] = __fmul2_rn(make_float2(t.z, t.w), u23);
          acc[0] = __ffma2_rn(x[k][0], p01, acc[0]);
          acc[1] = __ffma2_rn(x[k][1], p23, acc[1]);
        }
      } else if (UNI) {
        const f2 u01 = __ffma2_rn(C2, x[k][0], R2);
        const f2 u23 = __ffma2_rn(C2, x[k][1], R2);
        if (sel_quad(k)) {  // multiply the "small" cells by ratio (predicated, no select)
          const uint32_t w = mw[(k >> 3) & 1];
          const int b = 4 * (k & 7);
          float a0 = u01.x, a1 = u01.y, a2 = u23.x, a3 = u23.y;
          if (!((w >> b) & 1u)) a0 = __fmul_rn(a0, u_ratio);
          if (!((w >> (b + 1)) & 1u)) a1 = __fmul_rn(a1, u_ratio);
          if (!((w >> (b + 2)) & 1u)) a2 = __fmul_rn(a2, u_ratio);
          if (!((w >> (b + 3)) & 1u)) a3 = __fmul_rn(a3, u_ratio);
          x[k][0] = make_float2(a0, a1);
          x[k][1] = make_float2(a2, a3);
        } else {
          x[k][0] = __fmul2_rn(make_float2(t.x, t.y), u01);
          x[k][1] = __fmul2_rn(make_float2(t.z, t.w), u23);
        }
        acc[(2 * k) % NACC] = __fadd2_rn(acc[(2 * k) % NACC], x[k][0]);
        acc[(2 * k + 1) % NACC] = __fadd2_rn(acc[(2 * k + 1) % NACC], x[k][1]);
      } else {
        const f2 u01 = __ffma2_rn(C2, x[k][0], R2);
        const f2 u23 = __ffma2_rn(C2, x[k][1], R2);
        x[k][0] = __fmul2_rn(make_float2(t.x, t.y), u01);
        x[k][1] = __fmul2_rn(make_float2(t.z, t.w), u23);
        acc[0] = __fadd2_rn(acc[0], x[k][0]);
        acc[1] = __fadd2_rn(acc[1], x[k][1]);
        if (ST) {
          const int kw = ST ? k : 0;
          const f2 v01 = __fmul2_rn(make_float2(t.x, t.y), __ffma2_rn(CW2, wv[kw][0], RW2));
          const f2 v23 = __fmul2_rn(make_float2(t.z, t.w), __ffma2_rn(CW2, wv[kw][1], RW2));
          if (ST == 2) {  // + eta H x (the emission term of the mismatch statistic)
            const int q = k & 7, m = k >> 3;
            const uint32_t a = __byte_perm((q & 1) ? hw[m & 1] : lw[m & 1], lut_b, 0x7650u | (uint32_t)(q >> 1));
            const float4 hv = lds128(a - lut_base + hlut_base);
            wv[kw][0] = __ffma2_rn(make_float2(hv.x, hv.y), x[k][0], v01);
            wv[kw][1] = __ffma2_rn(make_float2(hv.z, hv.w), x[k][1], v23);
          } else {
            wv[kw][0] = v01;
            wv[kw][1] = v23;
          }
          accw0 = __fadd2_rn(accw0, wv[kw][0]);
          accw1 = __fadd2_rn(accw1, wv[kw][1]);
        }
      }
    }
    // junk cells: theta = mu in every lane (UNI: always the "small" factor, as their bits are 0)
    xs = UNI ? __fmul_rn(u_ratio, __fmaf_rn(cu, xs, ru)) : cur_thx * fmaf(c, xs, r);
    if (ST) {  // the same operations as a mismatch cell
      const float v = __fmul_rn(cur_thx, __fmaf_rn(cw, ws, rws));
      ws = ST == 2 ? __fmaf_rn(p.eta_vec ? p.eta_vec[l] : p.eta, xs, v) : v;
    }

    if (DIR == 0) {  // alpha^l is stored at the top of the next step (or after the loop)
      pend_slot = is_store && p.store ? p.store_slot[store_next] : -1;
      pend_save = save_here;
    } else {  // decoding: alpha^l is multiplied by t^l = theta^l beta^l at the top of the next step; the
              // decode kernel divides the product by theta^l (it reads the locus' alleles)
      pend_slot = is_store && p.alpha_dec ? p.store_slot[store_next] : -1;
    }
    if (is_store) {
      ++store_next;
      next_store_l = store_next < p.n_store ? p.store_loci[store_next] : -1;
    }

    // emission table of the next locus (mu varying per locus), into the other buffer
    if (MUV && tid < 64 && step + 1 < p.n_steps) {
      const int e = tid >> 2, k = tid & 3;
      if (UNI) {
        const float bs = fmaxf(nx_thm, nx_thx);
        lutf[((step + 1) & 1) * 64 + tid] = ((e >> k) & 1) ? 1.0f : (bs > 0.0f ? __fdiv_rn(fminf(nx_thm, nx_thx), bs) : 0.0f);
      } else {
        lutf[((step + 1) & 1) * 64 + tid] = ((e >> k) & 1) ? nx_thm : nx_thx;
      }
      if (ST == 2) s_hlut[(step + 1) & 1][tid] = ((e >> k) & 1) ? 0.0f : p.eta_vec[l + 1];
    }

    float wtot = 0.0f;
    // fold the NACC accumulator pairs (a power of two) pairwise, then the last pair
#pragma unroll
    for (int h = NACC / 2; h >= 2; h >>= 1)
#pragma unroll
      for (int a = 0; a < h; ++a) acc[a] = __fadd2_rn(acc[a], acc[a + h]);
    const float lsum = (acc[0].x + acc[0].y) + (acc[1].x + acc[1].y);
    const float tot = reduce2(lsum, (accw0.x + accw0.y) + (accw1.x + accw1.y), part + (step & 1) * 2 * TPW * W, wtot);
    if (ST) wsum_prev = wtot - n_junk * ws;
    float sig = tot - n_junk * xs;
    if (DIR == 1 && !PIM) sig *= p.pi_u;
    if (lane < TPW && lane % W == warp) lgr[lane * 32 + (step & 31)] = DIR == 0 ? sig : (add_log_prev ? sig_prev : 1.0f);
    if (EV && ((step & 31) == 31 || step == p.n_steps - 1)) flush_logs((step & 31) + 1);
    sig_prev = sig;
  };
  // the step loop, with the per-locus mu case as a compile-time flag of the step body
  auto run_steps = [&](auto muvc) {
    for (int step = 0; step < p.n_steps;) {
      // the next event step: the first step, the next fold of the log scales (every 32nd and the last
      // step), now if a store is pending, else the next store locus
      int ev = step == 0 ? 0 : min(step | 31, p.n_steps - 1);
      if (pend_slot >= 0) ev = step;
      else if (next_store_l >= 0) ev = min(ev, (next_store_l - p.l_first) * step_dir);
      // the steps that open a TMA ring block (every kRB-th) run in their own copy
      if (!kRingCopy) {
        for (; step < ev; ++step) body(step, std::integral_constant<int, 0>{}, muvc);
      }
      while (step < ev) {
        if ((step & (kRB - 1)) == 0) body(step++, std::integral_constant<int, 1>{}, muvc);
        const int e2 = min(ev, (step + kRB - 1) & ~(kRB - 1));
        for (; step < e2; ++step) body(step, std::integral_constant<int, 0>{}, muvc);
      }
      if (step < p.n_steps) body(step++, std::integral_constant<int, 2>{}, muvc);
    }
  };
  if (PIM == 1) run_steps(std::integral_constant<int, 2>{});
  else if (p.mu_vec) run_steps(std::integral_constant<int, 1>{});
  else run_steps(std::integral_constant<int, 0>{});

  if (DIR == 1 && pend_slot >= 0)  // decode product of the last locus
    store_tile(nullptr, p.alpha_dec + (size_t)pend_slot * p.state_rows * N, nullptr, false, 0.f, 0.f);
  if (DIR == 0 && (pend_slot >= 0 || pend_save)) {  // alpha of the last locus and the state, one pass
    store_tile(pend_slot >= 0 ? p.store + (size_t)pend_slot * p.state_rows * N : nullptr, nullptr,
               pend_save ? p.state : nullptr, false, 0.f, 0.f);
    if (ST)
      store_tile((pend_slot >= 0 && p.wstore) ? p.wstore + (size_t)pend_slot * p.state_rows * N : nullptr, nullptr,
                 pend_save ? p.wstate : nullptr, false, 0.f, 0.f, true);
  }
  __syncthreads();  // the log scales and status words were last written by other warps
  if (tid < TPW && cta_t + tid < t_end) {
    const int row = row0 + tid;
    const uint32_t stb = sts[tid] | (*flag ? 4u : 0u);  // 4 = LS_STATUS_TIMEOUT
    if (p.logs) p.logs[row] = lgs[tid];
    if (ST && p.stat_out) p.stat_out[row] = (double)wsum_prev / (double)sig_prev;
    if (p.status && stb) atomicOr(p.status + row, stb);
    if (*flag && p.err) atomicOr(p.err, 1);
  }
}

}  // namespace lsk
