// ls_sparse.cuh -- the LS recursions restricted to proposed donor sets.
//
// For target i and window w (WS consecutive loci) the copying state ranges over a set S_i^w of at
// most K donors (ascending ids, -1 padding at the end).  The prior keeps its dense value
// pi = 1/(N-1): recombination mass that would go to donors outside the set is dropped, so donors
// in the set follow exactly the dense recursions (Eq. fwd1 / Eq. bck1) up to a common factor per
// target and locus.  A transition from locus l (window w) to l+1 (window w') continues only for
// donors in both sets:
//   forward:  alpha'_k = theta_k ((1-rho) a_k [k in S] + rho pi),  a = alpha / sum_{S} alpha,
//   backward: beta_j   = (1-rho) [j in S'] t_j / S + rho,  t = theta beta,  S = pi sum_{k in S'} t_k,
// so the backward is the adjoint of the forward and p ~ alpha beta over S_i^w is the posterior of
// the restricted chain.  The normalised forward mass on donors that leave the set at a window
// change is the in-set check: its maximum per target is reported ("lost"), and targets above a
// tolerance are recomputed densely by the caller.
//
// Outside pool (pool = 1): the donors outside the set are carried as one aggregate state o (their
// total forward mass, or their total t = theta beta backward) with the average emission of the
// outside donors at each locus (from the locus' allele count minus the set's own matches):
//   o <- theta_out (c o) + r sum_{j out} theta_j,   theta_out = sum_{j out} theta_j / |out|,
// and the normalisers become set sum + o, as in the dense chain.  At a window change the mass of
// donors leaving the set joins the pool and each entering donor takes the pool's average.  The
// posterior is the pooled chain's own: its normaliser adds the pool's forward mass times the mean
// backward value of the outside donors, and each outside donor receives an equal share of the
// pool's posterior mass (an estimate, reported apart from the set donors' values).
//
// One warp per target, slot s of lane q <-> set index 32 s + q (coalesced set loads and stores);
// eight targets per CTA share the packed locus rows, staged up to eight rows at a time in shared
// memory together with the rows' per-locus constants, double-buffered: the asynchronous copies
// (cp.async) of the next block run while the current one is processed.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace lsk {

constexpr int kSparseWarps = 8;  // targets per CTA
constexpr int kSparseChunk = 32;  // loci per block: one 32-bit haplotype-major word per donor
constexpr int kSparseScal = 5;    // per-locus constants staged per block: 1-mu, mu, 1-rho, rho, n1

struct SparseParams {
  const uint32_t* hw;    // [ceil(L/256)][N][8] haplotype-major words: bit b of word k of (w, j) is
                         // haplotype j at locus 256 w + 32 k + b (0 beyond L)
  int N, L;
  int K;                 // set entries per target and window
  int WS;                // loci per window
  int Wn;                // windows, ceil(L / WS)
  const int32_t* idx;    // [N][Wn][K] donor ids, ascending, -1 padding at the end
  const float* omr;      // [L-1] 1 - rho
  const float* rho;      // [L-1] rho
  const float* thm;      // [L] 1 - mu
  const float* thx;      // [L] mu
  int t_begin, t_count;
  int n_store;
  int store_loci[64];    // processing order
  int store_slot[64];
  float* store;          // [slots][N][K]: forward writes alpha, backward overwrites it with p
  double* logs;          // [N] forward: log-likelihood of the restricted chain (may be null)
  float* lost;           // [N] forward: max normalised mass on leaving donors (may be null)
  uint32_t* status;      // [N] status bits (may be null)
  const int32_t* n1;     // [L] haplotypes carrying allele 1 at each locus (outside pool only)
  int pool;              // 1: carry the donors outside the set as one pooled state (below)
  float* poolf;          // [slots][N] forward: the pool's mass at the store loci (pool = 1)
  float* share;          // [slots][N] backward: posterior of one outside donor (pool = 1)
  float* pout;           // [slots][N] backward: posterior mass of all outside donors (may be null)
};

// posterior products alpha * (beta * 2^100): exact scaling that cancels in the normalisation and
// keeps products of small alpha and beta above FP32's underflow
constexpr float kSparseProdScale = 0x1p100f;

// two buffers of per-locus constants and the per-warp set copies used at window changes
__host__ __device__ inline int sparse_smem_bytes(int ks) {
  return 2 * kSparseScal * kSparseChunk * 4 + 2 * kSparseWarps * 32 * ks * 4;
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

#ifndef LS_SPARSE_PARAMS_ONLY  // the kernels live in ls_sparse.cu only

template <int DIR, int KS>
__global__ void __launch_bounds__(kSparseWarps * 32) ls_sparse_kernel(const SparseParams p) {
  constexpr float eps = 2.220446049250313e-16f;
  constexpr int INF_ID = 0x7fffffff;
  constexpr int CH = kSparseChunk;
  extern __shared__ __align__(16) unsigned char smem[];
  float* scal = reinterpret_cast<float*>(smem);  // [2][kSparseScal][CH]
  int* sid_all = reinterpret_cast<int*>(scal + 2 * kSparseScal * CH);
  float* sval_all = reinterpret_cast<float*>(sid_all + kSparseWarps * 32 * KS);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i_raw = p.t_begin + blockIdx.x * kSparseWarps + warp;
  const bool active = i_raw < p.t_begin + p.t_count;
  const int i = active ? i_raw : p.t_begin;  // idle warps shadow a valid target and write nothing
  int* sid = sid_all + warp * 32 * KS;
  float* sval = sval_all + warp * 32 * KS;
  const int K = p.K, L = p.L, N = p.N;
  const float pi = 1.0f / (float)(N - 1);  // dense uniform prior

  int id[KS];
  float x[KS];
  // mismatch words of the current block: bit k of mm[s] is 1 where entry s's donor differs from the
  // target at locus 32 b + k.  Padding entries (id -1) get all ones: they are updated like
  // mismatching donors, all start at 0 when their window starts and so hold one common value xs,
  // which the row sum subtracts (no per-entry branch in the locus loop).
  uint32_t mm[KS];
  uint32_t twd = 0u;  // the target's own word of the block
  float xs = 0.0f;
  int cur_w = -1;
  auto warp_sum = [&](float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
  };
  auto set_entry = [&](int w, int s) -> int {
    const int q = 32 * s + lane;
    return q < K ? p.idx[((size_t)i * p.Wn + w) * K + q] : -1;
  };
  // the words of block b (loci 32 b .. 32 b + 31) for the current set
  auto gather = [&](int b) {
    const uint32_t* hwb = p.hw + (size_t)(b >> 3) * N * 8 + (b & 7);
    twd = hwb[(size_t)i * 8];
#pragma unroll
    for (int s = 0; s < KS; ++s) mm[s] = id[s] >= 0 ? (hwb[(size_t)id[s] * 8] ^ twd) : 0xffffffffu;
  };
  // exact sum of the set's values, in the order the window map sums them
  auto set_sum = [&]() -> float {
    float v = 0.0f;
#pragma unroll
    for (int s = 0; s < KS; ++s) v += id[s] >= 0 ? x[s] : 0.0f;
    return warp_sum(v);
  };
  // enter window w: map the values of the old set onto the new one (`fill` for new donors); returns
  // the mapped total, and the number of entering donors and of set entries
  int n_enter = 0, nset = 0;
  auto enter = [&](int w, bool map, float fill) -> float {
    if (map) {
#pragma unroll
      for (int s = 0; s < KS; ++s) {
        sid[32 * s + lane] = id[s] >= 0 ? id[s] : INF_ID;
        sval[32 * s + lane] = x[s];
      }
      __syncwarp();
    }
    float mapped = 0.0f;
    int ne = 0, nv = 0;
#pragma unroll
    for (int s = 0; s < KS; ++s) {
      id[s] = set_entry(w, s);
      float v = 0.0f;
      if (map && id[s] >= 0) {
        int lo = 0, hi = 32 * KS;  // first position with sid >= id
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (sid[mid] < id[s]) lo = mid + 1;
          else hi = mid;
        }
        if (lo < 32 * KS && sid[lo] == id[s]) {
          v = sval[lo];
          mapped += v;
        } else {
          v = fill;
          ++ne;
        }
      }
      nv += id[s] >= 0;
      x[s] = v;
    }
    if (map) __syncwarp();
    cur_w = w;
    xs = 0.0f;  // every padding entry restarts at 0
    n_enter = __reduce_add_sync(0xffffffffu, ne);
    nset = __reduce_add_sync(0xffffffffu, nv);
    return warp_sum(mapped);
  };

  double logacc = 0.0;
  uint32_t stb = 0u;
  float lost_max = 0.0f;
  float sum_prev = 1.0f;  // forward: sum alpha; backward: sum t (set plus pool)
  float opool = 0.0f;     // outside pool (pool = 1)
  int store_next = 0;
  // blocks of CH loci aligned to multiples of CH, in processing order; the per-locus constants of
  // the next block are copied asynchronously (cp.async) while the current one is processed
  const int nb = (L + CH - 1) / CH;
  auto blk_of = [&](int t) { return DIR == 0 ? t : nb - 1 - t; };
  auto issue = [&](int t) {
    const int b = blk_of(t), base = CH * b, nrows = min(CH, L - base);
    const int f = threadIdx.x / CH, k = threadIdx.x % CH, l = base + k;
    if (threadIdx.x < kSparseScal * CH && k < nrows) {
      const int m = DIR == 0 ? l - 1 : l;  // interval entering locus l in processing order
      float* d = scal + ((t & 1) * kSparseScal + f) * CH + k;
      if (f == 0) cp_async4(d, p.thm + l);
      else if (f == 1) cp_async4(d, p.thx + l);
      else if (f == 2 && m >= 0 && m < L - 1) cp_async4(d, p.omr + m);
      else if (f == 3 && m >= 0 && m < L - 1) cp_async4(d, p.rho + m);
      else if (f == 4 && p.n1) cp_async4(d, p.n1 + l);
    }
  };
  issue(0);
  cp_async_commit();
  for (int t = 0; t < nb; ++t) {
    const int b = blk_of(t), base = CH * b, nrows = min(CH, L - base);
    __syncthreads();  // every warp is done with block t-1, whose buffer the next copies reuse
    if (t + 1 < nb) issue(t + 1);
    cp_async_commit();
    cp_async_wait1();  // this thread's copies of block t have landed
    __syncthreads();   // and everyone's
    const float* sc = scal + (t & 1) * kSparseScal * CH;
    bool need_gather = true;
    // One locus.  EV (compile-time) marks the event steps: the block's first (the words are
    // gathered), a window change and a store locus; the other steps run a copy without those
    // branches.
    auto body = [&](const int jj, auto evc) {
      constexpr bool EV = decltype(evc)::value;
      const int kr = DIR == 0 ? jj : nrows - 1 - jj;  // locus l = base + kr is bit kr of the words
      const int l = base + kr;
      const int w = l / p.WS;
      const float tm = sc[0 * CH + kr], tx = sc[1 * CH + kr];
      float c, r;
      if (EV && cur_w < 0) {  // initial locus: alpha = theta pi ; t = theta (beta = 1)
        enter(w, false, 0.0f);
        need_gather = true;
        c = 0.0f;
        r = DIR == 0 ? pi : 1.0f;
      } else {
        if (EV && w != cur_w) {
          const float s_set = set_sum();
          const int nout_old = N - 1 - nset;
          const float fill = (p.pool && nout_old > 0) ? opool / (float)nout_old : 0.0f;
          const float mapped = enter(w, true, fill);
          if (DIR == 0 && s_set > 0.0f) lost_max = fmaxf(lost_max, 1.0f - mapped / s_set);
          if (p.pool) opool = fmaxf(opool + (s_set - mapped) - (float)n_enter * fill, 0.0f);
          need_gather = true;
        }
        const float om = sc[2 * CH + kr], rh = sc[3 * CH + kr];  // interval entering locus l
        if (DIR == 0) {
          c = om / sum_prev;
          r = rh * pi;
        } else {
          // S = pi sum_{k in S'} t_k over the set of locus l+1 (the transition's target set)
          c = om / (pi * sum_prev);
          r = rh;
        }
      }
      if (EV && need_gather) {
        gather(b);
        need_gather = false;
      }
      const uint32_t tb = (twd >> kr) & 1u;
      const uint32_t mk = 1u << kr;
      const bool is_store = EV && store_next < p.n_store && p.store_loci[store_next] == l;
      float* srow = is_store ? p.store + ((size_t)p.store_slot[store_next] * N + i) * K : nullptr;
      if (DIR == 1 && is_store) {
        // posterior: alpha (stored by the forward) times beta = c t + r over the set, plus (pool) the
        // pool's forward mass times the outside donors' mean backward value c (o / n_out) + r
        constexpr float S = kSparseProdScale;
        float zb = 0.0f;
#pragma unroll
        for (int q = 0; q < KS; ++q) {
          const int sq = 32 * q + lane;
          if (sq < K && id[q] >= 0) zb += srow[sq] * (fmaf(c, x[q], r) * S);
        }
        zb = warp_sum(zb);
        const int nout = N - 1 - nset;
        const size_t so = (size_t)p.store_slot[store_next] * N + i;
        const float zp = (p.pool && nout > 0) ? p.poolf[so] * (fmaf(c, opool / (float)nout, r) * S) : 0.0f;
        const float z = zb + zp;
        const float inv = z > 0.0f ? 1.0f / z : 0.0f;
#pragma unroll
        for (int q = 0; q < KS; ++q) {
          const int sq = 32 * q + lane;
          if (active && sq < K)
            srow[sq] = id[q] < 0 ? 0.0f : (z > 0.0f ? srow[sq] * (fmaf(c, x[q], r) * S) * inv : eps);
        }
        if (p.pool && active && lane == 0) p.share[so] = (nout > 0 && z > 0.0f) ? zp * inv / (float)nout : 0.0f;
        if (p.pout && active && lane == 0) p.pout[so] = z > 0.0f ? zp * inv : 0.0f;
      }
      float s = 0.0f;
      int nmatch = 0;  // set entries matching the target's allele
#pragma unroll
      for (int q = 0; q < KS; ++q) {
        const bool mis = (mm[q] & mk) != 0u;
        nmatch += mis ? 0 : 1;
        x[q] = (mis ? tx : tm) * fmaf(c, x[q], r);  // theta (c x + r)
        s += x[q];
      }
      xs = tx * fmaf(c, xs, r);
      s = warp_sum(s) - (float)(32 * KS - nset) * xs;
      float tot = s;
      if (p.pool) {
        // outside donors: their count, how many match the target here, their summed emission
        const int n1 = __float_as_int(sc[4 * CH + kr]);
        const int mtot = (tb ? n1 : N - n1) - 1;  // matching donors, the target itself excluded
        const int nout = N - 1 - nset;
        const int mout = min(max(mtot - __reduce_add_sync(0xffffffffu, nmatch), 0), nout);
        const float thsum = tm * (float)mout + tx * (float)(nout - mout);
        const float thbar = nout > 0 ? thsum / (float)nout : 0.0f;
        opool = thbar * (c * opool) + r * thsum;
        tot = s + opool;
      }
      if (is_store) {
        if (DIR == 0) {
#pragma unroll
          for (int q = 0; q < KS; ++q) {
            const int sq = 32 * q + lane;
            if (active && sq < K) srow[sq] = id[q] >= 0 ? x[q] : 0.0f;
          }
          if (p.pool && active && lane == 0) p.poolf[(size_t)p.store_slot[store_next] * N + i] = opool;
        }
        ++store_next;
      }
      if (tot < 1.17549435e-38f) stb |= 1u;      // LS_STATUS_UNDERFLOW
      if (!(tot <= 3.40282347e+38f)) stb |= 2u;  // LS_STATUS_OVERFLOW (infinite or NaN)
      if (DIR == 0) logacc += (double)logf(tot);
      sum_prev = tot;
    };
    for (int jj = 0; jj < nrows;) {
      body(jj++, std::true_type{});
      // the next event in this block: a window change (the first step whose locus lies outside the
      // current window) or a store locus
      int ev = nrows;
      const int wlo = cur_w * p.WS, whi = wlo + p.WS;  // the current window's loci [wlo, whi)
      const int lb = DIR == 0 ? whi : wlo - 1;         // the first locus beyond it, in processing order
      if (lb >= base && lb < base + nrows) ev = min(ev, DIR == 0 ? lb - base : nrows - 1 - (lb - base));
      if (store_next < p.n_store) {
        const int ks = p.store_loci[store_next] - base;
        if (ks >= 0 && ks < nrows) ev = min(ev, DIR == 0 ? ks : nrows - 1 - ks);
      }
      for (; jj < ev; ++jj) body(jj, std::false_type{});
    }
  }
  if (active && lane == 0) {
    if (DIR == 0 && p.logs) p.logs[i] = logacc;
    if (DIR == 0 && p.lost) p.lost[i] = lost_max;
    if (p.status && stb) atomicOr(p.status + i, stb);
  }
}

// Half distances -log(max(p, eps))/2 of the sparse posteriors into dense [D][N][N] rows.  Every
// entry of row i is first set to the outside donors' estimate: the half distance of the pool's
// share (share != null), stored NEGATED so that it stays distinguishable (its sign bit, -0.0
// included), or NaN without a pool; then the set's donors get their own half distances (>= 0).
// grid (N, D), 256 threads.
__global__ void sparse_hdist_kernel(const float* __restrict__ P, const int32_t* __restrict__ idx, int N, int K, int Wn,
                                    const int* __restrict__ win_of_slot, const float* __restrict__ share,
                                    float* __restrict__ h) {
  constexpr float eps = 2.220446049250313e-16f;
  const int i = blockIdx.x, k = blockIdx.y;
  const int w = win_of_slot[k];
  const int32_t* ids = idx + ((size_t)i * Wn + w) * K;
  const float* pr = P + ((size_t)k * N + i) * K;
  float* hr = h + ((size_t)k * N + i) * N;
  // -log(p)/2 >= 0 for p <= 1: computed as |log(p)/2| so that p = 1 gives +0.0 (chain values keep
  // the sign bit clear); estimates are stored as -|log(share)/2| (sign bit set, -0.0 included)
  const float est =
      share ? -fabsf(0.5f * logf(fminf(fmaxf(share[(size_t)k * N + i], eps), 1.0f))) : __int_as_float(0xffffffff);
  for (int j = threadIdx.x; j < N; j += blockDim.x) hr[j] = j == i ? 0.0f : est;
  __syncthreads();
  for (int q = threadIdx.x; q < K; q += blockDim.x) {
    const int j = ids[q];
    if (j >= 0 && j < N && j != i) hr[j] = fabsf(0.5f * logf(fminf(fmaxf(pr[q], eps), 1.0f)));
  }
}

// d = |h| + |h^T| in place over D stacked N x N matrices of half distances, with trust bits:
// bit j of word j/32 of mask row i (mask [D][N][wpr], wpr = ceil(N/32)) is 1 where both halves are
// chain values (sign bit clear) and either both targets have dense rows (dense_row[i] and
// dense_row[j]) or d_ij <= d_trust.  A NaN half (no pool) leaves d NaN and the bit 0.  Tiles as in
// symmetrize_kernel; a warp holds 32 consecutive columns of one row, so one ballot gives a word.
__global__ void symmetrize_trust_kernel(float* __restrict__ d, int N, const uint8_t* __restrict__ dense_row,
                                        float d_trust, uint32_t* __restrict__ mask, int wpr) {
  const int bx = blockIdx.x, by = blockIdx.y;
  if (bx > by) return;
  float* m = d + (size_t)blockIdx.z * N * N;
  uint32_t* mk = mask ? mask + (size_t)blockIdx.z * N * wpr : nullptr;
  __shared__ float A[32][33], B[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int ra = bx * 32 + k, ca = by * 32 + tx;
    const int rb = by * 32 + k, cb = bx * 32 + tx;
    A[k][tx] = (ra < N && ca < N) ? m[(size_t)ra * N + ca] : 0.0f;
    B[k][tx] = (rb < N && cb < N) ? m[(size_t)rb * N + cb] : 0.0f;
  }
  __syncthreads();
  auto one = [&](int row, int col, float a, float b) {
    const bool in = row < N && col < N;
    const float v = row == col ? 0.0f : fabsf(a) + fabsf(b);
    const bool chain = !signbit(a) && !signbit(b) && v == v;
    const bool dense = dense_row && in && dense_row[row] && dense_row[col];
    const bool t = in && row != col && chain && (dense || v <= d_trust);
    if (in) m[(size_t)row * N + col] = v;
    const uint32_t word = __ballot_sync(0xffffffffu, t);
    if (mk && tx == 0 && row < N) mk[(size_t)row * wpr + (col >> 5)] = word;
  };
  for (int k = ty; k < 32; k += 8) {
    one(bx * 32 + k, by * 32 + tx, A[k][tx], B[tx][k]);
    if (bx != by) one(by * 32 + k, bx * 32 + tx, B[k][tx], A[tx][k]);
  }
}

// Dense fallback rows: products alpha^l t^l (t = theta beta, the dense backward's decode product)
// of nf listed targets ([D][nf][N]) divided by theta^l (the locus' alleles from the packed rows,
// decode locus of slot k in dloci[k]) and normalised into half distances of rows tlist[r] of h
// ([D][N][N]).  grid (nf, D), 256 threads.
__global__ void dense_rows_hdist_kernel(const float* __restrict__ prod, int nf, int N, const int* __restrict__ tlist,
                                        const uint32_t* __restrict__ bits, int row_words, const float* __restrict__ thm,
                                        const float* __restrict__ thx, const int* __restrict__ dloci,
                                        float* __restrict__ h) {
  constexpr float eps = 2.220446049250313e-16f;
  const int r = blockIdx.x, k = blockIdx.y;
  const int i = tlist[r];
  const int l = dloci[k];
  const uint32_t* row = bits + (size_t)l * row_words;
  const uint32_t ai = (row[i >> 5] >> (i & 31)) & 1u;
  const float im = thm[l] > 0.0f ? 1.0f / thm[l] : 0.0f, ix = thx[l] > 0.0f ? 1.0f / thx[l] : 0.0f;
  const float* a0 = prod + ((size_t)k * nf + r) * N;
  auto a = [&](int j) { return a0[j] * ((((row[j >> 5] >> (j & 31)) & 1u) == ai) ? im : ix); };
  float s = 0.0f;
  for (int j = threadIdx.x; j < N; j += blockDim.x)
    if (j != i) s += a(j);
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
  float* o = h + ((size_t)k * N + i) * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const float q = Z > 0.0f ? a(j) * invZ : eps;
    o[j] = j == i ? 0.0f : fabsf(0.5f * logf(fminf(fmaxf(q, eps), 1.0f)));  // +0.0 at q = 1 (a chain value)
  }
}

// Widened sets: U^w = S^w u S^{w+1} (span 1) or S^{w-1} u S^w u S^{w+1} (span 2), missing windows
// empty.  A donor proposed for window w+1 is already carried through window w, so it enters with
// a window of history; with span 2 a donor proposed for window w also stays through w+1, so the
// forward mass of donors about to mismatch decays inside the chain instead of being cut at the
// window change.  One thread per (target, window): a merge of up to three ascending lists with
// duplicates removed, -1 padding to (span + 1) K entries.
__global__ void lookahead_sets_kernel(const int32_t* __restrict__ idx, int N, int Wn, int K, int span,
                                      int32_t* __restrict__ U) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * Wn) return;
  const int w = (int)(t % Wn);
  const int32_t* lists[3];
  int pos[3] = {0, 0, 0};
  int nl = 0;
  if (span >= 2 && w > 0) lists[nl++] = idx + (t - 1) * K;
  lists[nl++] = idx + t * K;
  if (w + 1 < Wn) lists[nl++] = idx + (t + 1) * K;
  const int width = (span + 1) * K;
  int32_t* u = U + t * width;
  int o = 0, last = -1;
  while (true) {
    int best = -1;
    for (int q = 0; q < nl; ++q) {
      const int v = pos[q] < K ? lists[q][pos[q]] : -1;
      if (v >= 0 && (best < 0 || v < best)) best = v;
    }
    if (best < 0) break;
    for (int q = 0; q < nl; ++q)
      if (pos[q] < K && lists[q][pos[q]] == best) ++pos[q];
    if (best != last) u[o++] = best;
    last = best;
  }
  while (o < width) u[o++] = -1;
}

// Haplotypes carrying allele 1 at each locus: one warp per row, popcount of the first N bits.
__global__ void row_ones_kernel(const uint32_t* __restrict__ bits, int row_words, int N, int L, int32_t* __restrict__ n1) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= L) return;
  const uint32_t* r = bits + (size_t)wid * row_words;
  int c = 0;
  for (int k = lane; 32 * k < N; k += 32) {
    uint32_t v = r[k];
    const int rem = N - 32 * k;
    if (rem < 32) v &= (1u << rem) - 1u;
    c += __popc(v);
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if (lane == 0) n1[wid] = c;
}

#endif  // LS_SPARSE_PARAMS_ONLY

}  // namespace lsk
