/*
 * ls_oracle.c -- plain FP64 CPU oracle for the Li & Stephens (LS) all-vs-all hot path
 * described in the kalis paper (arXiv 2212.11403).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls this file;
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may use it.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * Every routine works on one recipient (target) haplotype i at a time, in double precision,
 * with the loops written exactly in the order of the equation it implements.  Loci are 0-based
 * here (the paper's variant l is our locus l-1).  Readings of the paper used throughout:
 *   - rho[l] (l = 0..L-2) is the recombination probability of the interval between loci l and
 *     l+1: the forward step l -> l+1 and the backward step l+1 -> l both use rho[l]
 *     (Sec. 2.1 "rho[i] between variants i and i+1"; Eq. fwd1 / bck1 index it by the earlier
 *     locus of the pair).
 *   - Pi is recipient-major: Pi[i*N + j] = the paper's Pi_ji, prior that recipient i copies
 *     donor j; Pi_ii = 0.  Pi == NULL means the uniform prior 1/(N-1) (Sec. 3.3 "Parameters").
 *   - mu has length 1 (scalar) or L (one value per locus), Table tab:pars.
 *   - The emission uses the numerically safe form theta = (1-H)(1-2mu)+mu, H = h_j XOR h_i
 *     (App. A.3).
 * Parity status of each routine is listed in its comment ("pinned by ...").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* epsilon of Eq. distmat: the double-precision machine epsilon (Sec. 2.1). */
static const double LSO_EPS = 2.220446049250313080847263336181640625e-16;

/* Eq. emission in the form of App. A.3.  Pinned by brute-force enumeration. */
static double lso_theta(int hj, int hi, double mu) {
  int H = (hj ^ hi) & 1;
  return (1.0 - H) * (1.0 - 2.0 * mu) + mu;
}

static double lso_mu(const double* mu, int mu_len, int l) { return mu_len == 1 ? mu[0] : mu[l]; }

/* The prior row of recipient i in a recipient-major Pi (NULL: the uniform prior). */
static const double* lso_prior_row(const double* Pi, int N, int i) { return Pi ? Pi + (size_t)i * N : NULL; }

/* Prior copying probability Pi_ji (Sec. 2.1, Sec. 3.3) from recipient i's row; uniform 1/(N-1) off
 * the diagonal when the row is NULL. */
static double lso_prior(const double* pirow, int N, int i, int j) {
  if (j == i) return 0.0;
  if (pirow == NULL) return 1.0 / (double)(N - 1);
  return pirow[j];
}

/* Eq. rho: rho = 1 - exp(-Ne * m^gamma), evaluated with expm1.  Pinned by the CalcRho values the
 * paper prints (Sec. 3.3). */
int lso_calc_rho(const double* m, int n, double Ne, double gamma, double* rho) {
  for (int k = 0; k < n; ++k) rho[k] = -expm1(-Ne * pow(m[k], gamma));
  return 0;
}

/* Paper's bit-packed haplotype cache layout (Sec. 4.1.1, fig:hapsmem): variant-major, 32
 * consecutive haplotypes per uint32 (haplotype i in bit i%32 of word i/32), each variant row
 * padded to a 32-byte boundary.  Returns the byte size; fills out (if not NULL) with
 * L * stride_words words.  Pinned by the printed cache size for 300 x 400 (Sec. 3.2). */
long lso_pack_paper_layout(const uint8_t* h, int N, int L, uint32_t* out) {
  long words = (N + 31) / 32;
  long stride_bytes = ((words * 4 + 31) / 32) * 32;
  long stride_words = stride_bytes / 4;
  if (out) {
    memset(out, 0, (size_t)stride_bytes * L);
    for (int l = 0; l < L; ++l)
      for (int i = 0; i < N; ++i)
        if (h[(size_t)l * N + i]) out[(size_t)l * stride_words + i / 32] |= (uint32_t)1u << (i % 32);
  }
  return stride_bytes * (long)L;
}

/*
 * Rescaled forward recursion, Eq. fwd0 / fwd1 (derivation App. A.1), recipient i.
 *   alpha^0_j = theta^0_j pi_j
 *   alpha^l_j = theta^l_j ( (1-rho[l-1]) alpha^{l-1}_j / sum_k alpha^{l-1}_k + rho[l-1] pi_j )
 * and log F^l = sum_{k<=l} log sum_j alpha^k_j (F^l = sum_j alpha~^l_j, Eq. F, since
 * alpha^l = alpha~^l / F^{l-1}).
 * slot[l] >= 0 asks for alpha^l (into alpha_out + slot*N) and log F^l (into logF_out[slot]).
 * Returns log F at the last locus = log P(h_i | h_-i) (Sec. 2.1, PAC term).
 * Pinned by brute force, the rho=0 / rho=1 closed forms and the raw recursion below.
 */
static double lso_forward_row(const uint8_t* h, int N, int L, const double* rho, const double* mu, int mu_len,
                              const double* pirow, int i, const int* slot, double* alpha_out, double* logF_out) {
  double* a = (double*)malloc(sizeof(double) * N);
  double* b = (double*)malloc(sizeof(double) * N);
  double logF = 0.0;
  for (int l = 0; l < L; ++l) {
    const uint8_t* hl = h + (size_t)l * N;
    double m = lso_mu(mu, mu_len, l);
    if (l == 0) {
      for (int j = 0; j < N; ++j) b[j] = lso_theta(hl[j], hl[i], m) * lso_prior(pirow, N, i, j);
    } else {
      double s = 0.0;
      for (int j = 0; j < N; ++j) s += a[j];
      double r = rho[l - 1];
      for (int j = 0; j < N; ++j)
        b[j] = lso_theta(hl[j], hl[i], m) * ((1.0 - r) * a[j] / s + r * lso_prior(pirow, N, i, j));
    }
    b[i] = 0.0; /* pi_ii = 0 makes alpha_ii identically zero */
    double s_new = 0.0;
    for (int j = 0; j < N; ++j) s_new += b[j];
    logF += log(s_new);
    double* t = a; a = b; b = t;
    if (slot && slot[l] >= 0) {
      if (alpha_out) memcpy(alpha_out + (size_t)slot[l] * N, a, sizeof(double) * N);
      if (logF_out) logF_out[slot[l]] = logF;
    }
  }
  free(a);
  free(b);
  return logF;
}

/*
 * Rescaled backward recursion, Eq. bck0 / bck1 (derivation App. A.2), recipient i.
 *   beta^{L-1}_j = 1
 *   beta^l_j = (1-rho[l]) beta^{l+1}_j theta^{l+1}_j / S^{l+1} + rho[l],
 *   S^{l+1} = sum_{j != i} beta^{l+1}_j theta^{l+1}_j pi_j
 * log G at locus l = sum_{k=l+1}^{L-1} log S^k (G^l of Eq. G with G at the last locus = 1).
 * slot[l] >= 0 asks for beta^l and log G at l.  beta_ii is reported as 0 (the diagonal carries
 * no probability: pi_ii = 0).
 * Returns log G^0-ish likelihood: log G at locus 0 + log sum_j beta^0_j theta^0_j pi_j, which
 * equals log P(h_i | h_-i).  Pinned by forward/backward likelihood agreement and brute force.
 */
static double lso_backward_row(const uint8_t* h, int N, int L, const double* rho, const double* mu, int mu_len,
                               const double* pirow, int i, const int* slot, double* beta_out, double* logG_out) {
  double* bt = (double*)malloc(sizeof(double) * N);
  double* nb = (double*)malloc(sizeof(double) * N);
  double logG = 0.0;
  for (int j = 0; j < N; ++j) bt[j] = 1.0;
  for (int l = L - 1; l >= 0; --l) {
    if (l < L - 1) {
      const uint8_t* h1 = h + (size_t)(l + 1) * N;
      double m1 = lso_mu(mu, mu_len, l + 1);
      double S = 0.0;
      for (int j = 0; j < N; ++j)
        if (j != i) S += bt[j] * lso_theta(h1[j], h1[i], m1) * lso_prior(pirow, N, i, j);
      double r = rho[l];
      for (int j = 0; j < N; ++j) nb[j] = (1.0 - r) * bt[j] * lso_theta(h1[j], h1[i], m1) / S + r;
      logG += log(S);
      double* t = bt; bt = nb; nb = t;
    }
    if (slot && slot[l] >= 0) {
      if (beta_out) {
        double* dst = beta_out + (size_t)slot[l] * N;
        memcpy(dst, bt, sizeof(double) * N);
        dst[i] = 0.0;
      }
      if (logG_out) logG_out[slot[l]] = logG;
    }
  }
  const uint8_t* h0 = h;
  double m0 = lso_mu(mu, mu_len, 0);
  double S0 = 0.0;
  for (int j = 0; j < N; ++j)
    if (j != i) S0 += bt[j] * lso_theta(h0[j], h0[i], m0) * lso_prior(pirow, N, i, j);
  free(bt);
  free(nb);
  return logG + log(S0);
}

/*
 * Posterior copying probabilities, Eq. postprob: p_j = alpha_j beta_j / sum_k alpha_k beta_k,
 * with p_j = eps for every j != i when the sum is 0 (Sec. 2.2).  p_ii = 0.
 * Pinned by sum-to-one, the rho closed forms and brute-force marginals.
 */
void lso_posterior(const double* alpha, const double* beta, int N, int i, double* p) {
  double s = 0.0;
  for (int j = 0; j < N; ++j)
    if (j != i) s += alpha[j] * beta[j];
  for (int j = 0; j < N; ++j) {
    if (j == i) p[j] = 0.0;
    else if (s == 0.0) p[j] = LSO_EPS;
    else p[j] = alpha[j] * beta[j] / s;
  }
}

/* Eq. distmat for one pair: d_ji = -(log(p_ji v eps) + log(p_ij v eps)) / 2 (d_ii = 0 by
 * convention).  p_ji = posterior that recipient i copies donor j. */
double lso_distance_pair(double p_ji, double p_ij) {
  double a = p_ji > LSO_EPS ? p_ji : LSO_EPS;
  double b = p_ij > LSO_EPS ? p_ij : LSO_EPS;
  return -(log(a) + log(b)) / 2.0;
}

double lso_forward_target(const uint8_t* h, int N, int L, const double* rho, const double* mu, int mu_len,
                          const double* Pi, int i, const int* slot, double* alpha_out, double* logF_out) {
  return lso_forward_row(h, N, L, rho, mu, mu_len, lso_prior_row(Pi, N, i), i, slot, alpha_out, logF_out);
}

double lso_backward_target(const uint8_t* h, int N, int L, const double* rho, const double* mu, int mu_len,
                           const double* Pi, int i, const int* slot, double* beta_out, double* logG_out) {
  return lso_backward_row(h, N, L, rho, mu, mu_len, lso_prior_row(Pi, N, i), i, slot, beta_out, logG_out);
}

/*
 * Raw (unscaled) recursions, Eq. raw_forward / raw_backward with F, G of Eq. F / Eq. G, for
 * tiny L only (no rescaling, so they underflow on long inputs).  Used to pin the rescaled
 * forms (App. A.1, A.2).  alpha_t[l*N + j] = alpha~^l_j, F[l] = F^l = sum_j alpha~^l_j;
 * beta_t[l*N + j] = beta~^l_j, G[l] = sum_j beta~^{l+1}_j theta^{l+1}_j pi_j (G[L-1] = 1).
 */
void lso_raw_forward_target(const uint8_t* h, int N, int L, const double* rho, const double* mu, int mu_len,
                            const double* Pi, int i, double* alpha_t, double* F) {
  const double* pirow = lso_prior_row(Pi, N, i);
  for (int l = 0; l < L; ++l) {
    const uint8_t* hl = h + (size_t)l * N;
    double m = lso_mu(mu, mu_len, l);
    for (int j = 0; j < N; ++j) {
      double pij = lso_prior(pirow, N, i, j);
      if (l == 0) alpha_t[j] = lso_theta(hl[j], hl[i], m) * pij;
      else
        alpha_t[(size_t)l * N + j] = lso_theta(hl[j], hl[i], m) *
                                     ((1.0 - rho[l - 1]) * alpha_t[(size_t)(l - 1) * N + j] + rho[l - 1] * F[l - 1] * pij);
    }
    F[l] = 0.0;
    for (int j = 0; j < N; ++j) F[l] += alpha_t[(size_t)l * N + j];
  }
}

void lso_raw_backward_target(const uint8_t* h, int N, int L, const double* rho, const double* mu, int mu_len,
                             const double* Pi, int i, double* beta_t, double* G) {
  const double* pirow = lso_prior_row(Pi, N, i);
  for (int j = 0; j < N; ++j) beta_t[(size_t)(L - 1) * N + j] = 1.0;
  G[L - 1] = 1.0;
  for (int l = L - 2; l >= 0; --l) {
    const uint8_t* h1 = h + (size_t)(l + 1) * N;
    double m1 = lso_mu(mu, mu_len, l + 1);
    double g = 0.0;
    for (int j = 0; j < N; ++j)
      g += beta_t[(size_t)(l + 1) * N + j] * lso_theta(h1[j], h1[i], m1) * lso_prior(pirow, N, i, j);
    G[l] = g;
    for (int j = 0; j < N; ++j)
      beta_t[(size_t)l * N + j] = (1.0 - rho[l]) * beta_t[(size_t)(l + 1) * N + j] * lso_theta(h1[j], h1[i], m1) + rho[l] * g;
  }
}

/*
 * Batch driver: forward + backward for each target in targets[0..nt), keeping the results at
 * the requested loci (any order, 0-based).  Outputs (any may be NULL):
 *   alpha, beta, post : [nt][nl][N]      logF, logG : [nt][nl]      llf, llb : [nt]
 * OpenMP over targets (each target is an independent HMM, Sec. 3.7.1).
 */
static int lso_run_impl(const uint8_t* h, int N, int L, const double* rho, const double* mu, int mu_len,
                        const double* Pi, int pi_rows, const int* targets, int nt, const int* loci, int nl,
                        double* alpha, double* beta, double* post, double* logF, double* logG, double* llf,
                        double* llb, int nthreads) {
  if (N < 2 || L < 1 || nt < 0 || nl < 0) return -1;
  for (int k = 0; k < nl; ++k)
    if (loci[k] < 0 || loci[k] >= L) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  int err = 0;
#pragma omp parallel
  {
    int* slot = (int*)malloc(sizeof(int) * L);
    double* A = (double*)malloc(sizeof(double) * (size_t)nl * N + 1);
    double* B = (double*)malloc(sizeof(double) * (size_t)nl * N + 1);
    double* lF = (double*)malloc(sizeof(double) * (nl + 1));
    double* lG = (double*)malloc(sizeof(double) * (nl + 1));
    for (int l = 0; l < L; ++l) slot[l] = -1;
    for (int k = 0; k < nl; ++k) slot[loci[k]] = k;
#pragma omp for schedule(dynamic, 1)
    for (int t = 0; t < nt; ++t) {
      int i = targets[t];
      if (i < 0 || i >= N) { err = -1; continue; }
      const double* pirow = pi_rows ? (Pi ? Pi + (size_t)t * N : NULL) : lso_prior_row(Pi, N, i);
      double f = lso_forward_row(h, N, L, rho, mu, mu_len, pirow, i, slot, A, lF);
      double b = lso_backward_row(h, N, L, rho, mu, mu_len, pirow, i, slot, B, lG);
      for (int k = 0; k < nl; ++k) {
        /* a locus may be requested twice: copy from the slot that was filled */
        int s = slot[loci[k]];
        if (alpha) memcpy(alpha + ((size_t)t * nl + k) * N, A + (size_t)s * N, sizeof(double) * N);
        if (beta) memcpy(beta + ((size_t)t * nl + k) * N, B + (size_t)s * N, sizeof(double) * N);
        if (post) lso_posterior(A + (size_t)s * N, B + (size_t)s * N, N, i, post + ((size_t)t * nl + k) * N);
        if (logF) logF[(size_t)t * nl + k] = lF[s];
        if (logG) logG[(size_t)t * nl + k] = lG[s];
      }
      if (llf) llf[t] = f;
      if (llb) llb[t] = b;
    }
    free(slot);
    free(A);
    free(B);
    free(lF);
    free(lG);
  }
  return err;
}

int lso_run(const uint8_t* h, int N, int L, const double* rho, const double* mu, int mu_len, const double* Pi,
            const int* targets, int nt, const int* loci, int nl, double* alpha, double* beta, double* post,
            double* logF, double* logG, double* llf, double* llb, int nthreads) {
  return lso_run_impl(h, N, L, rho, mu, mu_len, Pi, 0, targets, nt, loci, nl, alpha, beta, post, logF, logG, llf, llb,
                      nthreads);
}

/* The same with only the targets' prior rows: Pi_rows[t*N + j] = Pi_{j, targets[t]} (recipient-major
 * rows, diagonal entry ignored), so that large N needs no N x N host matrix. */
int lso_run_rows(const uint8_t* h, int N, int L, const double* rho, const double* mu, int mu_len,
                 const double* Pi_rows, const int* targets, int nt, const int* loci, int nl, double* alpha,
                 double* beta, double* post, double* logF, double* logG, double* llf, double* llb, int nthreads) {
  return lso_run_impl(h, N, L, rho, mu, mu_len, Pi_rows, 1, targets, nt, loci, nl, alpha, beta, post, logF, logG, llf,
                      llb, nthreads);
}

/*
 * Distances among a set of targets at one locus, Eq. distmat.  post[t*N + j] = p_{j, targets[t]}
 * (posterior of recipient targets[t] copying donor j).  d[a*nt + b] = d between targets[a] and
 * targets[b]; d[a*nt + a] = 0.
 */
void lso_distance_block(const double* post, const int* targets, int nt, int N, double* d) {
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      if (a == b) { d[(size_t)a * nt + b] = 0.0; continue; }
      double p_ba = post[(size_t)a * N + targets[b]]; /* recipient targets[a] copies targets[b] */
      double p_ab = post[(size_t)b * N + targets[a]];
      d[(size_t)a * nt + b] = lso_distance_pair(p_ba, p_ab);
    }
}

/*
 * Gradient of log P(h_i | h_-i) by the Fisher identity (score = posterior expectation of the
 * complete-data score), for one recipient.  Derived from Eq. emission and Eq. transition:
 *   d logP / d rho[m] = (1 - A_m) / (rho[m] + (1 - rho[m]) A_m),
 *     A_m = sum_j a_j theta^{m+1}_j b_j,  a = alpha^m / sum alpha^m,  b = beta^{m+1} / S^{m+1}
 *   d logP / d mu (scalar mu) = sum_l sum_{j != i} p^l_j (H ? 1/mu : -1/(1-mu))
 * Chain rule to the log parameters: d/dlog mu = mu d/dmu; with interval_of[m] = k in [0,K),
 * d/dlog rho_k = sum_{m in I_k} rho[m] d/drho[m].  Results are ADDED to dlogmu[0], dlogrho[k].
 * Stores alpha for all loci (L*N doubles), so it is meant for small N.
 * Pinned by central finite differences of the brute-force likelihood and of lso_forward_target.
 */
double lso_grad_target(const uint8_t* h, int N, int L, const double* rho, const double* mu, int mu_len,
                       const double* Pi, int i, const int* interval_of, double* dlogmu, double* dlogrho) {
  const double* pirow = lso_prior_row(Pi, N, i);
  double* A = (double*)malloc(sizeof(double) * (size_t)L * N); /* normalised alpha^l */
  double* a = (double*)malloc(sizeof(double) * N);
  double* b = (double*)malloc(sizeof(double) * N);
  double logF = 0.0;
  for (int l = 0; l < L; ++l) {
    const uint8_t* hl = h + (size_t)l * N;
    double m = lso_mu(mu, mu_len, l);
    if (l == 0) {
      for (int j = 0; j < N; ++j) b[j] = lso_theta(hl[j], hl[i], m) * lso_prior(pirow, N, i, j);
    } else {
      double r = rho[l - 1];
      for (int j = 0; j < N; ++j) b[j] = lso_theta(hl[j], hl[i], m) * ((1.0 - r) * a[j] + r * lso_prior(pirow, N, i, j));
    }
    b[i] = 0.0;
    double s = 0.0;
    for (int j = 0; j < N; ++j) s += b[j];
    logF += log(s);
    for (int j = 0; j < N; ++j) a[j] = b[j] / s;  /* a = alpha^l / sum alpha^l */
    memcpy(A + (size_t)l * N, a, sizeof(double) * N);
  }
  /* backward sweep with beta (Eq. bck1), forming A_m and the posteriors */
  double* bt = (double*)malloc(sizeof(double) * N);
  double* nb = (double*)malloc(sizeof(double) * N);
  for (int j = 0; j < N; ++j) bt[j] = 1.0;
  double gmu = 0.0;
  for (int l = L - 1; l >= 0; --l) {
    const uint8_t* hl = h + (size_t)l * N;
    double m = lso_mu(mu, mu_len, l);
    /* posterior at l from normalised alpha^l and beta^l */
    double z = 0.0;
    for (int j = 0; j < N; ++j)
      if (j != i) z += A[(size_t)l * N + j] * bt[j];
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      double p = A[(size_t)l * N + j] * bt[j] / z;
      int H = (hl[j] ^ hl[i]) & 1;
      double score = H ? 1.0 / m : -1.0 / (1.0 - m);
      gmu += m * p * score; /* mu d/dmu; for a per-locus mu vector this is the sum over loci */
    }
    if (l > 0) {
      int mm = l - 1; /* interval between loci l-1 and l */
      double S = 0.0;
      for (int j = 0; j < N; ++j)
        if (j != i) S += bt[j] * lso_theta(hl[j], hl[i], m) * lso_prior(pirow, N, i, j);
      double Am = 0.0;
      for (int j = 0; j < N; ++j)
        if (j != i) Am += A[(size_t)mm * N + j] * lso_theta(hl[j], hl[i], m) * bt[j] / S;
      double r = rho[mm];
      double g = (1.0 - Am) / (r + (1.0 - r) * Am);
      if (interval_of && dlogrho) dlogrho[interval_of[mm]] += r * g;
      for (int j = 0; j < N; ++j) nb[j] = (1.0 - r) * bt[j] * lso_theta(hl[j], hl[i], m) / S + r;
      double* t = bt; bt = nb; nb = t;
    }
  }
  if (dlogmu) dlogmu[0] += gmu;
  free(A);
  free(a);
  free(b);
  free(bt);
  free(nb);
  return logF;
}

/* PAC log-likelihood and its gradient summed over targets (OpenMP over targets). */
int lso_pac_grad(const uint8_t* h, int N, int L, const double* rho, const double* mu, int mu_len, const double* Pi,
                 const int* targets, int nt, const int* interval_of, int K, double* pac, double* dlogmu,
                 double* dlogrho, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  double tot = 0.0, gm = 0.0;
  double* gr = (double*)calloc((size_t)K + 1, sizeof(double));
#pragma omp parallel
  {
    double* lr = (double*)calloc((size_t)K + 1, sizeof(double));
    double lm = 0.0, lt = 0.0;
#pragma omp for schedule(dynamic, 1)
    for (int t = 0; t < nt; ++t) lt += lso_grad_target(h, N, L, rho, mu, mu_len, Pi, targets[t], interval_of, &lm, lr);
#pragma omp critical
    {
      tot += lt;
      gm += lm;
      for (int k = 0; k < K; ++k) gr[k] += lr[k];
    }
    free(lr);
  }
  if (pac) *pac = tot;
  if (dlogmu) *dlogmu = gm;
  if (dlogrho) memcpy(dlogrho, gr, sizeof(double) * K);
  free(gr);
  return 0;
}
