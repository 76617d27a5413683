// ls_api.cu -- host implementation of the libls C ABI (include/ls.h): haplotype cache, parameter
// handling, forward/backward tables, the launch planner and the fused all-vs-all pipeline.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ls.h"
#include "ls_aux.cuh"
#define LS_SPARSE_PARAMS_ONLY
#include "ls_sparse.cuh"
#include "ls_internal.h"

void ls_register_group0(std::vector<PropKernelInfo>& out);
void ls_register_group1(std::vector<PropKernelInfo>& out);
void ls_register_group2(std::vector<PropKernelInfo>& out);
void ls_register_group3(std::vector<PropKernelInfo>& out);
void ls_register_group4(std::vector<PropKernelInfo>& out);
void ls_register_group5(std::vector<PropKernelInfo>& out);
void ls_register_group6(std::vector<PropKernelInfo>& out);
void ls_register_group7(std::vector<PropKernelInfo>& out);
void ls_register_group8(std::vector<PropKernelInfo>& out);
void ls_register_group9(std::vector<PropKernelInfo>& out);
void ls_register_group10(std::vector<PropKernelInfo>& out);
void ls_register_group11(std::vector<PropKernelInfo>& out);
void ls_register_group12(std::vector<PropKernelInfo>& out);
void ls_register_group13(std::vector<PropKernelInfo>& out);
void ls_register_group14(std::vector<PropKernelInfo>& out);
void ls_register_group15(std::vector<PropKernelInfo>& out);
void ls_register_group16(std::vector<PropKernelInfo>& out);
void ls_register_group17(std::vector<PropKernelInfo>& out);

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(x)                                                                         \
  do {                                                                                      \
    cudaError_t e_ = (x);                                                                   \
    if (e_ != cudaSuccess) return fail(LS_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

std::vector<PropKernelInfo>& registry() {
  static std::vector<PropKernelInfo> v;
  static std::once_flag once;
  std::call_once(once, [] {
    ls_register_group0(v);
    ls_register_group1(v);
    ls_register_group2(v);
    ls_register_group3(v);
    ls_register_group4(v);
    ls_register_group5(v);
    ls_register_group6(v);
    ls_register_group7(v);
    ls_register_group8(v);
    ls_register_group9(v);
    ls_register_group10(v);
    ls_register_group11(v);
    ls_register_group12(v);
    ls_register_group13(v);
    ls_register_group14(v);
    ls_register_group15(v);
    ls_register_group16(v);
    ls_register_group17(v);
  });
  return v;
}

int dev_alloc(ls_ctx* c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(LS_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  if (c) c->bytes += bytes;
  return LS_OK;
}

uint64_t fnv1a(uint64_t h, const void* data, size_t n) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

// ---- launch planning -----------------------------------------------------------------------
struct Launch {
  const PropKernelInfo* k;
  int t_begin, t_count, grid, smem;
};

struct Cand {
  const PropKernelInfo* k;
  int smem, per_sm;
};

// Upper bound on compiled variants (the registry is a fixed list; the planner keeps its candidates
// in fixed arrays so that the allocation-free pipeline shares it).
constexpr int kMaxCand = 64;

// Every compiled propagation variant (no statistic passes) that serves N with the context's prior
// kind, fits the shared-memory limit and can be resident.  LS_PROP_VARIANT="tpw,w,kq" keeps only
// that variant: a measurement switch for tuning sweeps, honoured by every entry point alike.
int candidates(ls_ctx* c, Cand* out, int* nout) {
  *nout = 0;
  const int N = c->N;
  const int pim = c->Pi ? 1 : 0;
  int pa = 0, pb = 0, pk = 0;
  const char* ov = getenv("LS_PROP_VARIANT");
  const bool pin = ov && sscanf(ov, "%d,%d,%d", &pa, &pb, &pk) == 3;
  for (const auto& k : registry()) {
    if (*nout >= kMaxCand) break;
    if (k.st != 0 || (k.pim != 0) != (pim != 0) || !k.serves(N)) continue;
    // a prior matrix runs on the variants that hold it as bfloat16 exactly when it has the BF16 format
    if (pim && k.pi16 != c->prior_bf16) continue;
    if (pin && !(k.tpw == pa && k.w == pb && k.kq == pk)) continue;
    const int smem = k.smem_bytes(c->rw2);
    if (smem > 227 * 1024) continue;
    bool ok = true;
    for (int d = 0; d < 2 && ok; ++d)
      if (cudaFuncSetAttribute(k.func[d], cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) ok = false;
    int nb = 0;
    if (ok && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k.func[0], k.w * 32, smem) != cudaSuccess || nb < 1)) ok = false;
    if (!ok) {
      cudaGetLastError();
      continue;
    }
    out[(*nout)++] = Cand{&k, smem, nb};
  }
  if (*nout == 0) {
    if (pin) return fail(LS_ERR_UNSUPPORTED, "LS_PROP_VARIANT=%s does not serve N=%d", ov, N);
    if (pim && !c->prior_bf16 && N > 20480)
      return fail(LS_ERR_UNSUPPORTED, "a prior matrix at N=%d > 20480 needs the BF16 prior format (ls_set_prior_format)", N);
    return fail(LS_ERR_UNSUPPORTED, "no compiled propagation variant serves N=%d", N);
  }
  return LS_OK;
}

// modelled time of one launch: for every wave, (CTAs per SM in that wave) x warps x (slots per
// lane + a fixed per-locus overhead), summed over waves
double cost_of(const Cand& cd, int count, int nsm) {
  const long long ctas = (long long)((count + cd.k->tpw - 1) / cd.k->tpw) * cd.k->cpt;
  const long long per_wave = (long long)nsm * cd.per_sm;
  const long long full = ctas / per_wave, rem = ctas % per_wave;
  // fewer than two warps per scheduler leave the dependent FP32 chain exposed: count it double
  const double unit = cd.k->w * (cd.k->kq + 3.0) * (cd.per_sm * cd.k->w < 8 ? 2.0 : 1.0);
  double t = (double)full * cd.per_sm * unit;
  if (rem) t += (double)((rem + nsm - 1) / nsm) * unit;
  return t;
}

const Cand* best_for(const Cand* cs, int nc, int count, int nsm, double* cost) {
  const Cand* best = nullptr;
  double bc = 1e300;
  for (int i = 0; i < nc; ++i) {
    const Cand& cd = cs[i];
    const double cc = cost_of(cd, count, nsm);
    if (cc < bc * 0.999 || (cc <= bc * 1.001 && best && cd.k->tpw > best->k->tpw)) {
      bc = cc;
      best = &cd;
    }
  }
  *cost = bc;
  return best;
}

// Launch plan for targets [t_begin, t_begin + t_count): full waves of the best variant, then the
// remainder with the variant best for it when that is cheaper.  At most two launches; no heap use
// (the allocation-free pipeline plans with it too).
int plan(ls_ctx* c, int t_begin, int t_count, Launch* out, int* nout) {
  *nout = 0;
  Cand cs[kMaxCand];
  int nc = 0;
  int rc = candidates(c, cs, &nc);
  if (rc) return rc;
  double c1 = 0;
  const Cand* b1 = best_for(cs, nc, t_count, c->num_sms, &c1);
  const int per_wave_t = std::max(1, c->num_sms * b1->per_sm * b1->k->tpw / b1->k->cpt);
  if (t_count > per_wave_t && t_count % per_wave_t != 0) {
    const int main_t = (t_count / per_wave_t) * per_wave_t;
    double ct = 0;
    const double cm = cost_of(*b1, main_t, c->num_sms);
    const Cand* bt = best_for(cs, nc, t_count - main_t, c->num_sms, &ct);
    if (cm + ct < c1) {
      const int tt = t_count - main_t;
      out[0] = Launch{b1->k, t_begin, main_t, main_t / b1->k->tpw, b1->smem};
      out[1] = Launch{bt->k, t_begin + main_t, tt, (tt + bt->k->tpw - 1) / bt->k->tpw, bt->smem};
      *nout = 2;
      return LS_OK;
    }
  }
  out[0] = Launch{b1->k, t_begin, t_count, (t_count + b1->k->tpw - 1) / b1->k->tpw, b1->smem};
  *nout = 1;
  return LS_OK;
}

void base_params(ls_ctx* c, lsk::PropParams& p, int dir) {
  memset(&p, 0, sizeof p);
  p.bits2 = c->bits2;
  p.rw2 = c->rw2;
  p.N = c->N;
  p.L = c->L;
  p.dir = dir;
  p.mu_vec = c->mu_vec;
  p.omr = c->omr;
  p.rr = dir == 0 ? c->rr_f : c->rr_b;
  p.thm = c->thm;
  p.thx = c->thx;
  p.pi_u = c->pi_u;
  p.Pi = c->Pi;
  if (c->Pi && dir == 0) p.rr = c->rr_b;  // the matrix-prior kernel multiplies rho by pi_j itself
  p.err = c->err;
}

int run_launches(ls_ctx* c, lsk::PropParams p, int t_begin, int t_count, cudaStream_t s, int* nlaunch = nullptr) {
  Launch lp[2];
  int nlp = 0;
  int rc = plan(c, t_begin, t_count, lp, &nlp);
  if (rc) return rc;
  if (nlaunch) *nlaunch = nlp;
  // A main/tail plan: the tail (few targets, one small CTA per SM, latency-bound) goes first on a
  // side stream so that its CTAs share SMs with the main waves instead of running after them.
  // LS_TAIL_OVERLAP=0 (a measurement switch) runs both on the caller's stream, in order.
  const char* ov = getenv("LS_TAIL_OVERLAP");
  if (nlp == 2 && !(ov && ov[0] == '0')) {
    if (!c->side) {
      CUDA_TRY(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
      CUDA_TRY(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
      CUDA_TRY(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
    }
    CUDA_TRY(cudaEventRecord(c->fork_ev, s));
    CUDA_TRY(cudaStreamWaitEvent(c->side, c->fork_ev, 0));
    for (int k = 1; k >= 0; --k) {
      const Launch& L = lp[k];
      p.t_begin = L.t_begin;
      p.t_count = L.t_count;
      cudaError_t e = L.k->launch(p.dir, p, L.grid, L.smem, k == 1 ? c->side : s);
      if (e != cudaSuccess) return fail(LS_ERR_CUDA, "propagation launch (TPW=%d W=%d KQ=%d): %s", L.k->tpw, L.k->w,
                                        L.k->kq, cudaGetErrorString(e));
    }
    CUDA_TRY(cudaEventRecord(c->join_ev, c->side));
    CUDA_TRY(cudaStreamWaitEvent(s, c->join_ev, 0));
    return LS_OK;
  }
  for (int i = 0; i < nlp; ++i) {
    const Launch& L = lp[i];
    p.t_begin = L.t_begin;
    p.t_count = L.t_count;
    cudaError_t e = L.k->launch(p.dir, p, L.grid, L.smem, s);
    if (e != cudaSuccess) return fail(LS_ERR_CUDA, "propagation launch (TPW=%d W=%d KQ=%d): %s", L.k->tpw, L.k->w, L.k->kq,
                                      cudaGetErrorString(e));
  }
  return LS_OK;
}

int check_ctx(const ls_ctx* c) {
  if (!c) return fail(LS_ERR_ARG, "null context");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(LS_ERR_CUDA, "cudaSetDevice(%d) failed", c->device);
  return LS_OK;
}

int init_ctx_common(ls_ctx* c) {
  CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  // doubled rows: 2N bits per locus plus room for a lane's funnel-shift overrun
  c->rw2 = lsk::round_up((2 * c->N + 31) / 32 + 6, 4);
  int rc = dev_alloc(c, (void**)&c->bits2, sizeof(uint32_t) * (size_t)c->L * c->rw2);
  if (rc) return rc;
  {
    const long long n = (long long)c->L * c->rw2;
    lsk::double_rows_kernel<<<(unsigned)((n + 255) / 256), 256>>>(c->bits, c->row_words, c->N, c->L, c->bits2, c->rw2);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaDeviceSynchronize());
  }
  rc = dev_alloc(c, (void**)&c->err, sizeof(int));
  if (rc) return rc;
  CUDA_TRY(cudaMemset(c->err, 0, sizeof(int)));
  rc = dev_alloc(c, (void**)&c->logs_scratch, sizeof(double) * c->N);
  if (rc) return rc;
  return dev_alloc(c, (void**)&c->status_scratch, sizeof(uint32_t) * c->N);
}

void free_ctx(ls_ctx* c) {
  if (!c) return;
  cudaFree(c->bits);
  cudaFree(c->bits2);
  cudaFree(c->omr);
  cudaFree(c->rr_f);
  cudaFree(c->rr_b);
  cudaFree(c->thm);
  cudaFree(c->thx);
  cudaFree(c->Pi);
  cudaFree(c->logs_scratch);
  cudaFree(c->status_scratch);
  cudaFree(c->err);
  cudaFree(c->dscratch);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  if (c->side) cudaStreamDestroy(c->side);
  delete c;
}

int read_err_word(ls_ctx* c, cudaStream_t s) {
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (h) {
    cudaMemsetAsync(c->err, 0, sizeof(int), s);
    return fail(LS_ERR_DEVICE, "a device wait for staged haplotype rows ran out of time");
  }
  return LS_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// =============================================================================================
int ls_fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int ls_dev_alloc(void** p, size_t bytes) { return dev_alloc(nullptr, p, bytes); }

extern "C" {

const char* ls_version(void) {
  return "libls 0.1 for sm_103a: LS all-vs-all forward/backward (FP32 f32x2 tiles, TMA-staged rows), "
         "posterior, distance";
}

const char* ls_last_error(void) { return g_err.c_str(); }

int ls_create(ls_ctx** out, const uint8_t* haps, int32_t N, int32_t L) {
  if (!out || !haps) return fail(LS_ERR_ARG, "null pointer");
  if (N < 2 || L < 1) return fail(LS_ERR_ARG, "need N >= 2 and L >= 1 (got N=%d, L=%d)", N, L);
  ls_ctx* c = new ls_ctx;
  *out = nullptr;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return fail(LS_ERR_CUDA, "no CUDA device");
  }
  c->N = N;
  c->L = L;
  c->row_words = lsk::round_up((N + 31) / 32 + 1, 4);
  int rc = dev_alloc(c, (void**)&c->bits, sizeof(uint32_t) * (size_t)L * c->row_words);
  if (rc) { free_ctx(c); return rc; }
  uint8_t* tmp = nullptr;
  rc = dev_alloc(nullptr, (void**)&tmp, (size_t)N * L);
  if (rc) { free_ctx(c); return rc; }
  cudaError_t e = cudaMemset(c->bits, 0, sizeof(uint32_t) * (size_t)L * c->row_words);
  if (e == cudaSuccess) e = cudaMemcpy(tmp, haps, (size_t)N * L, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const long long threads = (long long)((N + 31) / 32) * L * 32;
    lsk::pack_kernel<<<(unsigned)((threads + 255) / 256), 256>>>(tmp, N, L, c->row_words, c->bits);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(tmp);
  if (e != cudaSuccess) { free_ctx(c); return fail(LS_ERR_CUDA, "packing haplotypes: %s", cudaGetErrorString(e)); }
  rc = init_ctx_common(c);
  if (rc) { free_ctx(c); return rc; }
  *out = c;
  return LS_OK;
}

int ls_create_packed(ls_ctx** out, const uint32_t* packed, int32_t N, int32_t L, int32_t row_words) {
  if (!out || !packed) return fail(LS_ERR_ARG, "null pointer");
  if (N < 2 || L < 1 || row_words < (N + 31) / 32) return fail(LS_ERR_ARG, "bad sizes N=%d L=%d row_words=%d", N, L, row_words);
  ls_ctx* c = new ls_ctx;
  *out = nullptr;
  cudaGetDevice(&c->device);
  c->N = N;
  c->L = L;
  c->row_words = lsk::round_up((N + 31) / 32 + 1, 4);
  int rc = dev_alloc(c, (void**)&c->bits, sizeof(uint32_t) * (size_t)L * c->row_words);
  if (rc) { free_ctx(c); return rc; }
  const int nw = (N + 31) / 32;
  cudaError_t e = cudaMemset(c->bits, 0, sizeof(uint32_t) * (size_t)L * c->row_words);
  if (e == cudaSuccess)
    e = cudaMemcpy2D(c->bits, sizeof(uint32_t) * c->row_words, packed, sizeof(uint32_t) * row_words, sizeof(uint32_t) * nw, L,
                     cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess && (N & 31)) {
    // clear the bits beyond N in the last word of every row
    std::vector<uint32_t> col(L);
    e = cudaMemcpy2D(col.data(), 4, c->bits + nw - 1, sizeof(uint32_t) * c->row_words, 4, L, cudaMemcpyDeviceToHost);
    for (auto& w : col) w &= (1u << (N & 31)) - 1u;
    if (e == cudaSuccess)
      e = cudaMemcpy2D(c->bits + nw - 1, sizeof(uint32_t) * c->row_words, col.data(), 4, 4, L, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) { free_ctx(c); return fail(LS_ERR_CUDA, "copying packed haplotypes: %s", cudaGetErrorString(e)); }
  rc = init_ctx_common(c);
  if (rc) { free_ctx(c); return rc; }
  *out = c;
  return LS_OK;
}

int ls_destroy(ls_ctx* ctx) {
  if (!ctx) return fail(LS_ERR_ARG, "null context");
  if (ctx->ntables) return fail(LS_ERR_STATE, "%d tables still alive", ctx->ntables);
  cudaSetDevice(ctx->device);
  free_ctx(ctx);
  return LS_OK;
}

int ls_info(const ls_ctx* ctx, int32_t* N, int32_t* L, int32_t* row_words, size_t* device_bytes) {
  if (!ctx) return fail(LS_ERR_ARG, "null context");
  if (N) *N = ctx->N;
  if (L) *L = ctx->L;
  if (row_words) *row_words = ctx->row_words;
  if (device_bytes) *device_bytes = ctx->bytes;
  return LS_OK;
}

int ls_query(const ls_ctx* ctx, const int32_t* loci, int32_t nl, const int32_t* haps, int32_t nh, uint8_t* out) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (nl < 0 || nh < 0 || (nl && !loci) || (nh && !haps) || (nl && nh && !out)) return fail(LS_ERR_ARG, "bad query arguments");
  for (int b = 0; b < nh; ++b)
    if (haps[b] < 0 || haps[b] >= ctx->N) return fail(LS_ERR_ARG, "haplotype %d out of range", haps[b]);
  std::vector<uint32_t> rowbuf(ctx->row_words);
  for (int a = 0; a < nl; ++a) {
    if (loci[a] < 0 || loci[a] >= ctx->L) return fail(LS_ERR_ARG, "locus %d out of range", loci[a]);
    CUDA_TRY(cudaMemcpy(rowbuf.data(), ctx->bits + (size_t)loci[a] * ctx->row_words, sizeof(uint32_t) * ctx->row_words,
                        cudaMemcpyDeviceToHost));
    for (int b = 0; b < nh; ++b) out[(size_t)a * nh + b] = (rowbuf[haps[b] >> 5] >> (haps[b] & 31)) & 1u;
  }
  return LS_OK;
}

int ls_export_packed(const ls_ctx* ctx, uint32_t* out) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (!out) return fail(LS_ERR_ARG, "null output");
  CUDA_TRY(cudaMemcpy(out, ctx->bits, sizeof(uint32_t) * (size_t)ctx->L * ctx->row_words, cudaMemcpyDeviceToHost));
  return LS_OK;
}

int ls_calc_rho(const double* m, int32_t n, double Ne, double gamma, double* rho_out) {
  if (n < 0 || (n && (!m || !rho_out))) return fail(LS_ERR_ARG, "bad arguments");
  if (!(Ne >= 0.0) || !std::isfinite(Ne) || !(gamma > 0.0) || !std::isfinite(gamma))
    return fail(LS_ERR_ARG, "need Ne >= 0 and gamma > 0");
  for (int k = 0; k < n; ++k) {
    if (!(m[k] >= 0.0) || !std::isfinite(m[k])) return fail(LS_ERR_ARG, "genetic distance m[%d] = %g is not >= 0", k, m[k]);
    rho_out[k] = -std::expm1(-Ne * std::pow(m[k], gamma));  // Eq. rho
  }
  return LS_OK;
}

int ls_set_prior_format(ls_ctx* ctx, int32_t format) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (format != LS_PRIOR_FP32 && format != LS_PRIOR_BF16) return fail(LS_ERR_ARG, "unknown prior format %d", format);
  ctx->prior_bf16 = format == LS_PRIOR_BF16 ? 1 : 0;
  return LS_OK;
}

int ls_set_params(ls_ctx* ctx, const double* rho, const double* mu, int32_t mu_len, const float* Pi, uint64_t* hash_out) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  const int N = ctx->N, L = ctx->L;
  if ((L > 1 && !rho) || !mu) return fail(LS_ERR_ARG, "null rho or mu");
  if (mu_len != 1 && mu_len != L) return fail(LS_ERR_ARG, "mu must have length 1 or L=%d (got %d)", L, mu_len);
  for (int l = 0; l + 1 < L; ++l)
    if (!(rho[l] >= 0.0 && rho[l] <= 1.0)) return fail(LS_ERR_ARG, "rho[%d] = %g is outside [0, 1]", l, rho[l]);
  for (int l = 0; l < mu_len; ++l)
    if (!(mu[l] >= 0.0 && mu[l] <= 1.0)) return fail(LS_ERR_ARG, "mu[%d] = %g is outside [0, 1]", l, mu[l]);
  uint64_t h = 1469598103934665603ull;
  h = fnv1a(h, &N, sizeof N);
  h = fnv1a(h, &L, sizeof L);
  if (L > 1) h = fnv1a(h, rho, sizeof(double) * (L - 1));
  h = fnv1a(h, &mu_len, sizeof mu_len);
  h = fnv1a(h, mu, sizeof(double) * mu_len);
  if (Pi) {
    // validated and fingerprinted on the GPU (one CTA per row); the host reads three words per row
    if (!is_device_ptr(Pi)) return fail(LS_ERR_ARG, "Pi must be device memory");
    void* chk = nullptr;
    const size_t bad_bytes = (((size_t)N * sizeof(int) + 7) / 8) * 8;  // the doubles start 8-byte aligned
    if ((rc = dev_alloc(nullptr, &chk, bad_bytes + (size_t)N * (sizeof(double) + sizeof(uint64_t))))) return rc;
    int* bad = static_cast<int*>(chk);
    double* sums = reinterpret_cast<double*>(static_cast<char*>(chk) + bad_bytes);
    unsigned long long* hs = reinterpret_cast<unsigned long long*>(sums + N);
    std::vector<int> bh(N);
    std::vector<double> sh(N);
    std::vector<unsigned long long> hh(N);
    lsk::prior_check_kernel<<<N, 256>>>(Pi, N, bad, sums, hs);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(bh.data(), bad, sizeof(int) * N, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(sh.data(), sums, sizeof(double) * N, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hh.data(), hs, sizeof(unsigned long long) * N, cudaMemcpyDeviceToHost);
    cudaFree(chk);
    if (e != cudaSuccess) return fail(LS_ERR_CUDA, "checking the prior: %s", cudaGetErrorString(e));
    for (int i = 0; i < N; ++i) {
      if (bh[i] & 1) return fail(LS_ERR_ARG, "prior row %d holds a negative or non-finite entry", i);
      if (bh[i] & 2) return fail(LS_ERR_ARG, "Pi[%d][%d] must be 0 (Sec. 2.1)", i, i);
      if (std::fabs(sh[i] - 1.0) > 1e-5) return fail(LS_ERR_ARG, "prior row %d sums to %.9g, not 1", i, sh[i]);
    }
    h = fnv1a(h, hh.data(), sizeof(unsigned long long) * hh.size());
    h = fnv1a(h, &ctx->prior_bf16, sizeof ctx->prior_bf16);
  }
  // per-locus FP32 constants, rounded once from double
  std::vector<float> omr(std::max(L - 1, 1)), rrf(std::max(L - 1, 1)), rrb(std::max(L - 1, 1)), thm(L), thx(L);
  const double pi_u = 1.0 / (double)(N - 1);
  for (int l = 0; l + 1 < L; ++l) {
    omr[l] = (float)(1.0 - rho[l]);
    rrf[l] = (float)(rho[l] * pi_u);
    rrb[l] = (float)rho[l];
  }
  for (int l = 0; l < L; ++l) {
    const double m = mu[mu_len == 1 ? 0 : l];
    thm[l] = (float)(1.0 - m);  // App. A.3: (1-H)(1-2mu)+mu with H = 0
    thx[l] = (float)m;          // and with H = 1
  }
  auto upload = [&](float*& dst, const std::vector<float>& v) -> int {
    if (!dst) {
      int r2 = dev_alloc(ctx, (void**)&dst, sizeof(float) * v.size());
      if (r2) return r2;
    }
    CUDA_TRY(cudaMemcpy(dst, v.data(), sizeof(float) * v.size(), cudaMemcpyHostToDevice));
    return LS_OK;
  };
  if ((rc = upload(ctx->omr, omr)) || (rc = upload(ctx->rr_f, rrf)) || (rc = upload(ctx->rr_b, rrb)) ||
      (rc = upload(ctx->thm, thm)) || (rc = upload(ctx->thx, thx)))
    return rc;
  if (Pi) {
    if (!ctx->Pi && (rc = dev_alloc(ctx, (void**)&ctx->Pi, sizeof(float) * (size_t)N * N))) return rc;
    CUDA_TRY(cudaMemcpy(ctx->Pi, Pi, sizeof(float) * (size_t)N * N, cudaMemcpyDeviceToDevice));
    if (ctx->prior_bf16) {
      const long long n = (long long)N * N;
      lsk::prior_bf16_kernel<<<(unsigned)((n + 255) / 256), 256>>>(ctx->Pi, n);
      CUDA_TRY(cudaGetLastError());
      CUDA_TRY(cudaDeviceSynchronize());
    }
  } else if (ctx->Pi) {
    cudaFree(ctx->Pi);
    ctx->bytes -= sizeof(float) * (size_t)N * N;
    ctx->Pi = nullptr;
  }
  ctx->pi_u = (float)pi_u;
  ctx->mu_vec = mu_len > 1 ? 1 : 0;
  ctx->rho_h.assign(rho, rho + std::max(L - 1, 0));
  ctx->mu_h.assign(mu, mu + mu_len);
  ctx->hash = h;
  ctx->have_params = true;
  if (hash_out) *hash_out = h;
  return LS_OK;
}

int ls_table_create(ls_ctx* ctx, int32_t kind, int32_t t_from, int32_t t_to, ls_table** out) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (!out) return fail(LS_ERR_ARG, "null output");
  if (kind != LS_FWD && kind != LS_BWD) return fail(LS_ERR_ARG, "kind must be LS_FWD or LS_BWD");
  if (!(0 <= t_from && t_from < t_to && t_to <= ctx->N)) return fail(LS_ERR_ARG, "bad target range [%d, %d)", t_from, t_to);
  if (!ctx->have_params) return fail(LS_ERR_STATE, "parameters not set");
  ls_table* t = new ls_table;
  t->ctx = ctx;
  t->kind = kind;
  t->t_from = t_from;
  t->t_to = t_to;
  const size_t T = (size_t)(t_to - t_from);
  if ((rc = dev_alloc(nullptr, (void**)&t->state, sizeof(float) * T * ctx->N)) ||
      (rc = dev_alloc(nullptr, (void**)&t->logs, sizeof(double) * T))) {
    cudaFree(t->state);
    delete t;
    return rc;
  }
  cudaMemset(t->state, 0, sizeof(float) * T * ctx->N);
  cudaMemset(t->logs, 0, sizeof(double) * T);
  ctx->ntables++;
  *out = t;
  return LS_OK;
}

int ls_table_destroy(ls_table* t) {
  if (!t) return fail(LS_ERR_ARG, "null table");
  cudaSetDevice(t->ctx->device);
  cudaFree(t->state);
  cudaFree(t->logs);
  t->ctx->ntables--;
  delete t;
  return LS_OK;
}

int ls_table_copy(ls_table* dst, const ls_table* src, ls_stream_t stream) {
  if (!dst || !src) return fail(LS_ERR_ARG, "null table");
  if (dst->ctx != src->ctx || dst->kind != src->kind || dst->t_from != src->t_from || dst->t_to != src->t_to)
    return fail(LS_ERR_RANGE, "tables differ in context, kind or target range");
  cudaSetDevice(dst->ctx->device);
  const size_t T = (size_t)(src->t_to - src->t_from);
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(dst->state, src->state, sizeof(float) * T * src->ctx->N, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(dst->logs, src->logs, sizeof(double) * T, cudaMemcpyDeviceToDevice, s));
  dst->locus = src->locus;
  dst->hash = src->hash;
  return LS_OK;
}

int ls_table_reset(ls_table* t) {
  if (!t) return fail(LS_ERR_ARG, "null table");
  t->locus = -1;
  t->hash = 0;
  return LS_OK;
}

int ls_table_info(const ls_table* t, int32_t* kind, int32_t* locus, int32_t* t_from, int32_t* t_to, uint64_t* hash) {
  if (!t) return fail(LS_ERR_ARG, "null table");
  if (kind) *kind = t->kind;
  if (locus) *locus = t->locus;
  if (t_from) *t_from = t->t_from;
  if (t_to) *t_to = t->t_to;
  if (hash) *hash = t->hash;
  return LS_OK;
}

int ls_table_read(const ls_table* t, float* state, double* logscale, ls_stream_t stream) {
  if (!t) return fail(LS_ERR_ARG, "null table");
  cudaSetDevice(t->ctx->device);
  const size_t T = (size_t)(t->t_to - t->t_from);
  cudaStream_t s = (cudaStream_t)stream;
  if (state) CUDA_TRY(cudaMemcpyAsync(state, t->state, sizeof(float) * T * t->ctx->N, cudaMemcpyDeviceToDevice, s));
  if (logscale) CUDA_TRY(cudaMemcpyAsync(logscale, t->logs, sizeof(double) * T, cudaMemcpyDeviceToDevice, s));
  return LS_OK;
}

static int propagate(ls_ctx* ctx, ls_table* tb, int dir, int32_t to, const int32_t* store, int32_t n_store, float* out,
                     uint32_t* status, ls_stream_t stream) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (!tb || tb->ctx != ctx) return fail(LS_ERR_ARG, "table does not belong to this context");
  if (tb->kind != (dir == 0 ? LS_FWD : LS_BWD)) return fail(LS_ERR_ARG, "wrong table kind for this direction");
  if (!ctx->have_params) return fail(LS_ERR_STATE, "parameters not set");
  const int L = ctx->L;
  if (to < 0 || to >= L) return fail(LS_ERR_ARG, "locus %d out of range [0, %d)", to, L);
  const bool init = tb->locus < 0;
  if (!init && tb->hash != ctx->hash) return fail(LS_ERR_PARAM_MISMATCH, "table was propagated under another parameter set");
  const int cur = tb->locus;
  if (!init && (dir == 0 ? to < cur : to > cur))
    return fail(LS_ERR_DIRECTION, "%s cannot move from locus %d to %d", dir == 0 ? "forward" : "backward", cur, to);
  if (n_store < 0 || (n_store > 0 && (!store || !out))) return fail(LS_ERR_ARG, "bad store arguments");
  // store loci: strictly monotone inside the range this call covers
  const int lo = dir == 0 ? (init ? 0 : cur + 1) : to;
  const int hi = dir == 0 ? to : (init ? L - 1 : cur - 1);
  for (int k = 0; k < n_store; ++k) {
    if (store[k] < lo || store[k] > hi) return fail(LS_ERR_ARG, "store locus %d outside [%d, %d]", store[k], lo, hi);
    if (k && (dir == 0 ? store[k] <= store[k - 1] : store[k] >= store[k - 1]))
      return fail(LS_ERR_ARG, "store loci must be strictly %s", dir == 0 ? "increasing" : "decreasing");
  }
  if (!init && to == cur) return LS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int T = tb->t_to - tb->t_from;
  int pos = init ? -1 : cur;  // locus the table state is at
  int k0 = 0;
  bool first = true;
  while (true) {
    const int k1 = std::min(n_store, k0 + lsk::kMaxStore);
    const int seg_end = (k1 < n_store) ? store[k1 - 1] : to;
    lsk::PropParams p;
    base_params(ctx, p, dir);
    const bool seg_init = first && init;
    if (dir == 0) {
      p.l_first = seg_init ? 0 : pos + 1;
      p.n_steps = seg_end - p.l_first + 1;
    } else {
      p.l_first = seg_init ? L - 1 : pos;  // a resumed backward step 0 re-applies theta at pos
      p.n_steps = p.l_first - seg_end + 1;
    }
    p.init = seg_init ? 1 : 0;
    p.tab_t0 = tb->t_from;
    p.state = tb->state;
    p.logs = tb->logs;
    p.status = status;
    p.state_rows = T;
    p.load_state = seg_init ? 0 : 1;
    p.save_state = 1;
    p.n_store = k1 - k0;
    for (int k = k0; k < k1; ++k) {
      p.store_loci[k - k0] = store[k];
      p.store_slot[k - k0] = k;
    }
    p.store = out;
    if (p.n_steps > 0) {
      rc = run_launches(ctx, p, tb->t_from, T, s);
      if (rc) return rc;
    }
    pos = seg_end;
    first = false;
    k0 = k1;
    if (k1 >= n_store) break;
  }
  tb->locus = to;
  tb->hash = ctx->hash;
  return LS_OK;
}

int ls_forward(ls_ctx* ctx, ls_table* fwd, int32_t to_locus, const int32_t* store_loci, int32_t n_store, float* alpha_out,
               uint32_t* status_out, ls_stream_t stream) {
  return propagate(ctx, fwd, 0, to_locus, store_loci, n_store, alpha_out, status_out, stream);
}

int ls_backward(ls_ctx* ctx, ls_table* bck, int32_t to_locus, const int32_t* store_loci, int32_t n_store, float* beta_out,
                uint32_t* status_out, ls_stream_t stream) {
  return propagate(ctx, bck, 1, to_locus, store_loci, n_store, beta_out, status_out, stream);
}

// ---- forward checkpoints (recursive-bisection loci) and replay --------------------------------
static void ckpt_free(ls_ckpt* ck) {
  cudaFree(ck->data);
  cudaFree(ck->scale);
  cudaFree(ck->logs);
  delete ck;
}

int ls_checkpoints(ls_ctx* ctx, ls_table* fwd, int32_t a, int32_t b, int32_t dtype, ls_ckpt** out,
                   uint32_t* status_out, ls_stream_t stream) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (!out) return fail(LS_ERR_ARG, "null output");
  if (!fwd || fwd->ctx != ctx || fwd->kind != LS_FWD) return fail(LS_ERR_ARG, "need a forward table of this context");
  if (dtype != LS_CKPT_F32 && dtype != LS_CKPT_F16) return fail(LS_ERR_ARG, "dtype must be LS_CKPT_F32 or LS_CKPT_F16");
  if (!ctx->have_params) return fail(LS_ERR_STATE, "parameters not set");
  if (!(0 <= a && a <= b && b < ctx->L)) return fail(LS_ERR_ARG, "bad locus range [%d, %d]", a, b);
  if (fwd->locus > a) return fail(LS_ERR_DIRECTION, "forward table at locus %d is beyond a = %d", fwd->locus, a);
  if (fwd->locus >= 0 && fwd->hash != ctx->hash)
    return fail(LS_ERR_PARAM_MISMATCH, "table was propagated under another parameter set");
  // K = ceil(log2(b - a + 1)) snapshots (one when a == b): c_0 = a, c_k = b - floor((b - a) / 2^k)
  int K = 1;
  while ((1ll << K) < (long long)(b - a + 1)) ++K;
  ls_ckpt* ck = new ls_ckpt;
  ck->ctx = ctx;
  ck->dtype = dtype;
  ck->t_from = fwd->t_from;
  ck->t_to = fwd->t_to;
  ck->loci.push_back(a);
  for (int k = 1; k < K; ++k) ck->loci.push_back(b - (int)((long long)(b - a) >> k));
  const size_t T = (size_t)(fwd->t_to - fwd->t_from), N = (size_t)ctx->N;
  const size_t esz = dtype == LS_CKPT_F16 ? 2 : 4;
  if ((rc = dev_alloc(nullptr, &ck->data, (size_t)K * T * N * esz)) ||
      (rc = dev_alloc(nullptr, (void**)&ck->logs, sizeof(double) * K * T)) ||
      (dtype == LS_CKPT_F16 && (rc = dev_alloc(nullptr, (void**)&ck->scale, sizeof(float) * K * T)))) {
    ckpt_free(ck);
    return rc;
  }
  ck->bytes = (size_t)K * T * (N * esz + 8 + (dtype == LS_CKPT_F16 ? 4 : 0));
  cudaStream_t s = (cudaStream_t)stream;
  for (int k = 0; k < K; ++k) {
    if ((rc = propagate(ctx, fwd, 0, ck->loci[k], nullptr, 0, nullptr, status_out, stream))) {
      ckpt_free(ck);
      return rc;
    }
    if (dtype == LS_CKPT_F32) {
      CUDA_TRY(cudaMemcpyAsync(static_cast<float*>(ck->data) + k * T * N, fwd->state, sizeof(float) * T * N,
                               cudaMemcpyDeviceToDevice, s));
    } else {
      lsk::ckpt_encode_f16_kernel<<<(unsigned)T, 256, 0, s>>>(fwd->state, (int)N, static_cast<__half*>(ck->data) + k * T * N,
                                                              ck->scale + k * T);
      CUDA_TRY(cudaGetLastError());
    }
    CUDA_TRY(cudaMemcpyAsync(ck->logs + k * T, fwd->logs, sizeof(double) * T, cudaMemcpyDeviceToDevice, s));
  }
  if ((rc = propagate(ctx, fwd, 0, b, nullptr, 0, nullptr, status_out, stream))) {
    ckpt_free(ck);
    return rc;
  }
  ck->hash = ctx->hash;
  *out = ck;
  return LS_OK;
}

int ls_ckpt_info(const ls_ckpt* ck, int32_t* n, int32_t* loci, int32_t* dtype, int32_t* t_from, int32_t* t_to,
                 size_t* device_bytes) {
  if (!ck) return fail(LS_ERR_ARG, "null checkpoint set");
  if (n) *n = (int32_t)ck->loci.size();
  if (loci)
    for (size_t k = 0; k < ck->loci.size(); ++k) loci[k] = ck->loci[k];
  if (dtype) *dtype = ck->dtype;
  if (t_from) *t_from = ck->t_from;
  if (t_to) *t_to = ck->t_to;
  if (device_bytes) *device_bytes = ck->bytes;
  return LS_OK;
}

static int ckpt_decode(const ls_ckpt* ck, int k, float* alpha, double* logs, cudaStream_t s) {
  const size_t T = (size_t)(ck->t_to - ck->t_from), N = (size_t)ck->ctx->N;
  if (alpha) {
    if (ck->dtype == LS_CKPT_F32) {
      CUDA_TRY(cudaMemcpyAsync(alpha, static_cast<const float*>(ck->data) + k * T * N, sizeof(float) * T * N,
                               cudaMemcpyDeviceToDevice, s));
    } else {
      lsk::ckpt_decode_f16_kernel<<<(unsigned)T, 256, 0, s>>>(static_cast<const __half*>(ck->data) + k * T * N,
                                                              ck->scale + k * T, (int)N, alpha);
      CUDA_TRY(cudaGetLastError());
    }
  }
  if (logs) CUDA_TRY(cudaMemcpyAsync(logs, ck->logs + k * T, sizeof(double) * T, cudaMemcpyDeviceToDevice, s));
  return LS_OK;
}

int ls_ckpt_read(const ls_ckpt* ck, int32_t k, float* alpha_out, double* logF_out, ls_stream_t stream) {
  if (!ck) return fail(LS_ERR_ARG, "null checkpoint set");
  if (k < 0 || k >= (int)ck->loci.size()) return fail(LS_ERR_ARG, "snapshot %d out of range [0, %zu)", k, ck->loci.size());
  cudaSetDevice(ck->ctx->device);
  return ckpt_decode(ck, k, alpha_out, logF_out, (cudaStream_t)stream);
}

int ls_ckpt_replay(ls_ctx* ctx, const ls_ckpt* ck, ls_table* fwd, int32_t locus, uint32_t* status_out,
                   ls_stream_t stream) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (!ck || ck->ctx != ctx) return fail(LS_ERR_ARG, "checkpoints do not belong to this context");
  if (!fwd || fwd->ctx != ctx || fwd->kind != LS_FWD) return fail(LS_ERR_ARG, "need a forward table of this context");
  if (fwd->t_from != ck->t_from || fwd->t_to != ck->t_to) return fail(LS_ERR_RANGE, "table and checkpoints cover different targets");
  if (ck->hash != ctx->hash) return fail(LS_ERR_PARAM_MISMATCH, "checkpoints were taken under another parameter set");
  if (locus < ck->loci[0] || locus >= ctx->L)
    return fail(LS_ERR_ARG, "locus %d outside [%d, %d)", locus, ck->loci[0], ctx->L);
  int k = (int)ck->loci.size() - 1;
  while (ck->loci[k] > locus) --k;
  if ((rc = ckpt_decode(ck, k, fwd->state, fwd->logs, (cudaStream_t)stream))) return rc;
  fwd->locus = ck->loci[k];
  fwd->hash = ck->hash;
  return propagate(ctx, fwd, 0, locus, nullptr, 0, nullptr, status_out, stream);
}

int ls_ckpt_destroy(ls_ckpt* ck) {
  if (!ck) return fail(LS_ERR_ARG, "null checkpoint set");
  cudaSetDevice(ck->ctx->device);
  ckpt_free(ck);
  return LS_OK;
}

static int check_pair(ls_ctx* ctx, const ls_table* fwd, const ls_table* bck) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (!fwd || !bck || fwd->ctx != ctx || bck->ctx != ctx) return fail(LS_ERR_ARG, "tables do not belong to this context");
  if (fwd->kind != LS_FWD || bck->kind != LS_BWD) return fail(LS_ERR_ARG, "need a forward and a backward table");
  if (fwd->t_from != bck->t_from || fwd->t_to != bck->t_to) return fail(LS_ERR_RANGE, "tables cover different targets");
  if (fwd->locus < 0 || bck->locus < 0) return fail(LS_ERR_STATE, "table not initialised");
  if (fwd->locus != bck->locus) return fail(LS_ERR_LOCUS_MISMATCH, "forward at locus %d, backward at %d", fwd->locus, bck->locus);
  if (fwd->hash != bck->hash) return fail(LS_ERR_PARAM_MISMATCH, "tables were propagated under different parameters");
  return LS_OK;
}

int ls_posterior(ls_ctx* ctx, const ls_table* fwd, const ls_table* bck, float* p_out, ls_stream_t stream) {
  int rc = check_pair(ctx, fwd, bck);
  if (rc) return rc;
  if (!p_out) return fail(LS_ERR_ARG, "null output");
  const int T = fwd->t_to - fwd->t_from;
  lsk::posterior_kernel<<<T, 256, 0, (cudaStream_t)stream>>>(fwd->state, bck->state, ctx->N, fwd->t_from, 0, p_out);
  CUDA_TRY(cudaGetLastError());
  return LS_OK;
}

int ls_distance(ls_ctx* ctx, const ls_table* fwd, const ls_table* bck, float* d_out, ls_stream_t stream) {
  int rc = check_pair(ctx, fwd, bck);
  if (rc) return rc;
  if (!d_out) return fail(LS_ERR_ARG, "null output");
  if (fwd->t_from != 0 || fwd->t_to != ctx->N) return fail(LS_ERR_RANGE, "the distance matrix needs tables over all N targets");
  const int N = ctx->N;
  cudaStream_t s = (cudaStream_t)stream;
  lsk::posterior_kernel<<<N, 256, 0, s>>>(fwd->state, bck->state, N, 0, 1, d_out);
  CUDA_TRY(cudaGetLastError());
  const int nt = (N + 31) / 32;
  lsk::symmetrize_kernel<<<dim3(nt, nt, 1), dim3(32, 8), 0, s>>>(d_out, N);
  CUDA_TRY(cudaGetLastError());
  return LS_OK;
}

int ls_run_all(ls_ctx* ctx, const int32_t* decode_loci, int32_t D, float* d_out, double* pac_out, uint32_t* status_out,
               ls_stream_t stream) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (!ctx->have_params) return fail(LS_ERR_STATE, "parameters not set");
  const int N = ctx->N, L = ctx->L;
  if (D < 0 || (D > 0 && (!decode_loci || !d_out))) return fail(LS_ERR_ARG, "bad decode arguments");
  if (D > lsk::kMaxStore) return fail(LS_ERR_UNSUPPORTED, "at most %d decode loci per call", lsk::kMaxStore);
  for (int k = 0; k < D; ++k) {
    if (decode_loci[k] < 0 || decode_loci[k] >= L) return fail(LS_ERR_ARG, "decode locus %d out of range", decode_loci[k]);
    if (k && decode_loci[k] <= decode_loci[k - 1]) return fail(LS_ERR_ARG, "decode loci must be strictly increasing");
  }
  cudaStream_t s = (cudaStream_t)stream;
  const bool host_out = D > 0 && !is_device_ptr(d_out);
  float* dd = d_out;
  const size_t dbytes = sizeof(float) * (size_t)D * N * N;
  if (host_out) {
    if (ctx->dscratch_bytes < dbytes) {
      cudaFree(ctx->dscratch);
      ctx->bytes -= ctx->dscratch_bytes;
      ctx->dscratch = nullptr;
      ctx->dscratch_bytes = 0;
      if ((rc = dev_alloc(ctx, (void**)&ctx->dscratch, dbytes))) return rc;
      ctx->dscratch_bytes = dbytes;
    }
    dd = ctx->dscratch;
  }
  uint32_t* stat = ctx->status_scratch;
  CUDA_TRY(cudaMemsetAsync(stat, 0, sizeof(uint32_t) * N, s));
  const bool prof = ctx->profile;
  if (prof) CUDA_TRY(cudaEventRecord(ctx->ev[0], s));
  // forward over all loci: alpha at the decode loci goes straight into the output buffer
  lsk::PropParams p;
  base_params(ctx, p, 0);
  p.l_first = 0;
  p.n_steps = L;
  p.init = 1;
  p.tab_t0 = 0;
  p.state_rows = N;
  p.logs = ctx->logs_scratch;
  p.status = stat;
  p.n_store = D;
  for (int k = 0; k < D; ++k) {
    p.store_loci[k] = decode_loci[k];
    p.store_slot[k] = k;
  }
  p.store = dd;
  if ((rc = run_launches(ctx, p, 0, N, s, &ctx->launches[0]))) return rc;
  if (prof) CUDA_TRY(cudaEventRecord(ctx->ev[1], s));
  // backward over all loci: alpha * beta overwrites alpha at the decode loci
  base_params(ctx, p, 1);
  p.l_first = L - 1;
  p.n_steps = L;
  p.init = 1;
  p.tab_t0 = 0;
  p.state_rows = N;
  p.status = stat;
  p.n_store = D;
  for (int k = 0; k < D; ++k) {
    p.store_loci[k] = decode_loci[D - 1 - k];
    p.store_slot[k] = D - 1 - k;
  }
  p.alpha_dec = dd;
  if ((rc = run_launches(ctx, p, 0, N, s, &ctx->launches[1]))) return rc;
  if (prof) CUDA_TRY(cudaEventRecord(ctx->ev[2], s));
  ctx->launches[2] = ctx->launches[3] = 0;
  if (D > 0) {
    lsk::DecodeLoci dl;
    for (int k = 0; k < D; ++k) dl.l[k] = decode_loci[k];
    lsk::decode_kernel<<<dim3(N, D), 256, 0, s>>>(dd, N, ctx->bits, ctx->row_words, ctx->thm, ctx->thx, dl);
    CUDA_TRY(cudaGetLastError());
    ctx->launches[2] = 1;
  }
  if (prof) CUDA_TRY(cudaEventRecord(ctx->ev[3], s));
  if (D > 0) {
    const int nt = (N + 31) / 32;
    lsk::symmetrize_kernel<<<dim3(nt, nt, D), dim3(32, 8), 0, s>>>(dd, N);
    CUDA_TRY(cudaGetLastError());
    ctx->launches[3] = 1;
  }
  if (prof) {
    CUDA_TRY(cudaEventRecord(ctx->ev[4], s));
    ctx->profiled = true;
  }
  if (status_out) CUDA_TRY(cudaMemcpyAsync(status_out, stat, sizeof(uint32_t) * N, cudaMemcpyDeviceToDevice, s));
  const bool sync = host_out || pac_out;
  if (host_out) CUDA_TRY(cudaMemcpyAsync(d_out, dd, dbytes, cudaMemcpyDeviceToHost, s));
  if (!sync) return LS_OK;
  std::vector<double> lf(N);
  std::vector<uint32_t> sh(N);
  CUDA_TRY(cudaMemcpyAsync(lf.data(), ctx->logs_scratch, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(sh.data(), stat, sizeof(uint32_t) * N, cudaMemcpyDeviceToHost, s));
  if ((rc = read_err_word(ctx, s))) return rc;
  if (pac_out) {
    double pac = 0.0;
    for (int i = 0; i < N; ++i) pac += lf[i];  // PAC log-likelihood (Sec. 1), fixed order
    *pac_out = pac;
  }
  uint32_t any = 0;
  for (auto v : sh) any |= v;
  // total underflow is reported first: the NaNs it leaves behind also trip the overflow check
  if (any & 1u) return LS_WARN_UNDERFLOW;
  if (any & 2u) return LS_WARN_OVERFLOW;
  return LS_OK;
}

// ---- adjoint: gradient of the PAC log-likelihood ------------------------------------------------
// Fisher identity: the score is the posterior expectation of the complete-data score.  With the
// recombination event B_m of interval m (probability rho_m, Eq. transition) and the mismatch
// indicator H_l (emission mu, App. A.3), per target
//   d log P / d log rho_m = (E[B_m] - rho_m) / (1 - rho_m),
//   d log P / d log mu    = sum_l (E[H_l] - mu_l) / (1 - mu_l)        (donors j != i, sum_j p_j = 1).
// E[sum_{m in I_k} B_m / (1 - rho_m)] for each group I_k of intervals comes from one forward
// statistic pass (ST 1, restarted per group, alpha and w stored at the group's end locus) and one
// backward pass (beta at those loci); E[sum_l H_l / (1 - mu_l)] from a second forward pass (ST 2)
// read at the last locus, where beta = 1.
}  // extern "C"

namespace {
struct StatPick {
  const PropKernelInfo* k = nullptr;
  int smem = 0;
};

int pick_stat(ls_ctx* c, StatPick* out) {
  double bc = 1e300;
  for (const auto& k : registry()) {
    if (k.st != 1 || !k.serves(c->N)) continue;
    const int smem = k.smem_bytes(c->rw2);
    if (smem > 227 * 1024) continue;
    bool ok = true;
    for (int d = 0; d < 2 && ok; ++d)
      if (cudaFuncSetAttribute(k.func[d], cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) ok = false;
    int nb = 0;
    if (ok && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k.func[1], k.w * 32, smem) != cudaSuccess || nb < 1))
      ok = false;
    if (!ok) {
      cudaGetLastError();
      continue;
    }
    const double cc = cost_of(Cand{&k, smem, nb}, c->N, c->num_sms);
    if (cc < bc) {
      bc = cc;
      out->k = &k;
      out->smem = smem;
    }
  }
  if (!out->k) return fail(LS_ERR_UNSUPPORTED, "no compiled statistic-pass variant serves N=%d", c->N);
  return LS_OK;
}

struct DevBufs {
  std::vector<void*> v;
  ~DevBufs() {
    for (void* p : v) cudaFree(p);
  }
  template <class T>
  int get(T** p, size_t n) {
    int rc = dev_alloc(nullptr, (void**)p, sizeof(T) * std::max<size_t>(n, 1));
    if (!rc) v.push_back(*p);
    return rc;
  }
};
// Device scratch ceiling of ls_pac_grad (targets are processed in blocks that fit it): 16 GiB, or
// the environment variable LS_GRAD_BUDGET_MB when it is set to a positive number of MiB.
size_t grad_budget() {
  const char* e = getenv("LS_GRAD_BUDGET_MB");
  const long long mb = e ? atoll(e) : 0;
  return mb > 0 ? (size_t)mb << 20 : (size_t)16 << 30;
}

// One block of targets [b0, b0 + TB) of ls_pac_grad: the two forward statistic passes and the
// backward pass, then the per-group sums of the block (sums [G + 2]: G recombination statistics,
// the mismatch statistic, the log-likelihood) and the status words of the block in stat.
int grad_block(ls_ctx* ctx, const StatPick& sp, int b0, int TB, int L, int G, const std::vector<int>& ge,
               const std::vector<float>& eta, const float* d_gam, const float* d_eta, const uint8_t* d_rst, float* A,
               float* Wst, float* B, float* xst, float* wst, double* logF, double* EM, double* Rg, double* sums,
               uint32_t* stat, cudaStream_t s) {
  const int N = ctx->N;
  int rc = LS_OK;
  CUDA_TRY(cudaMemsetAsync(stat, 0, sizeof(uint32_t) * TB, s));
  const int grid = (TB + sp.k->tpw - 1) / sp.k->tpw;
  auto launch = [&](int which, lsk::PropParams& p) -> int {
    p.t_begin = b0;
    p.t_count = TB;
    cudaError_t e = sp.k->launch(which, p, grid, sp.smem, s);
    if (e != cudaSuccess) return fail(LS_ERR_CUDA, "statistic pass launch: %s", cudaGetErrorString(e));
    return LS_OK;
  };
  // forward statistic pass 1 (recombinations per group), alpha and w stored at the group ends,
  // in launches of at most kMaxStore stores that carry alpha and w between them
  {
    int k0 = 0, pos = -1;
    do {
      const int k1 = std::min(G, k0 + lsk::kMaxStore);
      const int seg_end = k1 < G ? ge[k1 - 1] : L - 1;
      lsk::PropParams p;
      base_params(ctx, p, 0);
      p.l_first = pos + 1;
      p.n_steps = seg_end - pos;
      p.init = pos < 0 ? 1 : 0;
      p.load_state = pos < 0 ? 0 : 1;
      p.save_state = 1;
      p.tab_t0 = b0;
      p.state_rows = TB;
      p.state = xst;
      p.wstate = wst;
      p.logs = logF;
      p.status = stat;
      p.gam = d_gam;
      p.reset = d_rst;
      p.n_store = k1 - k0;
      for (int k = k0; k < k1; ++k) {
        p.store_loci[k - k0] = ge[k];
        p.store_slot[k - k0] = k;
      }
      p.store = A;
      p.wstore = Wst;
      if ((rc = launch(0, p))) return rc;
      pos = seg_end;
      k0 = k1;
    } while (pos < L - 1);
  }
  // forward statistic pass 2 (mismatches), read at the last locus
  {
    lsk::PropParams p;
    base_params(ctx, p, 0);
    p.l_first = 0;
    p.n_steps = L;
    p.init = 1;
    p.tab_t0 = b0;
    p.state_rows = TB;
    p.eta = eta[0];
    p.eta_vec = ctx->mu_vec ? d_eta : nullptr;
    p.stat_out = EM;
    if ((rc = launch(1, p))) return rc;
  }
  // backward: beta at the group ends (decreasing), in launches of at most kMaxStore stores
  if (G > 0) {
    int k0 = 0, pos = L;  // stores are taken in the order e_{G-1}, ..., e_0
    do {
      const int k1 = std::min(G, k0 + lsk::kMaxStore);
      const int seg_end = ge[G - k1];  // the lowest store locus of this launch
      lsk::PropParams p;
      base_params(ctx, p, 1);
      p.l_first = pos == L ? L - 1 : pos;
      p.n_steps = p.l_first - seg_end + 1;
      p.init = pos == L ? 1 : 0;
      p.load_state = pos == L ? 0 : 1;
      p.save_state = 1;
      p.tab_t0 = b0;
      p.state_rows = TB;
      p.state = xst;
      p.n_store = k1 - k0;
      for (int k = k0; k < k1; ++k) {
        p.store_loci[k - k0] = ge[G - 1 - k];
        p.store_slot[k - k0] = G - 1 - k;
      }
      p.store = B;
      if ((rc = run_launches(ctx, p, b0, TB, s))) return rc;
      pos = seg_end;
      k0 = k1;
    } while (k0 < G);
    lsk::grad_dot_kernel<<<dim3(TB, G), 256, 0, s>>>(A, Wst, B, N, TB, Rg);
    CUDA_TRY(cudaGetLastError());
    lsk::sum_rows_kernel<<<G, 256, 0, s>>>(Rg, TB, sums);
    CUDA_TRY(cudaGetLastError());
  }
  lsk::sum_rows_kernel<<<1, 256, 0, s>>>(EM, TB, sums + G);
  CUDA_TRY(cudaGetLastError());
  lsk::sum_rows_kernel<<<1, 256, 0, s>>>(logF, TB, sums + G + 1);
  CUDA_TRY(cudaGetLastError());
  return LS_OK;
}
}  // namespace

extern "C" {

int ls_pac_grad(ls_ctx* ctx, int32_t t_from, int32_t t_to, const int32_t* interval_of, int32_t K, double* pac_out,
                double* dlogmu_out, double* dlogrho_out, ls_stream_t stream) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (!ctx->have_params) return fail(LS_ERR_STATE, "parameters not set");
  if (ctx->Pi) return fail(LS_ERR_UNSUPPORTED, "the adjoint supports the uniform prior only");
  const int N = ctx->N, L = ctx->L;
  if (!(0 <= t_from && t_from < t_to && t_to <= N)) return fail(LS_ERR_ARG, "bad target range [%d, %d)", t_from, t_to);
  if (K < 1 || (L > 1 && !interval_of)) return fail(LS_ERR_ARG, "need K >= 1 and interval_of[L-1]");
  for (int m = 0; m + 1 < L; ++m) {
    if (interval_of[m] < 0 || interval_of[m] >= K) return fail(LS_ERR_ARG, "interval_of[%d] = %d outside [0, %d)", m, interval_of[m], K);
    if (m && interval_of[m] < interval_of[m - 1]) return fail(LS_ERR_ARG, "interval_of must be nondecreasing");
    if (!(ctx->rho_h[m] < 1.0)) return fail(LS_ERR_ARG, "the gradient needs rho < 1 (rho[%d] = %g)", m, ctx->rho_h[m]);
  }
  for (double m : ctx->mu_h)
    if (!(m < 1.0)) return fail(LS_ERR_ARG, "the gradient needs mu < 1");
  StatPick sp;
  if ((rc = pick_stat(ctx, &sp))) return rc;
  const int T = t_to - t_from;
  cudaStream_t s = (cudaStream_t)stream;
  // groups with at least one interval; their end loci e_g (the locus after the group's last interval)
  std::vector<int> gk, ge;
  for (int m = 0; m + 1 < L; ++m) {
    if (m + 1 == L - 1 || interval_of[m + 1] != interval_of[m]) {
      gk.push_back(interval_of[m]);
      ge.push_back(m + 1);
    }
  }
  const int G = (int)gk.size();
  if (G > 65535) return fail(LS_ERR_UNSUPPORTED, "at most 65535 nonempty intervals");
  std::vector<float> gam(std::max(L - 1, 1), 1.0f), eta(L);
  std::vector<uint8_t> rst(std::max(L - 1, 1), 0);
  for (int m = 0; m + 1 < L; ++m) {
    gam[m] = (float)(1.0 / (1.0 - ctx->rho_h[m]));
    rst[m] = (m == 0 || interval_of[m] != interval_of[m - 1]) ? 1 : 0;
  }
  for (int l = 0; l < L; ++l) eta[l] = (float)(1.0 / (1.0 - ctx->mu_h[ctx->mu_h.size() > 1 ? l : 0]));
  // Targets are processed in blocks whose device scratch (alpha, w and beta at every group end, plus
  // the carried alpha and w: (3 G + 2) floats per target and donor) stays within kGradBudget bytes;
  // blocks are whole waves of the statistic kernel where possible.
  const size_t per_target = ((size_t)3 * G + 2) * (size_t)N * sizeof(float);
  int Tb = (int)std::min<size_t>((size_t)T, std::max<size_t>(1, grad_budget() / per_target));
  if (Tb < T) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sp.k->func[0], sp.k->w * 32, sp.smem);
    const int wave = std::max(1, nb) * ctx->num_sms * sp.k->tpw;
    if (Tb >= wave) Tb = (Tb / wave) * wave;
  }
  Tb = std::min(Tb, T);
  DevBufs db;
  float *d_gam, *d_eta, *A, *Wst, *B, *xst, *wst;
  uint8_t* d_rst;
  double *logF, *EM, *Rg, *sums;
  uint32_t* stat;
  const size_t TN = (size_t)Tb * N;
  if ((rc = db.get(&d_gam, gam.size())) || (rc = db.get(&d_eta, eta.size())) || (rc = db.get(&d_rst, rst.size())) ||
      (rc = db.get(&A, (size_t)G * TN)) || (rc = db.get(&Wst, (size_t)G * TN)) || (rc = db.get(&B, (size_t)G * TN)) ||
      (rc = db.get(&xst, TN)) || (rc = db.get(&wst, TN)) || (rc = db.get(&logF, Tb)) || (rc = db.get(&EM, Tb)) ||
      (rc = db.get(&Rg, (size_t)std::max(G, 1) * Tb)) || (rc = db.get(&sums, (size_t)G + 2)) || (rc = db.get(&stat, Tb)))
    return rc;
  CUDA_TRY(cudaMemcpyAsync(d_gam, gam.data(), sizeof(float) * gam.size(), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(d_eta, eta.data(), sizeof(float) * eta.size(), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(d_rst, rst.data(), rst.size(), cudaMemcpyHostToDevice, s));
  std::vector<double> hs(G + 2, 0.0), hb(G + 2);
  std::vector<uint32_t> sh(Tb);
  uint32_t any = 0;
  for (int b0 = t_from; b0 < t_to; b0 += Tb) {
    const int TB = std::min(Tb, t_to - b0);
    if ((rc = grad_block(ctx, sp, b0, TB, L, G, ge, eta, d_gam, d_eta, d_rst, A, Wst, B, xst, wst, logF, EM, Rg, sums,
                         stat, s)))
      return rc;
    CUDA_TRY(cudaMemcpyAsync(hb.data(), sums, sizeof(double) * (G + 2), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(sh.data(), stat, sizeof(uint32_t) * TB, cudaMemcpyDeviceToHost, s));
    if ((rc = read_err_word(ctx, s))) return rc;
    for (int g = 0; g < G + 2; ++g) hs[g] += hb[g];
    for (int r = 0; r < TB; ++r) any |= sh[r];
  }
  // constant terms of the scores, FP64 on the host
  if (dlogrho_out) {
    for (int k = 0; k < K; ++k) dlogrho_out[k] = 0.0;
    std::vector<double> cst(K, 0.0);
    for (int m = 0; m + 1 < L; ++m) cst[interval_of[m]] += ctx->rho_h[m] / (1.0 - ctx->rho_h[m]);
    for (int g = 0; g < G; ++g) dlogrho_out[gk[g]] = hs[g] - (double)T * cst[gk[g]];
  }
  if (dlogmu_out) {
    double cm = 0.0;
    for (int l = 0; l < L; ++l) {
      const double m = ctx->mu_h[ctx->mu_h.size() > 1 ? l : 0];
      cm += m / (1.0 - m);
    }
    *dlogmu_out = hs[G] - (double)T * cm;
  }
  if (pac_out) *pac_out = hs[G + 1];
  if (any & 1u) return LS_WARN_UNDERFLOW;
  if (any & 2u) return LS_WARN_OVERFLOW;
  return LS_OK;
}

// ---- sparse recursions over proposed donor sets, with dense fallback ---------------------------
}  // extern "C"

namespace {
// dense propagation of a list of targets (one target per CTA), for the fallback rows
int run_list(ls_ctx* c, lsk::PropParams p, const int* d_tlist, int nf, cudaStream_t s) {
  Cand cs[kMaxCand], one[kMaxCand];
  int nc = 0, no = 0;
  int rc = candidates(c, cs, &nc);
  if (rc) return rc;
  for (int i = 0; i < nc; ++i)
    if (cs[i].k->tpw == 1) one[no++] = cs[i];
  if (no == 0) return fail(LS_ERR_UNSUPPORTED, "no one-target propagation variant serves N=%d", c->N);
  double cost = 0;
  const Cand* b = best_for(one, no, nf, c->num_sms, &cost);
  p.tlist = d_tlist;
  p.t_begin = 0;
  p.t_count = nf;
  cudaError_t e = b->k->launch(p.dir, p, nf, b->smem, s);
  if (e != cudaSuccess) return fail(LS_ERR_CUDA, "fallback propagation launch: %s", cudaGetErrorString(e));
  return LS_OK;
}
}  // namespace

extern "C" {

int ls_sparse_run_all(ls_ctx* ctx, const int32_t* idx, int32_t K, int32_t WS, int32_t lookahead, int32_t pool,
                      const int32_t* decode_loci, int32_t D, float* d_out, float lost_tol, float* lost_out,
                      double* pac_out, uint32_t* status_out, int32_t* n_fallback_out, float d_trust,
                      uint32_t* trust_out, float* pout_out, ls_stream_t stream) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (!ctx->have_params) return fail(LS_ERR_STATE, "parameters not set");
  if (ctx->Pi) return fail(LS_ERR_UNSUPPORTED, "the sparse recursions support the uniform prior only");
  const int N = ctx->N, L = ctx->L;
  if (lookahead < 0 || lookahead > 2) return fail(LS_ERR_ARG, "lookahead must be 0, 1 or 2");
  if (!idx || K < 1 || (lookahead + 1) * K > 1536)
    return fail(LS_ERR_ARG, "need donor sets with 1 <= K and (lookahead + 1) K <= 1536 entries");
  if (WS < 1) return fail(LS_ERR_ARG, "window size must be positive");
  if (D < 1 || !decode_loci || !d_out) return fail(LS_ERR_ARG, "bad decode arguments");
  if (D > lsk::kMaxStore) return fail(LS_ERR_UNSUPPORTED, "at most %d decode loci per call", lsk::kMaxStore);
  for (int k = 0; k < D; ++k) {
    if (decode_loci[k] < 0 || decode_loci[k] >= L) return fail(LS_ERR_ARG, "decode locus %d out of range", decode_loci[k]);
    if (k && decode_loci[k] <= decode_loci[k - 1]) return fail(LS_ERR_ARG, "decode loci must be strictly increasing");
  }
  if (!is_device_ptr(idx) || !is_device_ptr(d_out)) return fail(LS_ERR_ARG, "idx and d_out must be device memory");
  if (trust_out && !is_device_ptr(trust_out)) return fail(LS_ERR_ARG, "trust_out must be device memory");
  if (pout_out && !is_device_ptr(pout_out)) return fail(LS_ERR_ARG, "pout_out must be device memory");
  const int Wn = (L + WS - 1) / WS;
  cudaStream_t s = (cudaStream_t)stream;
  DevBufs db;
  float *P, *lost, *poolf = nullptr, *share = nullptr;
  double* logs;
  uint32_t* stat;
  int* wos;
  uint8_t* dense_row;
  if ((rc = db.get(&P, (size_t)D * N * K)) || (rc = db.get(&lost, N)) || (rc = db.get(&logs, N)) ||
      (rc = db.get(&stat, N)) || (rc = db.get(&wos, 2 * D)) || (rc = db.get(&dense_row, N)) ||
      (pool && ((rc = db.get(&poolf, (size_t)D * N)) || (rc = db.get(&share, (size_t)D * N)))))
    return rc;
  CUDA_TRY(cudaMemsetAsync(dense_row, 0, N, s));
  const int32_t* sets = idx;
  if (lookahead) {  // run window w on S^w u S^{w+1} (and S^{w-1} with lookahead 2)
    int32_t* U;
    if ((rc = db.get(&U, (size_t)N * Wn * (lookahead + 1) * K))) return rc;
    cudaError_t e0 = ls_launch_lookahead(idx, N, Wn, K, lookahead, U, s);
    if (e0 != cudaSuccess) return fail(LS_ERR_CUDA, "lookahead sets: %s", cudaGetErrorString(e0));
    sets = U;
    K = (lookahead + 1) * K;
    if ((rc = db.get(&P, (size_t)D * N * K))) return rc;  // the posteriors need the wider rows
  }
  std::vector<int> wh(2 * D);  // window of each decode slot, then the decode loci themselves
  for (int k = 0; k < D; ++k) {
    wh[k] = decode_loci[k] / WS;
    wh[D + k] = decode_loci[k];
  }
  CUDA_TRY(cudaMemcpyAsync(wos, wh.data(), sizeof(int) * 2 * D, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));  // wh is a host temporary
  const int* wos_loci = wos + D;
  CUDA_TRY(cudaMemsetAsync(stat, 0, sizeof(uint32_t) * N, s));
  // haplotype-major words: each set entry's 32 bits of a block of loci are one load
  uint32_t* hw;
  if ((rc = db.get(&hw, (size_t)((L + 255) / 256) * N * 8))) return rc;
  {
    cudaError_t eh = ls_launch_hapmajor(ctx->bits, ctx->row_words, N, L, hw, s);
    if (eh != cudaSuccess) return fail(LS_ERR_CUDA, "haplotype-major words: %s", cudaGetErrorString(eh));
  }
  lsk::SparseParams sp;
  memset(&sp, 0, sizeof sp);
  sp.hw = hw;
  sp.N = N;
  sp.L = L;
  sp.K = K;
  sp.WS = WS;
  sp.Wn = Wn;
  sp.idx = sets;
  sp.omr = ctx->omr;
  sp.rho = ctx->rr_b;
  sp.thm = ctx->thm;
  sp.thx = ctx->thx;
  sp.t_begin = 0;
  sp.t_count = N;
  sp.store = P;
  sp.status = stat;
  sp.n_store = D;
  for (int k = 0; k < D; ++k) {
    sp.store_loci[k] = decode_loci[k];
    sp.store_slot[k] = k;
  }
  sp.logs = logs;
  sp.lost = lost;
  sp.poolf = poolf;
  sp.share = share;
  sp.pout = pout_out;
  if (pool) {  // per-locus allele counts for the outside pool
    int32_t* n1;
    if ((rc = db.get(&n1, L))) return rc;
    cudaError_t e1 = ls_launch_row_ones(ctx->bits, ctx->row_words, N, L, n1, s);
    if (e1 != cudaSuccess) return fail(LS_ERR_CUDA, "allele counts: %s", cudaGetErrorString(e1));
    sp.n1 = n1;
    sp.pool = 1;
  }
  cudaError_t e = ls_launch_sparse(0, sp, s);
  if (e != cudaSuccess) return fail(LS_ERR_CUDA, "sparse forward launch: %s", cudaGetErrorString(e));
  for (int k = 0; k < D; ++k) {
    sp.store_loci[k] = decode_loci[D - 1 - k];
    sp.store_slot[k] = D - 1 - k;
  }
  sp.logs = nullptr;
  sp.lost = nullptr;
  e = ls_launch_sparse(1, sp, s);
  if (e != cudaSuccess) return fail(LS_ERR_CUDA, "sparse backward launch: %s", cudaGetErrorString(e));
  // half distances: the set's donors from the chains, the others the pool's share (negated) or NaN
  e = ls_launch_sparse_hdist(P, sets, N, K, Wn, wos, share, D, d_out, s);
  if (e != cudaSuccess) return fail(LS_ERR_CUDA, "sparse distance launch: %s", cudaGetErrorString(e));
  std::vector<float> lh(N);
  CUDA_TRY(cudaMemcpyAsync(lh.data(), lost, sizeof(float) * N, cudaMemcpyDeviceToHost, s));
  if (lost_out) CUDA_TRY(cudaMemcpyAsync(lost_out, lost, sizeof(float) * N, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int> fb;
  if (lost_tol >= 0.0f)
    for (int i = 0; i < N; ++i)
      if (!(lh[i] <= lost_tol)) fb.push_back(i);
  const int nf = (int)fb.size();
  if (nf > 0) {
    // dense rows of the targets whose set lost too much forward mass
    int* tl;
    float* prod;
    if ((rc = db.get(&tl, nf)) || (rc = db.get(&prod, (size_t)D * nf * N))) return rc;
    CUDA_TRY(cudaMemcpyAsync(tl, fb.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, s));
    lsk::PropParams p;
    base_params(ctx, p, 0);
    p.l_first = 0;
    p.n_steps = L;
    p.init = 1;
    p.tab_t0 = 0;
    p.state_rows = nf;
    p.status = nullptr;
    p.n_store = D;
    for (int k = 0; k < D; ++k) {
      p.store_loci[k] = decode_loci[k];
      p.store_slot[k] = k;
    }
    p.store = prod;
    if ((rc = run_list(ctx, p, tl, nf, s))) return rc;
    base_params(ctx, p, 1);
    p.l_first = L - 1;
    p.n_steps = L;
    p.init = 1;
    p.tab_t0 = 0;
    p.state_rows = nf;
    p.n_store = D;
    for (int k = 0; k < D; ++k) {
      p.store_loci[k] = decode_loci[D - 1 - k];
      p.store_slot[k] = D - 1 - k;
    }
    p.alpha_dec = prod;
    if ((rc = run_list(ctx, p, tl, nf, s))) return rc;
    e = ls_launch_dense_rows_hdist(prod, nf, N, tl, ctx->bits, ctx->row_words, ctx->thm, ctx->thx, wos_loci, D, d_out, s);
    if (e != cudaSuccess) return fail(LS_ERR_CUDA, "fallback distance launch: %s", cudaGetErrorString(e));
    std::vector<uint8_t> flag(N, 0);
    for (int t : fb) flag[t] = 1;
    CUDA_TRY(cudaMemcpyAsync(dense_row, flag.data(), N, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));  // the host flags are copied before they go out of scope
  }
  e = ls_launch_symmetrize_trust(d_out, N, D, dense_row, d_trust, trust_out, s);
  if (e != cudaSuccess) return fail(LS_ERR_CUDA, "symmetrisation launch: %s", cudaGetErrorString(e));
  if (status_out) CUDA_TRY(cudaMemcpyAsync(status_out, stat, sizeof(uint32_t) * N, cudaMemcpyDeviceToDevice, s));
  std::vector<double> lf(N);
  std::vector<uint32_t> sh(N);
  CUDA_TRY(cudaMemcpyAsync(lf.data(), logs, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(sh.data(), stat, sizeof(uint32_t) * N, cudaMemcpyDeviceToHost, s));
  if ((rc = read_err_word(ctx, s))) return rc;
  if (pac_out) {
    double pac = 0.0;
    for (int i = 0; i < N; ++i) pac += lf[i];
    *pac_out = pac;
  }
  if (n_fallback_out) *n_fallback_out = nf;
  uint32_t any = 0;
  for (auto v : sh) any |= v;
  if (any & 1u) return LS_WARN_UNDERFLOW;
  if (any & 2u) return LS_WARN_OVERFLOW;
  return LS_OK;
}

int ls_posterior_rows(ls_ctx* ctx, const float* alpha, const float* beta, int32_t t_from, int32_t T, float* p_out,
                      ls_stream_t stream) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (!alpha || !beta || !p_out || T < 1 || t_from < 0 || t_from + T > ctx->N) return fail(LS_ERR_ARG, "bad arguments");
  lsk::posterior_kernel<<<T, 256, 0, (cudaStream_t)stream>>>(alpha, beta, ctx->N, t_from, 0, p_out);
  CUDA_TRY(cudaGetLastError());
  return LS_OK;
}

int ls_set_profiling(ls_ctx* ctx, int32_t enable) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (enable && !ctx->ev[0])
    for (auto& e : ctx->ev) CUDA_TRY(cudaEventCreate(&e));
  ctx->profile = enable != 0;
  ctx->profiled = false;
  return LS_OK;
}

int ls_profile_read(ls_ctx* ctx, float* ms, int32_t* launches) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (!ms) return fail(LS_ERR_ARG, "null output");
  if (!ctx->profiled) return fail(LS_ERR_STATE, "no profiled ls_run_all yet");
  CUDA_TRY(cudaEventSynchronize(ctx->ev[4]));
  for (int k = 0; k < 4; ++k) {
    CUDA_TRY(cudaEventElapsedTime(&ms[k], ctx->ev[k], ctx->ev[k + 1]));
    if (launches) launches[k] = ctx->launches[k];
  }
  return LS_OK;
}

}  // extern "C"

// ---- the allocation-free pipeline -----------------------------------------------------------
// Its scratch lives in a file-scope device array (every GPU that loads the library holds it until
// exit).  Host code must never hand the symbol itself to a kernel: in host code the name is a
// stand-in, not a device address.  The address is looked up once per device.
namespace {

struct NoallocScratch {
  double logF[LS_NOALLOC_MAX_N];    // per-target log F at the last locus
  uint32_t status[LS_NOALLOC_MAX_N];
  double pac;                       // PAC log-likelihood
  uint32_t any;                     // OR of the status words
  int err;                          // device error word (timed-out waits)
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
NoallocScratch* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch area for the current device (looked up on first use).
int noalloc_scratch(int device, NoallocScratch** out) {
  if (device < 0 || device >= kMaxDevices) return fail(LS_ERR_UNSUPPORTED, "device %d beyond %d", device, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail(LS_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_noalloc_ptr[device] = static_cast<NoallocScratch*>(p);
  }
  *out = g_noalloc_ptr[device];
  return LS_OK;
}

// PAC = sum_i log F_i in a fixed order (one CTA, strided partial sums, then a fixed tree), and
// the OR of the status words.
__global__ void pac_reduce_kernel(const double* __restrict__ logF, const uint32_t* __restrict__ status, int N,
                                  double* __restrict__ pac, uint32_t* __restrict__ any) {
  __shared__ double sd[256];
  __shared__ uint32_t su[256];
  double s = 0.0;
  uint32_t u = 0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    s += logF[i];
    u |= status[i];
  }
  sd[threadIdx.x] = s;
  su[threadIdx.x] = u;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sd[threadIdx.x] += sd[threadIdx.x + w];
      su[threadIdx.x] |= su[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *pac = sd[0];
    *any = su[0];
  }
}

}  // namespace

extern "C" int ls_run_all_noalloc(ls_ctx* ctx, const int32_t* decode_loci, int32_t D, float* d_out, double* pac_out,
                                  uint32_t* status_out, ls_stream_t stream) {
  int rc = check_ctx(ctx);
  if (rc) return rc;
  if (!ctx->have_params) return fail(LS_ERR_STATE, "parameters not set");
  const int N = ctx->N, L = ctx->L;
  if (N > LS_NOALLOC_MAX_N)
    return fail(LS_ERR_UNSUPPORTED, "ls_run_all_noalloc: N=%d exceeds its fixed scratch (LS_NOALLOC_MAX_N=%d targets)", N,
                LS_NOALLOC_MAX_N);
  if (D < 0 || (D > 0 && (!decode_loci || !d_out))) return fail(LS_ERR_ARG, "bad decode arguments");
  if (D > lsk::kMaxStore) return fail(LS_ERR_UNSUPPORTED, "at most %d decode loci per call", lsk::kMaxStore);
  for (int k = 0; k < D; ++k) {
    if (decode_loci[k] < 0 || decode_loci[k] >= L) return fail(LS_ERR_ARG, "decode locus %d out of range", decode_loci[k]);
    if (k && decode_loci[k] <= decode_loci[k - 1]) return fail(LS_ERR_ARG, "decode loci must be strictly increasing");
  }
  if (D > 0 && !is_device_ptr(d_out)) return fail(LS_ERR_ARG, "ls_run_all_noalloc needs d_out in device memory");
  // the same launch plan as ls_run_all (one planner, fixed arrays); planned before anything is
  // enqueued, so that an N no variant serves is refused with nothing queued
  Launch lp[2];
  int nl = 0;
  if ((rc = plan(ctx, 0, N, lp, &nl))) return rc;
  NoallocScratch* sc = nullptr;
  if ((rc = noalloc_scratch(ctx->device, &sc))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // what must start at zero: the status words (log F is written in full).  The error word is not
  // cleared here: a timed-out wait of an earlier asynchronous call stays recorded until a call
  // with pac_out reads (and then clears) it.
  CUDA_TRY(cudaMemsetAsync(sc->status, 0, sizeof(uint32_t) * N, s));
  for (int dir = 0; dir < 2; ++dir) {
    lsk::PropParams p;
    base_params(ctx, p, dir);
    p.err = &sc->err;
    p.l_first = dir == 0 ? 0 : L - 1;
    p.n_steps = L;
    p.init = 1;
    p.tab_t0 = 0;
    p.state_rows = N;
    p.status = sc->status;
    p.n_store = D;
    for (int k = 0; k < D; ++k) {
      p.store_loci[k] = dir == 0 ? decode_loci[k] : decode_loci[D - 1 - k];
      p.store_slot[k] = dir == 0 ? k : D - 1 - k;
    }
    if (dir == 0) {
      p.logs = sc->logF;
      p.store = d_out;
    } else {
      p.alpha_dec = d_out;
    }
    for (int i = 0; i < nl; ++i) {
      p.t_begin = lp[i].t_begin;
      p.t_count = lp[i].t_count;
      cudaError_t e = lp[i].k->launch(dir, p, lp[i].grid, lp[i].smem, s);
      if (e != cudaSuccess) return fail(LS_ERR_CUDA, "propagation launch: %s", cudaGetErrorString(e));
    }
  }
  if (D > 0) {
    lsk::DecodeLoci dl;
    for (int k = 0; k < D; ++k) dl.l[k] = decode_loci[k];
    lsk::decode_kernel<<<dim3(N, D), 256, 0, s>>>(d_out, N, ctx->bits, ctx->row_words, ctx->thm, ctx->thx, dl);
    CUDA_TRY(cudaGetLastError());
    const int nt = (N + 31) / 32;
    lsk::symmetrize_kernel<<<dim3(nt, nt, D), dim3(32, 8), 0, s>>>(d_out, N);
    CUDA_TRY(cudaGetLastError());
  }
  pac_reduce_kernel<<<1, 256, 0, s>>>(sc->logF, sc->status, N, &sc->pac, &sc->any);
  CUDA_TRY(cudaGetLastError());
  if (status_out) CUDA_TRY(cudaMemcpyAsync(status_out, sc->status, sizeof(uint32_t) * N, cudaMemcpyDeviceToDevice, s));
  if (!pac_out) return LS_OK;
  double pac = 0.0;
  uint32_t any = 0;
  int err = 0;
  CUDA_TRY(cudaMemcpyAsync(&pac, &sc->pac, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(&any, &sc->any, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(&err, &sc->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (err) {
    CUDA_TRY(cudaMemsetAsync(&sc->err, 0, sizeof(int), s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return fail(LS_ERR_DEVICE, "a device wait for staged haplotype rows ran out of time (this or an earlier call)");
  }
  *pac_out = pac;
  if (any & 1u) return LS_WARN_UNDERFLOW;
  if (any & 2u) return LS_WARN_OVERFLOW;
  return LS_OK;
}
