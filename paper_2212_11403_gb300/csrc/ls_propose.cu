// ls_propose.cu -- C ABI of the learned donor proposal: window features, the MLP (training and
// BF16 inference) and the proposal of per-window donor sets for ls_sparse_run_all.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ls.h"
#include "ls_internal.h"
#include "ls_mlp.cuh"
#include "ls_propose.cuh"
#include "ls_mlp_tc.cuh"

struct ls_mlp {
  int device = 0;
  float* p = nullptr;       // [kMlpParams] FP32 master weights
  float* g = nullptr;       // gradient
  float* m = nullptr;       // Adam moments
  float* v = nullptr;
  long long t = 0;          // Adam step count
  __nv_bfloat16* w1t = nullptr;  // [256][16]
  __nv_bfloat16* w2t = nullptr;  // [256][256]
  float b3 = 0.0f;
  int* err = nullptr;            // device word: a scorer wait ran out of time
};

namespace {

template <class... A>
int fail(int code, const char* fmt, A... a) {
  return ls_fail(code, fmt, a...);
}
int dev_alloc(void*, void** p, size_t n) { return ls_dev_alloc(p, n); }

#define TRY(x)                                                                                 \
  do {                                                                                         \
    cudaError_t e_ = (x);                                                                      \
    if (e_ != cudaSuccess) return fail(LS_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_));     \
  } while (0)

struct Bufs {
  std::vector<void*> v;
  ~Bufs() {
    for (void* q : v) cudaFree(q);
  }
  template <class T>
  int get(T** q, size_t n) {
    int rc = dev_alloc(nullptr, (void**)q, sizeof(T) * std::max<size_t>(n, 1));
    if (!rc) v.push_back(*q);
    return rc;
  }
};

// BF16 transposed copies for the MMA kernel
__global__ void mlp_refresh_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ w1t,
                                   __nv_bfloat16* __restrict__ w2t) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < 256 * 256) {
    const int n = e >> 8, k = e & 255;
    w2t[e] = __float2bfloat16_rn(p[lsk::kOffW2 + k * 256 + n]);
  }
  if (e < 256 * lsk::kFeat) {
    const int n = e >> 4, k = e & 15;
    w1t[e] = __float2bfloat16_rn(k < lsk::kMlpIn ? p[lsk::kOffW1 + k * 256 + n] : 0.0f);
  }
}

__global__ void to_bf16_feat_kernel(const float* __restrict__ X, long long n, __nv_bfloat16* __restrict__ Xb) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * lsk::kFeat) return;
  const long long r = e / lsk::kFeat;
  const int k = (int)(e % lsk::kFeat);
  Xb[e] = __float2bfloat16_rn(k < lsk::kMlpIn ? X[r * lsk::kMlpIn + k] : 0.0f);
}

int refresh(ls_mlp* m) {
  mlp_refresh_kernel<<<256, 256>>>(m->p, m->w1t, m->w2t);
  TRY(cudaGetLastError());
  TRY(cudaMemcpy(&m->b3, m->p + lsk::kOffB3, sizeof(float), cudaMemcpyDeviceToHost));
  return LS_OK;
}

// Scores of n BF16 feature rows on the tensor cores (persistent CTAs, one per SM).
int launch_scores(const ls_mlp* m, const __nv_bfloat16* X, long long n, float* scores, int nsm, cudaStream_t s) {
  TRY(cudaFuncSetAttribute(lsk::mlp_score_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lsk::kTcSmem));
  lsk::MlpTcDev d;
  d.w1t = m->w1t;
  d.b1 = m->p + lsk::kOffB1;
  d.w2t = m->w2t;
  d.b2 = m->p + lsk::kOffB2;
  d.w3 = m->p + lsk::kOffW3;
  d.b3 = m->b3;
  d.err = m->err;
  const long long tiles = (n + lsk::kTcRows - 1) / lsk::kTcRows;
  const int grid = (int)std::min<long long>(nsm, tiles);
  lsk::mlp_score_tc_kernel<<<grid, lsk::kTcThreads, lsk::kTcSmem, s>>>(d, X, n, scores);
  TRY(cudaGetLastError());
  return LS_OK;
}

// the error word of the scorer: LS_ERR_DEVICE (and cleared) when a wait ran out of time
int scorer_status(const ls_mlp* m, cudaStream_t s) {
  int h = 0;
  TRY(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if (h) {
    cudaMemsetAsync(m->err, 0, sizeof(int), s);
    return fail(LS_ERR_DEVICE, "a wait of the tensor-core scorer ran out of time");
  }
  return LS_OK;
}

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

void gemm(cudaStream_t s, int M, int N, int K, const float* A, int lda, int ta, const float* B, int ldb, int tb, float* C,
          int ldc, float beta) {
  lsk::gemm_f32_kernel<<<dim3((N + 15) / 16, (M + 15) / 16), 256, 0, s>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, beta);
}

// forward + backward of a batch (X [B][8], y [B]) into m->g; loss sum into *loss
int batch_grad(ls_mlp* m, const float* X, const float* y, int B, cudaStream_t s, double* loss) {
  Bufs b;
  float *Z1, *H1, *Z2, *H2, *ds, *dH2, *dH1;
  double* part;
  const int nb = (int)blocks(B);
  int rc;
  if ((rc = b.get(&Z1, (size_t)B * 256)) || (rc = b.get(&H1, (size_t)B * 256)) || (rc = b.get(&Z2, (size_t)B * 256)) ||
      (rc = b.get(&H2, (size_t)B * 256)) || (rc = b.get(&ds, B)) || (rc = b.get(&dH2, (size_t)B * 256)) ||
      (rc = b.get(&dH1, (size_t)B * 256)) || (rc = b.get(&part, nb)))
    return rc;
  const float* p = m->p;
  float* g = m->g;
  const long long n256 = (long long)B * 256;
  gemm(s, B, 256, lsk::kMlpIn, X, lsk::kMlpIn, 0, p + lsk::kOffW1, 256, 0, Z1, 256, 0.0f);
  lsk::bias_relu_kernel<<<blocks(n256), 256, 0, s>>>(Z1, p + lsk::kOffB1, B, 256, H1);
  gemm(s, B, 256, 256, H1, 256, 0, p + lsk::kOffW2, 256, 0, Z2, 256, 0.0f);
  lsk::bias_relu_kernel<<<blocks(n256), 256, 0, s>>>(Z2, p + lsk::kOffB2, B, 256, H2);
  lsk::head_kernel<<<nb, 256, 0, s>>>(H2, p + lsk::kOffW3, p + lsk::kOffB3, y, B, ds, part);
  // output layer
  gemm(s, 256, 1, B, H2, 256, 1, ds, 1, 0, g + lsk::kOffW3, 1, 0.0f);
  lsk::colsum_kernel<<<1, 32, 0, s>>>(ds, B, 1, g + lsk::kOffB3);
  // hidden layer 2
  lsk::outer_kernel<<<blocks(n256), 256, 0, s>>>(ds, p + lsk::kOffW3, B, dH2);
  lsk::relu_back_kernel<<<blocks(n256), 256, 0, s>>>(dH2, Z2, n256);
  gemm(s, 256, 256, B, H1, 256, 1, dH2, 256, 0, g + lsk::kOffW2, 256, 0.0f);
  lsk::colsum_kernel<<<1, 256, 0, s>>>(dH2, B, 256, g + lsk::kOffB2);
  // hidden layer 1
  gemm(s, B, 256, 256, dH2, 256, 0, p + lsk::kOffW2, 256, 1, dH1, 256, 0.0f);
  lsk::relu_back_kernel<<<blocks(n256), 256, 0, s>>>(dH1, Z1, n256);
  gemm(s, lsk::kMlpIn, 256, B, X, lsk::kMlpIn, 1, dH1, 256, 0, g + lsk::kOffW1, 256, 0.0f);
  lsk::colsum_kernel<<<1, 256, 0, s>>>(dH1, B, 256, g + lsk::kOffB1);
  TRY(cudaGetLastError());
  if (loss) {
    std::vector<double> h(nb);
    TRY(cudaMemcpyAsync(h.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    double t = 0.0;
    for (double v : h) t += v;
    *loss = t;
  } else {
    TRY(cudaStreamSynchronize(s));  // the batch buffers are freed on return
  }
  return LS_OK;
}

}  // namespace

extern "C" {

int ls_mlp_create(const float* params, uint64_t seed, ls_mlp** out) {
  if (!out) return fail(LS_ERR_ARG, "null output");
  ls_mlp* m = new ls_mlp;
  cudaGetDevice(&m->device);
  const size_t P = lsk::kMlpParams;
  int rc;
  if ((rc = dev_alloc(nullptr, (void**)&m->p, sizeof(float) * P)) || (rc = dev_alloc(nullptr, (void**)&m->g, sizeof(float) * P)) ||
      (rc = dev_alloc(nullptr, (void**)&m->m, sizeof(float) * P)) || (rc = dev_alloc(nullptr, (void**)&m->v, sizeof(float) * P)) ||
      (rc = dev_alloc(nullptr, (void**)&m->w1t, 2 * 256 * lsk::kFeat)) || (rc = dev_alloc(nullptr, (void**)&m->w2t, 2 * 256 * 256)) ||
      (rc = dev_alloc(nullptr, (void**)&m->err, sizeof(int)))) {
    cudaFree(m->p);
    cudaFree(m->g);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->w1t);
    cudaFree(m->w2t);
    delete m;
    return rc;
  }
  cudaMemset(m->err, 0, sizeof(int));
  std::vector<float> h(P, 0.0f);
  if (params) {
    memcpy(h.data(), params, sizeof(float) * P);
  } else {
    // He-uniform initialisation from a seeded splitmix64 stream; biases 0
    uint64_t s = seed;
    auto uni = [&]() { return (float)((double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0)) * 2.0f - 1.0f; };
    const float a1 = std::sqrt(6.0f / 7.0f), a2 = std::sqrt(6.0f / 256.0f), a3 = std::sqrt(3.0f / 256.0f);
    for (int k = 0; k < 7; ++k)
      for (int n = 0; n < 256; ++n) h[lsk::kOffW1 + k * 256 + n] = a1 * uni();
    for (int e = 0; e < 256 * 256; ++e) h[lsk::kOffW2 + e] = a2 * uni();
    for (int e = 0; e < 256; ++e) h[lsk::kOffW3 + e] = a3 * uni();
  }
  cudaMemcpy(m->p, h.data(), sizeof(float) * P, cudaMemcpyHostToDevice);
  cudaMemset(m->m, 0, sizeof(float) * P);
  cudaMemset(m->v, 0, sizeof(float) * P);
  if ((rc = refresh(m))) {
    ls_mlp_destroy(m);
    return rc;
  }
  *out = m;
  return LS_OK;
}

int ls_mlp_destroy(ls_mlp* m) {
  if (!m) return fail(LS_ERR_ARG, "null network");
  cudaSetDevice(m->device);
  cudaFree(m->p);
  cudaFree(m->g);
  cudaFree(m->m);
  cudaFree(m->v);
  cudaFree(m->w1t);
  cudaFree(m->w2t);
  cudaFree(m->err);
  delete m;
  return LS_OK;
}

int ls_mlp_get(const ls_mlp* m, float* params) {
  if (!m || !params) return fail(LS_ERR_ARG, "null argument");
  TRY(cudaMemcpy(params, m->p, sizeof(float) * lsk::kMlpParams, cudaMemcpyDeviceToHost));
  return LS_OK;
}

int ls_mlp_set(ls_mlp* m, const float* params) {
  if (!m || !params) return fail(LS_ERR_ARG, "null argument");
  TRY(cudaMemcpy(m->p, params, sizeof(float) * lsk::kMlpParams, cudaMemcpyHostToDevice));
  return refresh(m);
}

int ls_mlp_forward(const ls_mlp* m, const float* X, int64_t n, float* scores, ls_stream_t stream) {
  if (!m || (n > 0 && (!X || !scores))) return fail(LS_ERR_ARG, "null argument");
  if (n <= 0) return LS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Bufs b;
  __nv_bfloat16* Xb;
  int rc;
  if ((rc = b.get(&Xb, (size_t)n * lsk::kFeat))) return rc;
  to_bf16_feat_kernel<<<blocks(n * lsk::kFeat), 256, 0, s>>>(X, n, Xb);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
  if ((rc = launch_scores(m, Xb, n, scores, nsm, s))) return rc;
  return scorer_status(m, s);
}

int ls_mlp_grad(ls_mlp* m, const float* X, const float* y, int32_t n, float* grad, double* loss, ls_stream_t stream) {
  if (!m || !X || !y || n < 1) return fail(LS_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = batch_grad(m, X, y, n, s, loss);
  if (rc) return rc;
  if (loss) *loss /= n;
  if (grad) TRY(cudaMemcpy(grad, m->g, sizeof(float) * lsk::kMlpParams, cudaMemcpyDeviceToHost));
  return LS_OK;
}

int ls_mlp_train(ls_mlp* m, const float* X, const float* y, int64_t n, int32_t steps, int32_t batch, float lr,
                 uint64_t seed, double* loss_out, ls_stream_t stream) {
  if (!m || !X || !y || n < 1 || steps < 0 || batch < 1) return fail(LS_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  Bufs b;
  float *Xb, *yb;
  int* sel;
  int rc;
  if ((rc = b.get(&Xb, (size_t)batch * lsk::kMlpIn)) || (rc = b.get(&yb, batch)) || (rc = b.get(&sel, batch))) return rc;
  std::vector<int> hs(batch);
  uint64_t st = seed;
  double tail = 0.0;
  int ntail = 0;
  for (int it = 0; it < steps; ++it) {
    for (int r = 0; r < batch; ++r) hs[r] = (int)(splitmix(st) % (uint64_t)n);
    TRY(cudaMemcpyAsync(sel, hs.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, s));
    lsk::gather_rows_kernel<<<blocks((long long)batch * lsk::kMlpIn), 256, 0, s>>>(X, y, sel, batch, Xb, yb);
    const bool want = it >= steps - std::max(1, steps / 10);
    double l = 0.0;
    if ((rc = batch_grad(m, Xb, yb, batch, s, want ? &l : nullptr))) return rc;
    if (want) {
      tail += l / batch;
      ++ntail;
    }
    ++m->t;
    const float c1 = 1.0f - std::pow(0.9f, (float)m->t), c2 = 1.0f - std::pow(0.999f, (float)m->t);
    lsk::adam_kernel<<<blocks(lsk::kMlpParams), 256, 0, s>>>(m->p, m->g, m->m, m->v, lsk::kMlpParams, lr, 0.9f, 0.999f, c1,
                                                              c2, 1e-8f);
    TRY(cudaGetLastError());
  }
  TRY(cudaStreamSynchronize(s));
  if (loss_out) *loss_out = ntail ? tail / ntail : 0.0;
  return refresh(m);
}

}  // extern "C"

namespace {
struct PropWork {
  int N = 0, L = 0, Wn = 0, Np = 0;
  uint32_t* hw = nullptr;
  uint8_t* ring[7] = {};
  int ring_w[7] = {-1, -1, -1, -1, -1, -1, -1};
  std::vector<int> nv;
};

int prop_setup(ls_ctx* c, Bufs& b, PropWork& pw, cudaStream_t s) {
  pw.N = c->N;
  pw.L = c->L;
  pw.Wn = (c->L + lsk::kPropWS - 1) / lsk::kPropWS;
  pw.Np = lsk::round_up(c->N, 64);
  int rc;
  if ((rc = b.get(&pw.hw, (size_t)pw.Wn * pw.N * 8))) return rc;
  for (int k = 0; k < 7; ++k)
    if ((rc = b.get(&pw.ring[k], (size_t)pw.N * pw.Np))) return rc;
  lsk::hapmajor_kernel<<<dim3((pw.N + 31) / 32, 8, pw.Wn), 32, 0, s>>>(c->bits, c->row_words, pw.N, pw.L, pw.hw);
  TRY(cudaGetLastError());
  pw.nv.resize(pw.Wn);
  for (int w = 0; w < pw.Wn; ++w) pw.nv[w] = std::min(lsk::kPropWS, pw.L - w * lsk::kPropWS);
  return LS_OK;
}

int ensure(PropWork& pw, int w, cudaStream_t s) {
  const int slot = w % 7;
  if (pw.ring_w[slot] == w) return LS_OK;
  const int nb = pw.Np / 64;
  lsk::mismatch_kernel<<<dim3(nb, (pw.N + 63) / 64), 256, 0, s>>>(pw.hw + (size_t)w * pw.N * 8, pw.N, pw.Np, pw.ring[slot]);
  TRY(cudaGetLastError());
  pw.ring_w[slot] = w;
  return LS_OK;
}

int stage1(PropWork& pw, int w, int C, int32_t* cand, long long cstride, __nv_bfloat16* feat, float* feat32,
           cudaStream_t s) {
  for (int d = -3; d <= 3; ++d) {
    const int ww = std::min(std::max(w + d, 0), pw.Wn - 1);
    int rc = ensure(pw, ww, s);
    if (rc) return rc;
  }
  lsk::Stage1Args a;
  for (int d = 0; d < 7; ++d) {
    const int ww = std::min(std::max(w + d - 3, 0), pw.Wn - 1);
    a.Ms[d] = pw.ring[ww % 7];
    a.inv_nv[d] = 1.0f / (float)pw.nv[ww];
  }
  a.use[0] = w - 1 >= 0;
  a.use[1] = 1;
  a.use[2] = w + 1 < pw.Wn;
  (void)cstride;
  lsk::stage1_kernel<<<pw.N, 256, 0, s>>>(a, pw.N, pw.Np, C, cand, feat, feat32);
  TRY(cudaGetLastError());
  return LS_OK;
}
}  // namespace

extern "C" {

int ls_propose_window(ls_ctx* ctx, int32_t C, int32_t w, int32_t* cand_out, float* feat_out, ls_stream_t stream) {
  if (!ctx || C < 1 || !cand_out) return fail(LS_ERR_ARG, "bad arguments");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  Bufs b;
  PropWork pw;
  int rc = prop_setup(ctx, b, pw, s);
  if (rc) return rc;
  if (w < 0 || w >= pw.Wn) return fail(LS_ERR_ARG, "window %d outside [0, %d)", w, pw.Wn);
  if ((rc = stage1(pw, w, C, cand_out, C, nullptr, feat_out, s))) return rc;
  TRY(cudaStreamSynchronize(s));
  return LS_OK;
}

int ls_propose_labels(ls_ctx* ctx, const float* P, const int32_t* cand, int32_t C, float* y_out, ls_stream_t stream) {
  if (!ctx || !P || !cand || !y_out || C < 1) return fail(LS_ERR_ARG, "bad arguments");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  lsk::label_kernel<<<8 * ctx->num_sms, 256, 0, s>>>(P, cand, ctx->N, C, 1e-12f, y_out);
  TRY(cudaGetLastError());
  TRY(cudaStreamSynchronize(s));
  return LS_OK;
}

int ls_propose(ls_ctx* ctx, int32_t C, int32_t K, const ls_mlp* mlp, int32_t* idx_out, ls_stream_t stream) {
  if (!ctx || K < 1 || K > 512 || !idx_out) return fail(LS_ERR_ARG, "bad arguments (1 <= K <= 512)");
  if (mlp && (C < K || C > 2048)) return fail(LS_ERR_ARG, "need K <= C <= 2048 candidates for the MLP stage");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  Bufs b;
  PropWork pw;
  int rc = prop_setup(ctx, b, pw, s);
  if (rc) return rc;
  const int N = pw.N, Wn = pw.Wn;
  const int Ce = mlp ? C : K;
  int32_t* cand;
  __nv_bfloat16* feat = nullptr;
  float* scores = nullptr;
  if ((rc = b.get(&cand, (size_t)N * Ce))) return rc;
  if (mlp && ((rc = b.get(&feat, (size_t)N * Ce * lsk::kFeat)) || (rc = b.get(&scores, (size_t)N * Ce)))) return rc;
  int P = 1;
  while (P < Ce) P <<= 1;
  // topk needs P * 8 <= 16 KB of dynamic shared memory, within the default limit
  for (int w = 0; w < Wn; ++w) {
    if ((rc = stage1(pw, w, Ce, cand, Ce, feat, nullptr, s))) return rc;
    if (mlp && (rc = launch_scores(mlp, feat, (long long)N * Ce, scores, ctx->num_sms, s))) return rc;
    // the K best (by score, or by the stage-1 order when there is no network) in ascending id order
    lsk::topk_kernel<<<N, 256, P * 8, s>>>(cand, mlp ? scores : nullptr, Ce, K, P, Wn, w, idx_out);
    TRY(cudaGetLastError());
  }
  TRY(cudaStreamSynchronize(s));
  return mlp ? scorer_status(mlp, s) : LS_OK;
}

}  // extern "C"

// haplotype-major words of the packed rows: hw [ceil(L/256)][N][8] (the sparse recursions read
// their donors' bits from it)
cudaError_t ls_launch_hapmajor(const uint32_t* bits, int row_words, int N, int L, uint32_t* hw, cudaStream_t s) {
  const int Wn = (L + lsk::kPropWS - 1) / lsk::kPropWS;
  lsk::hapmajor_kernel<<<dim3((N + 31) / 32, 8, Wn), 32, 0, s>>>(bits, row_words, N, L, hw);
  return cudaGetLastError();
}
