// ls_internal.h -- host-side structures shared by the libls translation units.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "ls_prop.cuh"

// One compiled variant of the propagation kernel: TPW targets per CTA, W warps, KQ quads per lane
// (forward and backward instantiations).
struct PropKernelInfo {
  int tpw, w, kq;
  int pim;  // prior-matrix variant: 1 FP32 prior values, 2 bfloat16 (0: uniform prior)
  int st;   // 1: statistic-pass variant (launch's dir argument picks ST 1 or ST 2)
  const void* func[2];
  cudaError_t (*launch)(int dir, const lsk::PropParams& p, int grid, int smem, cudaStream_t s);
  int (*smem_bytes)(int rw2);
  bool (*serves)(int N);
  int cpt = 1;  // CTAs per target (2: a thread-block cluster of two CTAs shares one target)
  int pi16 = 0; // 1: holds the prior matrix on chip as bfloat16 (needs the BF16 prior format)
};

void ls_register_prop_kernels(std::vector<PropKernelInfo>& out);

// shared by the translation units: set the thread's error message and return code; device
// allocation with LS_ERR_OOM on failure
int ls_fail(int code, const char* fmt, ...);
int ls_dev_alloc(void** p, size_t bytes);

namespace lsk {
struct SparseParams;
}
cudaError_t ls_launch_sparse(int dir, const lsk::SparseParams& p, cudaStream_t s);
cudaError_t ls_launch_row_ones(const uint32_t* bits, int row_words, int N, int L, int32_t* n1, cudaStream_t s);
cudaError_t ls_launch_hapmajor(const uint32_t* bits, int row_words, int N, int L, uint32_t* hw, cudaStream_t s);
cudaError_t ls_launch_lookahead(const int32_t* idx, int N, int Wn, int K, int span, int32_t* U, cudaStream_t s);
cudaError_t ls_launch_sparse_hdist(const float* P, const int32_t* idx, int N, int K, int Wn, const int* win_of_slot,
                                   const float* share, int D, float* h, cudaStream_t s);
cudaError_t ls_launch_symmetrize_trust(float* d, int N, int D, const uint8_t* dense_row, float d_trust, uint32_t* mask,
                                       cudaStream_t s);
cudaError_t ls_launch_dense_rows_hdist(const float* prod, int nf, int N, const int* tlist, const uint32_t* bits,
                                       int row_words, const float* thm, const float* thx, const int* dloci, int D, float* h,
                                       cudaStream_t s);

struct ls_ctx {
  int device = 0;
  int N = 0, L = 0, row_words = 0;
  uint32_t* bits = nullptr;       // [L][row_words], the packed cache
  uint32_t* bits2 = nullptr;      // [L][rw2], every row doubled (2N bits) for the propagation kernel
  int rw2 = 0;
  size_t bytes = 0;               // device bytes owned
  // parameters
  bool have_params = false;
  uint64_t hash = 0;
  float* omr = nullptr;           // [L-1] 1 - rho
  float* rr_f = nullptr;          // [L-1] rho * pi (forward)
  float* rr_b = nullptr;          // [L-1] rho (backward)
  float* thm = nullptr;           // [L] 1 - mu
  float* thx = nullptr;           // [L] mu
  float* Pi = nullptr;            // [N][N] prior matrix copy (null: uniform)
  int prior_bf16 = 0;             // LS_PRIOR_BF16: Pi rounded to bfloat16 by ls_set_params
  float pi_u = 0.0f;
  int mu_vec = 0;                 // mu given per locus
  std::vector<double> rho_h, mu_h;  // host copies (the gradient's constant terms)
  // scratch
  double* logs_scratch = nullptr; // [N]
  uint32_t* status_scratch = nullptr;  // [N]
  int* err = nullptr;             // device error word
  float* dscratch = nullptr;      // host-output staging for ls_run_all
  size_t dscratch_bytes = 0;
  int num_sms = 0;
  int ntables = 0;
  // profiling of ls_run_all phases
  bool profile = false;
  bool profiled = false;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // side stream for the tail launch of a main/tail plan (fork/join events on the caller's stream)
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  int launches[4] = {0, 0, 0, 0};
};

struct ls_ckpt {
  ls_ctx* ctx = nullptr;
  int dtype = 0;
  int t_from = 0, t_to = 0;
  std::vector<int> loci;     // c_0 < c_1 < ... < c_{K-1}
  uint64_t hash = 0;
  void* data = nullptr;      // [K][T][N] float or binary16
  float* scale = nullptr;    // [K][T] (binary16 only)
  double* logs = nullptr;    // [K][T]
  size_t bytes = 0;
};

struct ls_table {
  ls_ctx* ctx = nullptr;
  int kind = 0;
  int t_from = 0, t_to = 0;
  int locus = -1;
  uint64_t hash = 0;
  float* state = nullptr;   // [T][N]
  double* logs = nullptr;   // [T]
};
