// ls_sparse.cu -- instantiations and launchers of the sparse (proposed-set) recursions.
#include "ls_internal.h"
#include "ls_sparse.cuh"

namespace {
template <int KS>
cudaError_t launch_ks(int dir, const lsk::SparseParams& p0, cudaStream_t s) {
  const lsk::SparseParams& p = p0;
  const int smem = lsk::sparse_smem_bytes(KS);
  const void* f = dir == 0 ? (const void*)lsk::ls_sparse_kernel<0, KS> : (const void*)lsk::ls_sparse_kernel<1, KS>;
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int grid = (p.t_count + lsk::kSparseWarps - 1) / lsk::kSparseWarps;
  if (dir == 0) lsk::ls_sparse_kernel<0, KS><<<grid, lsk::kSparseWarps * 32, smem, s>>>(p);
  else lsk::ls_sparse_kernel<1, KS><<<grid, lsk::kSparseWarps * 32, smem, s>>>(p);
  return cudaGetLastError();
}
}  // namespace

// slots per lane: the smallest of 1, 2, 4, 8, 16, 32, 48 with 32 * KS >= K (K <= 1536)
cudaError_t ls_launch_sparse(int dir, const lsk::SparseParams& p, cudaStream_t s) {
  if (p.K <= 32) return launch_ks<1>(dir, p, s);
  if (p.K <= 64) return launch_ks<2>(dir, p, s);
  if (p.K <= 128) return launch_ks<4>(dir, p, s);
  if (p.K <= 256) return launch_ks<8>(dir, p, s);
  if (p.K <= 512) return launch_ks<16>(dir, p, s);
  if (p.K <= 1024) return launch_ks<32>(dir, p, s);
  return launch_ks<48>(dir, p, s);
}

cudaError_t ls_launch_lookahead(const int32_t* idx, int N, int Wn, int K, int span, int32_t* U, cudaStream_t s) {
  const long long n = (long long)N * Wn;
  lsk::lookahead_sets_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(idx, N, Wn, K, span, U);
  return cudaGetLastError();
}

cudaError_t ls_launch_sparse_hdist(const float* P, const int32_t* idx, int N, int K, int Wn, const int* win_of_slot,
                                   const float* share, int D, float* h, cudaStream_t s) {
  lsk::sparse_hdist_kernel<<<dim3(N, D), 256, 0, s>>>(P, idx, N, K, Wn, win_of_slot, share, h);
  return cudaGetLastError();
}

cudaError_t ls_launch_symmetrize_trust(float* d, int N, int D, const uint8_t* dense_row, float d_trust, uint32_t* mask,
                                       cudaStream_t s) {
  const int nt = (N + 31) / 32;
  lsk::symmetrize_trust_kernel<<<dim3(nt, nt, D), dim3(32, 8), 0, s>>>(d, N, dense_row, d_trust, mask, nt);
  return cudaGetLastError();
}

cudaError_t ls_launch_dense_rows_hdist(const float* prod, int nf, int N, const int* tlist, const uint32_t* bits,
                                       int row_words, const float* thm, const float* thx, const int* dloci, int D, float* h,
                                       cudaStream_t s) {
  lsk::dense_rows_hdist_kernel<<<dim3(nf, D), 256, 0, s>>>(prod, nf, N, tlist, bits, row_words, thm, thx, dloci, h);
  return cudaGetLastError();
}

cudaError_t ls_launch_row_ones(const uint32_t* bits, int row_words, int N, int L, int32_t* n1, cudaStream_t s) {
  const long long threads = 32ll * L;
  lsk::row_ones_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(bits, row_words, N, L, n1);
  return cudaGetLastError();
}
