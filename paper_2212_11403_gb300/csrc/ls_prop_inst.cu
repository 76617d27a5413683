// ls_prop_inst.cu -- compiled variants of the propagation kernel and their registry.
//
// A variant is (TPW targets per CTA, W warps, KQ quads of 4 donor slots per lane); a CTA covers
// W * 32 / TPW slices of up to 4*KQ donors.  PropCfg::serves(N) decides which variants fit a
// given N; the host planner picks the one with the fewest CTA waves x slots per lane.  Variants
// are spread over translation units (LS_INST_GROUP) so the build compiles them in parallel.
#include "ls_internal.h"
#include "ls_hyb.cuh"

namespace {

template <int TPW, int W, int KQ, int PIM>
cudaError_t launch_prop(int dir, const lsk::PropParams& p, int grid, int smem, cudaStream_t s) {
  if (dir == 0) lsk::ls_prop_kernel<0, TPW, W, KQ, PIM, 0><<<grid, W * 32, smem, s>>>(p);
  else lsk::ls_prop_kernel<1, TPW, W, KQ, PIM, 0><<<grid, W * 32, smem, s>>>(p);
  return cudaGetLastError();
}

// statistic passes (forward only): dir selects ST 1 (0) or ST 2 (1)
template <int TPW, int W, int KQ>
cudaError_t launch_stat(int which, const lsk::PropParams& p, int grid, int smem, cudaStream_t s) {
  if (which == 0) lsk::ls_prop_kernel<0, TPW, W, KQ, 0, 1><<<grid, W * 32, smem, s>>>(p);
  else lsk::ls_prop_kernel<0, TPW, W, KQ, 0, 2><<<grid, W * 32, smem, s>>>(p);
  return cudaGetLastError();
}

template <int TPW, int W, int KQ, int PIM>
int smem_prop(int rw2) {
  return lsk::PropCfg<TPW, W, KQ>::layout(rw2, PIM).total;
}

template <int TPW, int W, int KQ>
bool serves_prop(int N) {
  return lsk::PropCfg<TPW, W, KQ>::serves(N);
}

// grid = number of targets; CL CTAs (a thread-block cluster when CL = 2) per target
template <int QS, int CL, int PIM>
cudaError_t launch_hyb(int dir, const lsk::PropParams& p, int grid, int smem, cudaStream_t s) {
  if (CL == 1) {
    if (dir == 0) lsk::ls_hyb_kernel<0, QS, 1, PIM><<<grid, lsk::kHybThreads, smem, s>>>(p);
    else lsk::ls_hyb_kernel<1, QS, 1, PIM><<<grid, lsk::kHybThreads, smem, s>>>(p);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(CL * grid), 1, 1);
  cfg.blockDim = dim3(lsk::kHybThreads, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (dir == 0) return cudaLaunchKernelEx(&cfg, lsk::ls_hyb_kernel<0, QS, CL, PIM>, p);
  return cudaLaunchKernelEx(&cfg, lsk::ls_hyb_kernel<1, QS, CL, PIM>, p);
}
template <int QS, int PIM>
int smem_hyb(int) {
  return lsk::HybCfg<QS, PIM>::smem_bytes();
}
template <int QS, int CL, int PIM>
bool serves_hyb(int N) {
  return lsk::HybCfg<QS, PIM>::serves(N, CL);
}

}  // namespace

// large-N variants: one target per CTA of 16 warps, 12 quads per thread in registers and QS in
// shared memory
#define LS_REGHX(QS, CL, P)                                                                         \
  out.push_back(PropKernelInfo{1, lsk::kHybThreads / 32, lsk::kHybQR + QS, P, 0,                    \
                               {(const void*)lsk::ls_hyb_kernel<0, QS, CL, P>, (const void*)lsk::ls_hyb_kernel<1, QS, CL, P>}, \
                               launch_hyb<QS, CL, P>, smem_hyb<QS, P>, serves_hyb<QS, CL, P>, CL, P})
#define LS_REGH(QS) LS_REGHX(QS, 1, 0)
// a cluster of two CTAs (on two SMs) per target: N in (57344, 2 x 2048 (12 + QS)]
#define LS_REGH2(QS) LS_REGHX(QS, 2, 0)
// prior matrix, held on chip as bfloat16 (the BF16 prior format): N in (20480, 53248] with one CTA,
// (53248, 2 x 2048 (12 + QS)] with a cluster of two
#define LS_REGHP(QS) LS_REGHX(QS, 1, 1)
#define LS_REGH2P(QS) LS_REGHX(QS, 2, 1)

#define LS_REGP(T, Wp, K, P)                                                                        \
  out.push_back(PropKernelInfo{T, Wp, K, P, 0,                                                      \
                               {(const void*)lsk::ls_prop_kernel<0, T, Wp, K, P, 0>,                \
                                (const void*)lsk::ls_prop_kernel<1, T, Wp, K, P, 0>},               \
                               launch_prop<T, Wp, K, P>, smem_prop<T, Wp, K, P>, serves_prop<T, Wp, K>, 1, P == 2})
#define LS_REG(T, Wp, K) LS_REGP(T, Wp, K, 0)
// statistic-pass variants: func[0] = ST 1, func[1] = ST 2
#define LS_REGS(T, Wp, K)                                                                           \
  out.push_back(PropKernelInfo{T, Wp, K, 0, 1,                                                      \
                               {(const void*)lsk::ls_prop_kernel<0, T, Wp, K, 0, 1>,                \
                                (const void*)lsk::ls_prop_kernel<0, T, Wp, K, 0, 2>},               \
                               launch_stat<T, Wp, K>, smem_prop<T, Wp, K, 0>, serves_prop<T, Wp, K>})

#if LS_INST_GROUP == 0
void ls_register_group0(std::vector<PropKernelInfo>& out) {
  // 4 targets per CTA, two CTAs per SM: N up to 5120
  LS_REG(4, 4, 40);
  LS_REG(4, 8, 20);
}
#elif LS_INST_GROUP == 1
void ls_register_group1(std::vector<PropKernelInfo>& out) {
  LS_REG(4, 4, 32);
  LS_REG(4, 4, 24);
  LS_REG(4, 4, 16);
}
#elif LS_INST_GROUP == 2
void ls_register_group2(std::vector<PropKernelInfo>& out) {
  // 8 targets per CTA for N up to 2560
  LS_REG(8, 4, 40);
  LS_REG(8, 4, 32);
  LS_REG(8, 4, 24);
}
#elif LS_INST_GROUP == 3
void ls_register_group3(std::vector<PropKernelInfo>& out) {
  LS_REG(8, 4, 16);
  LS_REG(8, 4, 8);
  LS_REG(8, 4, 4);
  LS_REG(8, 4, 2);
}
#elif LS_INST_GROUP == 4
void ls_register_group4(std::vector<PropKernelInfo>& out) {
  // 2 or 1 targets per CTA: larger N and short tails
  LS_REG(2, 4, 40);
  LS_REG(1, 4, 40);
  LS_REG(1, 4, 32);
}
#elif LS_INST_GROUP == 5
void ls_register_group5(std::vector<PropKernelInfo>& out) {
  LS_REG(1, 4, 24);
  LS_REG(1, 4, 16);
  LS_REG(1, 4, 8);
  LS_REG(1, 4, 1);
}
#elif LS_INST_GROUP == 6
void ls_register_group6(std::vector<PropKernelInfo>& out) {
  // prior-matrix variants: one target per CTA covers every N up to 20480
  LS_REGP(1, 4, 1, 1);
  LS_REGP(1, 4, 8, 1);
  LS_REGP(1, 4, 16, 1);
  LS_REGP(1, 4, 24, 1);
}
#elif LS_INST_GROUP == 7
void ls_register_group7(std::vector<PropKernelInfo>& out) {
  LS_REGP(1, 4, 32, 1);
  LS_REGP(1, 4, 40, 1);
  LS_REGP(1, 8, 20, 1);
  LS_REGP(8, 4, 16, 1);
}
#elif LS_INST_GROUP == 10
void ls_register_group10(std::vector<PropKernelInfo>& out) {
  // two-CTA clusters: N in (57344, 81920]
  LS_REGH2(4);
  LS_REGH2(8);
}
#elif LS_INST_GROUP == 11
void ls_register_group11(std::vector<PropKernelInfo>& out) {
  // N in (81920, 114688]
  LS_REGH2(12);
  LS_REGH2(13);
  LS_REGH2(16);
}
#elif LS_INST_GROUP == 12
void ls_register_group12(std::vector<PropKernelInfo>& out) {
  // register + shared-memory state, N in (20480, 40960]
  LS_REGH(0);
  LS_REGH(2);
  LS_REGH(4);
  LS_REGH(6);
  LS_REGH(8);
}
#elif LS_INST_GROUP == 13
void ls_register_group13(std::vector<PropKernelInfo>& out) {
  // N in (40960, 57344]
  LS_REGH(10);
  LS_REGH(12);
  LS_REGH(13);
  LS_REGH(14);
  LS_REGH(16);
}
#elif LS_INST_GROUP == 16
void ls_register_group16(std::vector<PropKernelInfo>& out) {
  // prior matrix held as bfloat16 (the BF16 prior format), N up to 20480
  LS_REGP(1, 4, 1, 2);
  LS_REGP(1, 4, 8, 2);
  LS_REGP(1, 4, 16, 2);
  LS_REGP(1, 4, 24, 2);
}
#elif LS_INST_GROUP == 17
void ls_register_group17(std::vector<PropKernelInfo>& out) {
  LS_REGP(1, 4, 32, 2);
  LS_REGP(1, 4, 40, 2);
  LS_REGP(1, 8, 20, 2);
  LS_REGP(8, 4, 16, 2);
}
#elif LS_INST_GROUP == 14
void ls_register_group14(std::vector<PropKernelInfo>& out) {
  // prior matrix (BF16 format), one CTA per target: N in (20480, 53248]
  LS_REGHP(0);
  LS_REGHP(4);
  LS_REGHP(8);
  LS_REGHP(14);
}
#elif LS_INST_GROUP == 15
void ls_register_group15(std::vector<PropKernelInfo>& out) {
  // prior matrix (BF16 format), two-CTA clusters: N in (53248, 106496]
  LS_REGH2P(4);
  LS_REGH2P(8);
  LS_REGH2P(14);
}
#elif LS_INST_GROUP == 8
void ls_register_group8(std::vector<PropKernelInfo>& out) {
  // statistic passes of the adjoint (uniform prior), one target per CTA
  LS_REGS(1, 4, 1);
  LS_REGS(1, 4, 8);
}
#elif LS_INST_GROUP == 9
void ls_register_group9(std::vector<PropKernelInfo>& out) {
  LS_REGS(1, 4, 16);
  LS_REGS(1, 4, 20);
}
#endif
