// ls_prop_inst.cu -- compiled variants of the propagation kernel and their registry.
//
// A variant is (TPW targets per CTA, W warps, KQ quads of 4 donor slots per lane); a CTA covers
// W * 32 / TPW slices of up to 4*KQ donors, so a variant serves N up to 4 * KQ * W * 32 / TPW.
// The host planner picks, for each launch, the variant with the fewest CTA waves x slots per lane.
// The variants are split over translation units (LS_INST_GROUP) so the build compiles them in
// parallel.
#include "ls_internal.h"

namespace {

template <int TPW, int W, int KQ>
cudaError_t launch_prop(const lsk::PropParams& p, int grid, int smem, cudaStream_t s) {
  lsk::ls_prop_kernel<TPW, W, KQ><<<grid, W * 32, smem, s>>>(p);
  return cudaGetLastError();
}

template <int TPW, int W, int KQ>
int smem_prop(int N, int row_words) {
  return lsk::PropCfg<TPW, W, KQ>::layout(N, row_words).total;
}

}  // namespace

#define LS_REG(T, Wp, K) \
  out.push_back(PropKernelInfo{T, Wp, K, (const void*)lsk::ls_prop_kernel<T, Wp, K>, launch_prop<T, Wp, K>, smem_prop<T, Wp, K>})

#if LS_INST_GROUP == 0
void ls_register_group0(std::vector<PropKernelInfo>& out) {
  // 4 targets per CTA: N up to 5120 (tile 4 x N floats in registers, two CTAs per SM)
  LS_REG(4, 4, 40);
  LS_REG(4, 5, 32);
  LS_REG(4, 4, 30);
  LS_REG(4, 4, 20);
}
#elif LS_INST_GROUP == 1
void ls_register_group1(std::vector<PropKernelInfo>& out) {
  // 8 targets per CTA for N up to 2560
  LS_REG(8, 4, 40);
  LS_REG(8, 4, 20);
  LS_REG(8, 4, 10);
  LS_REG(8, 4, 5);
  LS_REG(8, 4, 2);
}
#elif LS_INST_GROUP == 2
void ls_register_group2(std::vector<PropKernelInfo>& out) {
  // 2 or 1 targets per CTA: larger N, short tails, tiny N
  LS_REG(2, 4, 40);
  LS_REG(1, 4, 40);
  LS_REG(1, 4, 20);
  LS_REG(1, 4, 10);
  LS_REG(1, 4, 5);
  LS_REG(1, 4, 1);
}
#endif
