// eval_float_seg_k4.cu -- instantiation of the several-populations launch of
// the binary32 interpreters (eval_float_seg_kernel) for K = 4.
#include "launch.h"

namespace gpdev {
cudaError_t launch_float_seg_k4(const FloatArgs& a, const SegTable& t, bool xreg, int block, int grid,
                                size_t smem, cudaStream_t s) {
  static std::atomic<size_t> set_reg{0}, set_smem{0};
  if (xreg) {
    ensure_dynamic_smem(eval_float_seg_kernel<4, true>, smem, set_reg);
    eval_float_seg_kernel<4, true><<<grid, block, smem, s>>>(a, t);
  } else {
    ensure_dynamic_smem(eval_float_seg_kernel<4, false>, smem, set_smem);
    eval_float_seg_kernel<4, false><<<grid, block, smem, s>>>(a, t);
  }
  return cudaGetLastError();
}
}  // namespace gpdev
