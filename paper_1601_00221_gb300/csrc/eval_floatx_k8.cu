// eval_floatx_k8.cu -- instantiation of the extended S-form interpreter
// (the full float function sets of Sec. 4.2) for K = 8 fitness cases per
// thread per pass.
#include "launch.h"

namespace gpdev {
cudaError_t launch_floatx_k8(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                             cudaStream_t s) {
  static std::atomic<size_t> set_reg{0}, set_smem{0};
  if (xreg) {
    ensure_dynamic_smem(eval_float_kernel<8, true, 1>, smem, set_reg);
    eval_float_kernel<8, true, 1><<<grid, block, smem, s>>>(a);
  } else {
    ensure_dynamic_smem(eval_float_kernel<8, false, 1>, smem, set_smem);
    eval_float_kernel<8, false, 1><<<grid, block, smem, s>>>(a);
  }
  return cudaGetLastError();
}
}  // namespace gpdev
