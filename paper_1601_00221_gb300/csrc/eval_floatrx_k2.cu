// eval_floatrx_k2.cu -- instantiation of the extended RPN interpreter (the
// full float function sets of Sec. 4.2 in postfix form) for K = 2 fitness
// cases per thread per pass.
#include "launch.h"

namespace gpdev {
cudaError_t launch_floatrx_k2(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                              cudaStream_t s) {
  static std::atomic<size_t> set_reg{0}, set_smem{0};
  if (xreg) {
    ensure_dynamic_smem(eval_float_kernel<2, true, 2>, smem, set_reg);
    eval_float_kernel<2, true, 2><<<grid, block, smem, s>>>(a);
  } else {
    ensure_dynamic_smem(eval_float_kernel<2, false, 2>, smem, set_smem);
    eval_float_kernel<2, false, 2><<<grid, block, smem, s>>>(a);
  }
  return cudaGetLastError();
}
}  // namespace gpdev
