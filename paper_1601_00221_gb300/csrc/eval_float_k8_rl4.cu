// eval_float_k8_rl4.cu -- the S-form interpreter for K = 8 with stack levels
// 4..7 in shared memory (gp_config.stack_registers = 4).
#include "launch.h"

namespace gpdev {
cudaError_t launch_float_k8_rl4(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                                cudaStream_t s) {
  static std::atomic<size_t> set_reg{0}, set_smem{0};
  if (xreg) {
    ensure_dynamic_smem(eval_float_kernel<8, true, 0, 4>, smem, set_reg);
    eval_float_kernel<8, true, 0, 4><<<grid, block, smem, s>>>(a);
  } else {
    ensure_dynamic_smem(eval_float_kernel<8, false, 0, 4>, smem, set_smem);
    eval_float_kernel<8, false, 0, 4><<<grid, block, smem, s>>>(a);
  }
  return cudaGetLastError();
}
}  // namespace gpdev
