// eval_float_k4.cu -- instantiation of the binary32 interpreters for K = 4
// fitness cases per thread per pass.
#include "launch.h"

namespace gpdev {
cudaError_t launch_float_k4(const FloatArgs& a, bool xreg, int block, int grid, cudaStream_t s) {
  if (xreg) eval_float_kernel<4, true><<<grid, block, 0, s>>>(a);
  else eval_float_kernel<4, false><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}
}  // namespace gpdev
