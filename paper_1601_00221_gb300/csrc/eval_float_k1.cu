// eval_float_k1.cu -- instantiation of the binary32 interpreters for K = 1
// fitness cases per thread per pass.
#include "launch.h"

namespace gpdev {
cudaError_t launch_float_k1(const FloatArgs& a, bool xreg, int block, int grid, cudaStream_t s) {
  if (xreg) eval_float_kernel<1, true><<<grid, block, 0, s>>>(a);
  else eval_float_kernel<1, false><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}
}  // namespace gpdev
