// eval_bool.cu -- instantiations of the bit-packed Boolean interpreter.
#include "eval_bool.cuh"
#include "launch.h"

namespace gpdev {
cudaError_t launch_bool(const BoolArgs& a, int k, int block, int grid, cudaStream_t s) {
  switch (k) {
    case 1: eval_bool_kernel<1><<<grid, block, 0, s>>>(a); break;
    case 2: eval_bool_kernel<2><<<grid, block, 0, s>>>(a); break;
    case 4: eval_bool_kernel<4><<<grid, block, 0, s>>>(a); break;
    default: eval_bool_kernel<8><<<grid, block, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}
}  // namespace gpdev
