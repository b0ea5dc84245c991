// launch.h -- host-side launchers of the interpreter kernels (one translation
// unit per K keeps the build parallel).
#pragma once
#include <cuda_runtime.h>

#include "eval_float.cuh"

namespace gpdev {
struct BoolArgs;
// Float kernels: K in {1,2,4,8}; xreg = the single input is held in registers.
cudaError_t launch_float_k1(const FloatArgs& a, bool xreg, int block, int grid, cudaStream_t s);
cudaError_t launch_float_k2(const FloatArgs& a, bool xreg, int block, int grid, cudaStream_t s);
cudaError_t launch_float_k4(const FloatArgs& a, bool xreg, int block, int grid, cudaStream_t s);
cudaError_t launch_float_k8(const FloatArgs& a, bool xreg, int block, int grid, cudaStream_t s);
cudaError_t launch_blockgp(const FloatArgs& a, int block, int grid, cudaStream_t s);
// Boolean kernels: K words per thread.
cudaError_t launch_bool(const BoolArgs& a, int k, int block, int grid, cudaStream_t s);
}  // namespace gpdev
