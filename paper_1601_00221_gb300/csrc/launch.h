// launch.h -- host-side launchers of the interpreter kernels (one translation
// unit per K keeps the build parallel).
#pragma once
#include <cuda_runtime.h>

#include "eval_float.cuh"

#include <atomic>

namespace gpdev {
// Raises a kernel's dynamic shared-memory limit the first time a launch
// needs more than the default (static + dynamic > 48 KB needs the opt-in).
template <typename F>
inline void ensure_dynamic_smem(F* kernel, size_t bytes, std::atomic<size_t>& configured) {
  if (bytes <= configured.load(std::memory_order_relaxed)) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  configured.store(bytes, std::memory_order_relaxed);
}
}  // namespace gpdev

namespace gpdev {
struct BoolArgs;
// Float kernels: K in {1,2,4,8}; xreg = the single input is held in registers;
// smem = dynamic shared memory (float_tile_bytes).
cudaError_t launch_float_k1(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                            cudaStream_t s);
cudaError_t launch_float_k2(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                            cudaStream_t s);
cudaError_t launch_float_k4(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                            cudaStream_t s);
cudaError_t launch_float_k8(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                            cudaStream_t s);
// The extended S-form interpreter (the full float function sets), same shapes.
cudaError_t launch_floatx_k1(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                             cudaStream_t s);
cudaError_t launch_floatx_k2(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                             cudaStream_t s);
cudaError_t launch_floatx_k4(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                             cudaStream_t s);
cudaError_t launch_floatx_k8(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                             cudaStream_t s);
// The extended RPN interpreter, same shapes.
cudaError_t launch_floatrx_k1(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                              cudaStream_t s);
cudaError_t launch_floatrx_k2(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                              cudaStream_t s);
cudaError_t launch_floatrx_k4(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                              cudaStream_t s);
cudaError_t launch_floatrx_k8(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                              cudaStream_t s);
// K = 8, stack levels 4..7 in shared memory (S-form only); smem includes them.
cudaError_t launch_float_k8_rl4(const FloatArgs& a, bool xreg, int block, int grid, size_t smem,
                                cudaStream_t s);
cudaError_t launch_blockgp(const FloatArgs& a, int block, int grid, cudaStream_t s);
// Several populations in one launch (the basic interpreters, K in {1,2,4,8}):
// a carries the launch-wide fields (program arrays, fitness measure, tile,
// program buffer, order, the partials and counters spanning all segments).
cudaError_t launch_float_seg_k1(const FloatArgs& a, const SegTable& t, bool xreg, int block, int grid,
                                size_t smem, cudaStream_t s);
cudaError_t launch_float_seg_k2(const FloatArgs& a, const SegTable& t, bool xreg, int block, int grid,
                                size_t smem, cudaStream_t s);
cudaError_t launch_float_seg_k4(const FloatArgs& a, const SegTable& t, bool xreg, int block, int grid,
                                size_t smem, cudaStream_t s);
cudaError_t launch_float_seg_k8(const FloatArgs& a, const SegTable& t, bool xreg, int block, int grid,
                                size_t smem, cudaStream_t s);
// Register programs with the register file in shared memory
// (GP_VARIANT_REGISTER_FILE, eval_linear.cu); smem = the program buffer plus
// linear_rf_bytes(k, block); blocks of at most 256 threads.
size_t linear_rf_bytes(int k, int block);
cudaError_t launch_linear_rf(const FloatArgs& a, int k, int block, int grid, size_t smem, cudaStream_t s);
// The width split's classes (programs reading at most `split` distinct
// inputs: class 0; the rest: class 1), each longest first in order[c * n ..],
// their sizes in counts[0..1]; one block, n bytes of dynamic shared memory
// (n <= 160000), n_inputs <= GP_COMPACT_MAX_INPUTS.
cudaError_t launch_split_by_inputs(const uint32_t* programs, const int64_t* offsets, const int32_t* lengths,
                                   int32_t n, int32_t n_inputs, int32_t split, int32_t* order, int32_t* counts,
                                   cudaStream_t s);
// one block per segment: zero Boolean hit counts, and with `order` write each
// segment's programs longest first into order[prog_begin ..]
cudaError_t launch_segment_prep(const SegTable& t, const int32_t* lengths, int32_t* order, bool zero_hits,
                                cudaStream_t s);
// order[0 .. n) = the programs by decreasing instruction count (from their
// lengths), for FloatArgs::order; one block
cudaError_t launch_order_by_size(const int32_t* lengths, int32_t n, int32_t* order, cudaStream_t s);
// order the blocks by program size when the population fills this many
// blocks per SM (below that every block starts in the first wave anyway) and
// each program sees this many cases (below that the whole evaluation takes
// tens of microseconds and the ordering launch would be a visible part of it)
constexpr int kOrderMinProgsPerSm = 2;
constexpr int64_t kOrderMinCases = 16384;
inline bool order_blocks(int32_t n_progs, int64_t n_cases, int sms) {
  return n_progs >= kOrderMinProgsPerSm * sms && n_cases >= kOrderMinCases;
}
// the automatic case chunk aims at this many blocks per SM: with the programs
// taken longest first, few long blocks beat many short ones (the per-block
// costs dominate, the tail does not)
constexpr int kAutoBlocksPerSm = 16;
// Boolean kernels: K words per thread.
cudaError_t launch_bool(const BoolArgs& a, int k, int block, int grid, size_t smem, cudaStream_t s);
// Boolean, several populations in one launch (hits zeroed by launch_segment_prep)
cudaError_t launch_bool_seg(const BoolArgs& a, const SegTable& t, int k, int block, int grid, size_t smem,
                            cudaStream_t s);
// Boolean, one program per lane over w <= 4 words (one warp per block).
cudaError_t launch_bool_lanes(const BoolArgs& a, int w, int grid, size_t smem, cudaStream_t s);
// Boolean, a warp per program (block / 32 programs per block over one staged
// case set); smem = bool_warps_smem
cudaError_t launch_bool_warps(const BoolArgs& a, int k, int block, int grid, size_t smem, cudaStream_t s);
}  // namespace gpdev
