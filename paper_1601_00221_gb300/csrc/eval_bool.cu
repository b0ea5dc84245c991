// eval_bool.cu -- instantiations of the bit-packed Boolean interpreter.
#include "eval_bool.cuh"
#include "launch.h"

namespace gpdev {
template <int K, bool COMPACT>
static void launch_kc(const BoolArgs& a, int block, int grid, size_t smem, cudaStream_t s) {
  static std::atomic<size_t> configured{0};
  ensure_dynamic_smem(eval_bool_kernel<K, COMPACT>, smem, configured);
  eval_bool_kernel<K, COMPACT><<<grid, block, smem, s>>>(a);
}
// the listing kernel when a block runs at least four passes (its own check
// decides per block; segments always take it)
template <int K>
static void launch_k(const BoolArgs& a, int block, int grid, size_t smem, cudaStream_t s) {
  if (a.chunk_words >= 4 * (int64_t)block * K) launch_kc<K, true>(a, block, grid, smem, s);
  else launch_kc<K, false>(a, block, grid, smem, s);
}

cudaError_t launch_bool(const BoolArgs& a, int k, int block, int grid, size_t smem, cudaStream_t s) {
  switch (k) {
    case 1: launch_k<1>(a, block, grid, smem, s); break;
    case 2: launch_k<2>(a, block, grid, smem, s); break;
    case 4: launch_k<4>(a, block, grid, smem, s); break;
    default: launch_k<8>(a, block, grid, smem, s); break;
  }
  return cudaGetLastError();
}
template <int K>
static void launch_seg_k(const BoolArgs& a, const SegTable& t, int block, int grid, size_t smem, cudaStream_t s) {
  static std::atomic<size_t> configured{0};
  ensure_dynamic_smem(eval_bool_seg_kernel<K>, smem, configured);
  eval_bool_seg_kernel<K><<<grid, block, smem, s>>>(a, t);
}

cudaError_t launch_bool_seg(const BoolArgs& a, const SegTable& t, int k, int block, int grid, size_t smem,
                            cudaStream_t s) {
  switch (k) {
    case 1: launch_seg_k<1>(a, t, block, grid, smem, s); break;
    case 2: launch_seg_k<2>(a, t, block, grid, smem, s); break;
    case 4: launch_seg_k<4>(a, t, block, grid, smem, s); break;
    default: launch_seg_k<8>(a, t, block, grid, smem, s); break;
  }
  return cudaGetLastError();
}

template <int K>
static void launch_warps_k(const BoolArgs& a, int block, int grid, size_t smem, cudaStream_t s) {
  static std::atomic<size_t> configured{0};
  ensure_dynamic_smem(eval_bool_warps_kernel<K>, smem, configured);
  eval_bool_warps_kernel<K><<<grid, block, smem, s>>>(a);
}

cudaError_t launch_bool_warps(const BoolArgs& a, int k, int block, int grid, size_t smem, cudaStream_t s) {
  switch (k) {
    case 1: launch_warps_k<1>(a, block, grid, smem, s); break;
    case 2: launch_warps_k<2>(a, block, grid, smem, s); break;
    case 4: launch_warps_k<4>(a, block, grid, smem, s); break;
    default: launch_warps_k<8>(a, block, grid, smem, s); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_bool_lanes(const BoolArgs& a, int w, int grid, size_t smem, cudaStream_t s) {
  switch (w) {
    case 1: eval_bool_lanes_kernel<1><<<grid, 32, smem, s>>>(a); break;
    case 2: eval_bool_lanes_kernel<2><<<grid, 32, smem, s>>>(a); break;
    default: eval_bool_lanes_kernel<4><<<grid, 32, smem, s>>>(a); break;
  }
  return cudaGetLastError();
}
}  // namespace gpdev
