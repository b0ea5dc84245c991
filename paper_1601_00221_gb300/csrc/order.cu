// order.cu -- the order in which the evaluation kernels take the programs:
// longest first.
//
// A block evaluates one (program, chunk of cases) pair and the hardware
// starts blocks in index order.  Programs of a population differ in length
// by two orders of magnitude (ramped half-and-half trees of depth 2 to 8), so
// in the caller's order long programs land in the last wave and the GPU idles
// behind them.  Taking the programs longest first (a counting sort of the
// instruction counts, read from the program lengths) leaves only short blocks
// for the end, the classic longest-processing-time schedule.  Results do not
// depend on the order: each program's partial sums are combined in chunk
// order by whichever block finishes last.  Programs of equal length keep no
// particular order among themselves.
#include <cuda_runtime.h>
#include <stdint.h>

#include "isa.h"
#include "launch.h"

namespace gpdev {
namespace {

// instruction counts 0 .. MAX_INSTR (longer lengths share the last bucket)
constexpr int kBuckets = gpisa::MAX_INSTR + 1;
constexpr int kPerLane = (kBuckets + 31) / 32;

__device__ __forceinline__ int size_bucket(int32_t len) {
  // an encoded program: a 4-word header, then 4 words per instruction
  const int n = len < 4 ? 0 : (len - 4) >> 2;
  return n < kBuckets ? n : kBuckets - 1;
}

// order[base + i], i = 0 .. n: the programs base .. base + n by decreasing
// instruction count (one block)
__device__ __forceinline__ void order_range(const int32_t* __restrict__ lengths, int32_t base, int32_t n,
                                            int32_t* __restrict__ order, int* start) {
  const int tid = threadIdx.x;
  for (int i = tid; i < kPerLane * 32; i += blockDim.x) start[i] = 0;
  __syncthreads();
  for (int p = tid; p < n; p += blockDim.x) atomicAdd(&start[kBuckets - 1 - size_bucket(lengths[base + p])], 1);
  __syncthreads();
  if (tid < 32) {  // exclusive prefix sum over the (reversed) buckets: lane l owns kPerLane of them
    int sum = 0;
    for (int j = 0; j < kPerLane; ++j) sum += start[tid * kPerLane + j];
    int before = sum;
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, before, d);
      if (tid >= d) before += v;
    }
    before -= sum;
    for (int j = 0; j < kPerLane; ++j) {
      const int c = start[tid * kPerLane + j];
      start[tid * kPerLane + j] = before;
      before += c;
    }
  }
  __syncthreads();
  for (int p = tid; p < n; p += blockDim.x)
    order[base + atomicAdd(&start[kBuckets - 1 - size_bucket(lengths[base + p])], 1)] = base + p;
}

__global__ void __launch_bounds__(1024) order_by_size_kernel(const int32_t* __restrict__ lengths, int32_t n,
                                                             int32_t* __restrict__ order) {
  __shared__ int start[kPerLane * 32];  // bucket b at start[kBuckets - 1 - b]: longest first
  order_range(lengths, 0, n, order, start);
}

// One block per segment of a several-populations launch: zero the segment's
// hit counts (Boolean, which the kernel accumulates) and, with `order`, take
// the segment's programs longest first.
__global__ void __launch_bounds__(1024) segment_prep_kernel(const __grid_constant__ SegTable t,
                                                            const int32_t* __restrict__ lengths,
                                                            int32_t* __restrict__ order, int zero_hits) {
  __shared__ int start[kPerLane * 32];
  const SegDesc& d = t.s[blockIdx.x];
  if (zero_hits)
    for (int i = threadIdx.x; i < d.n_progs; i += blockDim.x) static_cast<unsigned long long*>(d.out)[i] = 0ull;
  if (order) order_range(lengths, d.prog_begin, d.n_progs, order, start);
}

}  // namespace

cudaError_t launch_order_by_size(const int32_t* lengths, int32_t n, int32_t* order, cudaStream_t s) {
  order_by_size_kernel<<<1, 1024, 0, s>>>(lengths, n, order);
  return cudaGetLastError();
}

cudaError_t launch_segment_prep(const SegTable& t, const int32_t* lengths, int32_t* order, bool zero_hits,
                                cudaStream_t s) {
  segment_prep_kernel<<<t.n, 1024, 0, s>>>(t, lengths, order, zero_hits ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace gpdev
