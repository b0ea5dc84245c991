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

// The two classes of a width split (one block of 1024 threads): a program
// reading at most `split` distinct inputs goes to class 0, every other (and
// any program whose header is not a float tree's) to class 1; each class is
// written longest first into order[c * n ..], and its size into counts[c].
// Warp w scans programs w, w + 32, ...: its lanes mark the inputs the
// instructions read in the warp's bitmap (n_inputs <= GP_COMPACT_MAX_INPUTS)
// and count them.
__global__ void __launch_bounds__(1024) split_by_inputs_kernel(const uint32_t* __restrict__ programs,
                                                               const int64_t* __restrict__ offsets,
                                                               const int32_t* __restrict__ lengths, int32_t n,
                                                               int32_t n_inputs, int32_t split,
                                                               int32_t* __restrict__ order,
                                                               int32_t* __restrict__ counts) {
  using namespace gpisa;
  constexpr int kWords = GP_COMPACT_MAX_INPUTS / 32;
  __shared__ uint32_t used_s[32][kWords];
  __shared__ int start[2][kPerLane * 32];
  __shared__ int n_class[2];
  extern __shared__ uint8_t cls_s[];  // the class of each program (dynamic: n bytes)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nw = (n_inputs + 31) >> 5;
  for (int p = warp; p < n; p += 32) {
    for (int i = lane; i < nw; i += 32) used_s[warp][i] = 0u;
    __syncwarp();
    int wide = 1;
    const int64_t off = offsets[p];
    const int32_t len = lengths[p];
    if ((off & 3) == 0 && len >= 4) {
      const uint4 h = *reinterpret_cast<const uint4*>(programs + off);
      const uint32_t kind = h.x & 0xffu;
      const int64_t ni = (int64_t)h.y;
      if ((kind == K_SFORM || kind == K_RPN || kind == K_SFORMX || kind == K_RPNX) && 4 + 4 * ni <= len) {
        const uint4* ins = reinterpret_cast<const uint4*>(programs + off) + 1;
        for (int64_t i = lane; i < ni; i += 32) {
          const uint4 in = ins[i];
          const uint32_t f = input_fields(kind, in.x);
          if ((f & 1u) && in.y < (uint32_t)n_inputs) atomicOr(&used_s[warp][in.y >> 5], 1u << (in.y & 31));
          if ((f & 2u) && in.z < (uint32_t)n_inputs) atomicOr(&used_s[warp][in.z >> 5], 1u << (in.z & 31));
          if ((f & 4u) && in.w < (uint32_t)n_inputs) atomicOr(&used_s[warp][in.w >> 5], 1u << (in.w & 31));
        }
        __syncwarp();
        int c = 0;
        for (int i = lane; i < nw; i += 32) c += __popc(used_s[warp][i]);
        c = __reduce_add_sync(0xffffffffu, c);
        wide = c > split ? 1 : 0;
      }
    }
    if (lane == 0) cls_s[p] = (uint8_t)wide;
    __syncwarp();
  }
  for (int i = tid; i < 2 * kPerLane * 32; i += blockDim.x) (&start[0][0])[i] = 0;
  if (tid < 2) n_class[tid] = 0;
  __syncthreads();
  for (int p = tid; p < n; p += blockDim.x) {
    atomicAdd(&start[cls_s[p]][kBuckets - 1 - size_bucket(lengths[p])], 1);
    atomicAdd(&n_class[cls_s[p]], 1);
  }
  __syncthreads();
  if (tid < 64) {  // exclusive prefix sums over each class's (reversed) buckets: warp c, class c
    const int c = tid >> 5, l = tid & 31;
    int sum = 0;
    for (int j = 0; j < kPerLane; ++j) sum += start[c][l * kPerLane + j];
    int before = sum;
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, before, d);
      if (l >= d) before += v;
    }
    before -= sum;
    for (int j = 0; j < kPerLane; ++j) {
      const int v = start[c][l * kPerLane + j];
      start[c][l * kPerLane + j] = before;
      before += v;
    }
  }
  __syncthreads();
  for (int p = tid; p < n; p += blockDim.x) {
    const int c = cls_s[p];
    order[(int64_t)c * n + atomicAdd(&start[c][kBuckets - 1 - size_bucket(lengths[p])], 1)] = p;
  }
  if (tid < 2) counts[tid] = n_class[tid];
}

}  // namespace

cudaError_t launch_split_by_inputs(const uint32_t* programs, const int64_t* offsets, const int32_t* lengths,
                                   int32_t n, int32_t n_inputs, int32_t split, int32_t* order, int32_t* counts,
                                   cudaStream_t s) {
  static std::atomic<size_t> configured{0};
  const size_t smem = (size_t)n;
  ensure_dynamic_smem(split_by_inputs_kernel, smem, configured);
  split_by_inputs_kernel<<<1, 1024, smem, s>>>(programs, offsets, lengths, n, n_inputs, split, order, counts);
  return cudaGetLastError();
}

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
