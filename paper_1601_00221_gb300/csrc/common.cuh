// common.cuh -- device helpers shared by the interpreters: K-wide binary32
// arithmetic on case pairs, protected division, compensated summation and
// the per-program fitness reduction.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "isa.h"

namespace gpdev {

// ---------------------------------------------------------------------------
// Arithmetic.  Each function node is one binary32 operation rounded to nearest
// even, never fused with another (the library is built with -fmad=false, and
// the explicit _rn forms also forbid contraction).  Pairs of fitness cases use
// the packed f32x2 instructions of sm_100+/sm_103a: one instruction, two
// independent IEEE operations, so the K-wide body of Sec. 6.1 (float2/float4
// "SSE" types, which on the paper's GK104 had no wide ALU behind them) issues
// K/2 instructions here.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long ua = *reinterpret_cast<unsigned long long*>(&a);
  unsigned long long ub = *reinterpret_cast<unsigned long long*>(&b);
  unsigned long long ud;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(ud) : "l"(ua), "l"(ub));
  return *reinterpret_cast<float2*>(&ud);
}

// Protected division: a zero denominator (+0 or -0) gives 1.0f, otherwise the
// correctly rounded IEEE quotient (CUDA's __fdiv_rn, subnormals kept).
__device__ __forceinline__ float pdiv(float a, float b) {
  return (b == 0.0f) ? 1.0f : __fdiv_rn(a, b);
}
__device__ __forceinline__ float2 pdiv2(float2 a, float2 b) {
  return make_float2(pdiv(a.x, b.x), pdiv(a.y, b.y));
}

template <int OP>
__device__ __forceinline__ float2 fop2(float2 a, float2 b) {
  if constexpr (OP == gpisa::F_ADD) return add2(a, b);
  else if constexpr (OP == gpisa::F_SUB) return sub2(a, b);
  else if constexpr (OP == gpisa::F_MUL) return mul2(a, b);
  else return pdiv2(a, b);
}
template <int OP>
__device__ __forceinline__ float fop1(float a, float b) {
  if constexpr (OP == gpisa::F_ADD) return __fadd_rn(a, b);
  else if constexpr (OP == gpisa::F_SUB) return __fsub_rn(a, b);
  else if constexpr (OP == gpisa::F_MUL) return __fmul_rn(a, b);
  else return pdiv(a, b);
}

// K values of one stack level (or one register) of one thread: K/2 packed
// pairs for K >= 2, a scalar for K == 1.
template <int K>
struct Vec {
  float2 p[K / 2];
};
template <>
struct Vec<1> {
  float s;
};

template <int K>
__device__ __forceinline__ void vbroadcast(Vec<K>& d, float c) {
  if constexpr (K == 1) d.s = c;
  else {
#pragma unroll
    for (int i = 0; i < K / 2; ++i) d.p[i] = make_float2(c, c);
  }
}

template <int OP, int K>
__device__ __forceinline__ void vop(Vec<K>& d, const Vec<K>& a, const Vec<K>& b) {
  if constexpr (K == 1) d.s = fop1<OP>(a.s, b.s);
  else {
#pragma unroll
    for (int i = 0; i < K / 2; ++i) d.p[i] = fop2<OP>(a.p[i], b.p[i]);
  }
}

template <int K>
__device__ __forceinline__ float vget(const Vec<K>& v, int j) {
  if constexpr (K == 1) return v.s;
  else return (j & 1) ? v.p[j >> 1].y : v.p[j >> 1].x;
}
template <int K>
__device__ __forceinline__ void vset(Vec<K>& v, int j, float x) {
  if constexpr (K == 1) v.s = x;
  else if (j & 1) v.p[j >> 1].y = x;
  else v.p[j >> 1].x = x;
}

// K consecutive binary32 values starting at element `c0` of `src`; lanes past
// `n` read 0.  `vec_ok` says src + c0 is 16-byte aligned when K >= 4 (8-byte
// when K == 2) and all K values are in range.
template <int K>
__device__ __forceinline__ void vload(Vec<K>& d, const float* __restrict__ src, int64_t c0,
                                      int64_t n, bool vec_ok) {
  if constexpr (K == 1) {
    d.s = (c0 < n) ? __ldg(src + c0) : 0.0f;
  } else {
    if (vec_ok) {
      if constexpr (K == 2) {
        d.p[0] = __ldg(reinterpret_cast<const float2*>(src + c0));
      } else {
#pragma unroll
        for (int i = 0; i < K / 4; ++i) {
          float4 v = __ldg(reinterpret_cast<const float4*>(src + c0) + i);
          d.p[2 * i] = make_float2(v.x, v.y);
          d.p[2 * i + 1] = make_float2(v.z, v.w);
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < K; ++j) vset<K>(d, j, (c0 + j < n) ? __ldg(src + c0 + j) : 0.0f);
    }
  }
}

template <int K>
__device__ __forceinline__ void vstore(float* __restrict__ dst, const Vec<K>& v, int64_t c0,
                                       int64_t n, bool vec_ok) {
  if constexpr (K == 1) {
    if (c0 < n) dst[c0] = v.s;
  } else {
    if (vec_ok) {
      if constexpr (K == 2) {
        *reinterpret_cast<float2*>(dst + c0) = v.p[0];
      } else {
#pragma unroll
        for (int i = 0; i < K / 4; ++i)
          reinterpret_cast<float4*>(dst + c0)[i] =
              make_float4(v.p[2 * i].x, v.p[2 * i].y, v.p[2 * i + 1].x, v.p[2 * i + 1].y);
      }
    } else {
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (c0 + j < n) dst[c0 + j] = vget<K>(v, j);
    }
  }
}

// ---------------------------------------------------------------------------
// Compensated summation (Neumaier's variant of Kahan summation).  All terms
// are non-negative absolute errors, so the relative error of the sum is a few
// units in the last place of binary32 regardless of the number of terms.
// ---------------------------------------------------------------------------
struct CSum {
  float s, c;
};
__device__ __forceinline__ void csum_add(CSum& a, float x) {
  float t = __fadd_rn(a.s, x);
  float big = fmaxf(a.s, x), small = fminf(a.s, x);  // both >= 0
  a.c = __fadd_rn(a.c, __fadd_rn(__fsub_rn(big, t), small));
  a.s = t;
}
// exact error-free merge of two compensated sums (TwoSum on the heads)
__device__ __forceinline__ CSum csum_merge(CSum a, CSum b) {
  float s = __fadd_rn(a.s, b.s);
  float bp = __fsub_rn(s, a.s);
  float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bp)), __fsub_rn(b.s, bp));
  CSum r;
  r.s = s;
  r.c = __fadd_rn(__fadd_rn(a.c, b.c), err);
  return r;
}

// per-block partial of one program over one chunk of cases
struct Partial {
  float s, c;
  uint32_t flags;  // bit 0: a non-finite error; bit 1: malformed program
  uint32_t pad;
};
constexpr uint32_t FLAG_NONFINITE = 1u;
constexpr uint32_t FLAG_BAD = 2u;

// Block-wide reduction of (CSum, flags) in a fixed order: lanes by xor
// butterfly, then warps in index order.  `scratch` holds one entry per warp.
__device__ __forceinline__ void block_reduce(CSum& v, uint32_t& flags, Partial* scratch,
                                             int nwarps) {
  const unsigned full = 0xffffffffu;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    CSum o;
    o.s = __shfl_xor_sync(full, v.s, off);
    o.c = __shfl_xor_sync(full, v.c, off);
    flags |= __shfl_xor_sync(full, flags, off);
    // combine in lane order so every lane holds the same bits
    const int lane = threadIdx.x & 31;
    v = (lane & off) ? csum_merge(o, v) : csum_merge(v, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) scratch[warp] = Partial{v.s, v.c, flags, 0u};
  __syncthreads();
  if (threadIdx.x == 0) {
    CSum t = {scratch[0].s, scratch[0].c};
    uint32_t f = scratch[0].flags;
    for (int w = 1; w < nwarps; ++w) {
      t = csum_merge(t, CSum{scratch[w].s, scratch[w].c});
      f |= scratch[w].flags;
    }
    v = t;
    flags = f;
  }
}

// Writes the block's partial and, in the last block of program p to finish,
// sums all of p's partials in chunk order in binary64 (Sec. 4.1 leaves the
// per-thread results to a later reduction; here it is fused).  Call from
// thread 0 only.
__device__ __forceinline__ void finish_program(Partial* __restrict__ partials,
                                               unsigned* __restrict__ counters, int p,
                                               int chunk, int n_chunks, CSum v, uint32_t flags,
                                               double* __restrict__ fitness_out,
                                               double divisor = 1.0) {
  if (n_chunks == 1) {
    if (fitness_out) {
      double f = ((double)v.s + (double)v.c) / divisor;
      if (flags & FLAG_BAD) f = __longlong_as_double(0x7ff8000000000000ll);
      else if ((flags & FLAG_NONFINITE) || !(f <= 1.7976931348623157e308))  // (a binary32 sum overflowed)
        f = __longlong_as_double(0x7ff0000000000000ll);
      fitness_out[p] = f;
    }
    return;
  }
  Partial* mine = partials + (int64_t)p * n_chunks;
  mine[chunk] = Partial{v.s, v.c, flags, 0u};
  __threadfence();
  unsigned prev = atomicAdd(&counters[p], 1u);
  if (prev != (unsigned)(n_chunks - 1)) return;
  __threadfence();
  double f = 0.0;
  uint32_t fl = 0;
  for (int c = 0; c < n_chunks; ++c) {
    volatile Partial* q = mine + c;
    f += (double)q->s + (double)q->c;
    fl |= q->flags;
  }
  counters[p] = 0u;  // ready for the next launch
  if (fitness_out) {
    f = f / divisor;
    if (fl & FLAG_BAD) f = __longlong_as_double(0x7ff8000000000000ll);
    else if ((fl & FLAG_NONFINITE) || !(f <= 1.7976931348623157e308))  // (a binary32 sum overflowed)
      f = __longlong_as_double(0x7ff0000000000000ll);
    fitness_out[p] = f;
  }
}

// Per-case error of the fitness measures (gp_fitness; Sec. 4.2 parameter
// table): 0 |o - y|, 1 (o - y)^2, 2 a misclassification (the output rounded
// to the nearest integer, ties to even, differs from the label).  Every step
// is one binary32 operation.
constexpr int FIT_SUM_ABS = 0, FIT_MSE = 1, FIT_CLASS = 2;
__device__ __forceinline__ float case_error(float o, float y, int kind) {
  if (kind == FIT_CLASS) return (rintf(o) == y) ? 0.0f : 1.0f;
  const float d = __fsub_rn(o, y);
  return kind == FIT_MSE ? __fmul_rn(d, d) : fabsf(d);
}
// the binary64 divisor of the summed errors
__host__ __device__ __forceinline__ double fitness_divisor(int kind, int64_t n_cases) {
  return (kind == FIT_MSE && n_cases > 0) ? (double)n_cases : 1.0;
}

}  // namespace gpdev
