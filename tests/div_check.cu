// div_check.cu -- checks the library's protected division (the generated PTX
// sequences GP_PTX_PDIV_K4 / GP_PTX_PDIV_K1 with the slow path decided per
// warp, as the basic interpreters run it, and GP_PTX_PDIV_LANE_K4 /
// GP_PTX_PDIV_LANE_K1 with a per-lane branch, as the extended ones do; and
// the division by a constant with its reciprocal, GP_PTX_PDIVI_K4 / _K1
// with the numerator test and GP_PTX_PDIVI_NT_K4 / _K1 without it, wherever
// the encoder would choose them) against CUDA's correctly rounded division:
// q == (b == 0 ? 1 : a / b) bit for bit, any NaN equal to any NaN.  Every lane of a warp runs the same
// sequence of calls, as the warp decision requires.  Test tool, built by
// tests/test_division.py.
//
// Modes (argv[1]):
//   mant <slice> <nslices>   every pair of significands with a in [1, 2) and
//                            b in [1, 2) and in (-2, -1] (all 2^46 pairs of
//                            each over nslices launches; this run covers
//                            slice `slice` only, or all if slice < 0)
//   rand <n_per_thread> <seed>  random bit patterns over every exponent,
//                            including zeros, subnormals, infinities, NaN
//   exps <n_per_thread> <seed>  random significands under every pair of
//                            exponents (the fast path's range boundaries)
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include <cuda_runtime.h>

#include "gen_interp.h"

__device__ unsigned long long g_bad;
__device__ unsigned long long g_first[3];  // a bits, b bits, got bits

__device__ __forceinline__ float ref_pdiv(float a, float b) {
  return (b == 0.0f) ? 1.0f : __fdiv_rn(a, b);
}

__device__ __forceinline__ bool same(float x, float y) {
  return (__float_as_uint(x) == __float_as_uint(y)) || (x != x && y != y);
}

__device__ __forceinline__ void report(float a, float b, float q) {
  unsigned long long n = atomicAdd(&g_bad, 1ull);
  if (n == 0) {
    g_first[0] = __float_as_uint(a);
    g_first[1] = __float_as_uint(b);
    g_first[2] = __float_as_uint(q);
  }
}

template <bool LANE>
__device__ __forceinline__ void pdiv4(const float (&a)[4], const float (&b)[4], float (&q)[4]) {
  unsigned long long a0, a1, b0, b1, q0, q1;
  float2 t;
  t = make_float2(a[0], a[1]); a0 = *reinterpret_cast<unsigned long long*>(&t);
  t = make_float2(a[2], a[3]); a1 = *reinterpret_cast<unsigned long long*>(&t);
  t = make_float2(b[0], b[1]); b0 = *reinterpret_cast<unsigned long long*>(&t);
  t = make_float2(b[2], b[3]); b1 = *reinterpret_cast<unsigned long long*>(&t);
  if constexpr (LANE)
    asm volatile(GP_PTX_PDIV_LANE_K4 : "=l"(q0), "=l"(q1) : "l"(a0), "l"(a1), "l"(b0), "l"(b1));
  else
    asm volatile(GP_PTX_PDIV_K4 : "=l"(q0), "=l"(q1) : "l"(a0), "l"(a1), "l"(b0), "l"(b1));
  t = *reinterpret_cast<float2*>(&q0); q[0] = t.x; q[1] = t.y;
  t = *reinterpret_cast<float2*>(&q1); q[2] = t.x; q[3] = t.y;
}

template <bool LANE>
__device__ __forceinline__ float pdiv1(float a, float b) {
  float q;
  if constexpr (LANE)
    asm volatile(GP_PTX_PDIV_LANE_K1 : "=f"(q) : "f"(a), "f"(b));
  else
    asm volatile(GP_PTX_PDIV_K1 : "=f"(q) : "f"(a), "f"(b));
  return q;
}

// the division by a constant with its reciprocal (SF_XI / SF_SI: the
// numerators tested, one decision per warp; NT: SF_CI, no test): every lane
// of the warp calls these, with its own b; the results count only where the
// encoder would choose these forms (b, and for NT also a, in the fast range)
__device__ __forceinline__ void pdivi4(const float (&a)[4], float b, float (&q)[4], bool test) {
  unsigned long long a0, a1, q0, q1;
  float2 t;
  const float y = __frcp_rn(b);
  t = make_float2(a[0], a[1]); a0 = *reinterpret_cast<unsigned long long*>(&t);
  t = make_float2(a[2], a[3]); a1 = *reinterpret_cast<unsigned long long*>(&t);
  if (test)
    asm volatile(GP_PTX_PDIVI_K4 : "=l"(q0), "=l"(q1) : "l"(a0), "l"(a1), "f"(b), "f"(y));
  else
    asm volatile(GP_PTX_PDIVI_NT_K4 : "=l"(q0), "=l"(q1) : "l"(a0), "l"(a1), "f"(b), "f"(y));
  t = *reinterpret_cast<float2*>(&q0); q[0] = t.x; q[1] = t.y;
  t = *reinterpret_cast<float2*>(&q1); q[2] = t.x; q[3] = t.y;
}

__device__ __forceinline__ float pdivi1(float a, float b, bool test) {
  float q;
  const float y = __frcp_rn(b);
  if (test)
    asm volatile(GP_PTX_PDIVI_K1 : "=f"(q) : "f"(a), "f"(b), "f"(y));
  else
    asm volatile(GP_PTX_PDIVI_NT_K1 : "=f"(q) : "f"(a), "f"(b), "f"(y));
  return q;
}

__device__ __forceinline__ bool fast_operand(float v) {
  const uint32_t m = __float_as_uint(v) & 0x7fffffffu;
  return m >= 0x26800000u && m <= 0x58800000u;
}

// a[j] / b[0] for j = 0..3 through the pair forms, a[j] / b[j] through the
// scalar ones
__device__ __forceinline__ void check4i(const float (&a)[4], const float (&b)[4]) {
  float q[4], n[4];
  pdivi4(a, b[0], q, true);
  pdivi4(a, b[0], n, false);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float s = pdivi1(a[j], b[j], true);
    const float u = pdivi1(a[j], b[j], false);
    if (fast_operand(b[0])) {
      const float r = ref_pdiv(a[j], b[0]);
      if (!same(q[j], r)) report(a[j], b[0], q[j]);
      if (fast_operand(a[j]) && !same(n[j], r)) report(a[j], b[0], n[j]);
    }
    if (fast_operand(b[j])) {
      const float r = ref_pdiv(a[j], b[j]);
      if (!same(s, r)) report(a[j], b[j], s);
      if (fast_operand(a[j]) && !same(u, r)) report(a[j], b[j], u);
    }
  }
}

__device__ __forceinline__ void check4(const float (&a)[4], const float (&b)[4]) {
  check4i(a, b);
  float q[4], p[4];
  pdiv4<false>(a, b, q);
  pdiv4<true>(a, b, p);
  float s[4], u[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    s[j] = pdiv1<false>(a[j], b[j]);
    u[j] = pdiv1<true>(a[j], b[j]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float r = ref_pdiv(a[j], b[j]);
    if (!same(q[j], r)) report(a[j], b[j], q[j]);
    if (!same(p[j], r)) report(a[j], b[j], p[j]);
    if (!same(s[j], r)) report(a[j], b[j], s[j]);
    if (!same(u[j], r)) report(a[j], b[j], u[j]);
  }
}

// every significand pair: thread = one b significand, loop over a slice of a;
// b with the sign bit `neg` (the pair path takes the reciprocal of -b, so
// both signs reach the reciprocal unit with every significand)
__global__ void k_mant(uint32_t a_begin, uint32_t a_end, uint32_t neg) {
  const uint32_t mb = blockIdx.x * blockDim.x + threadIdx.x;
  if (mb >= (1u << 23)) return;
  const float bv = __uint_as_float(0x3f800000u | mb | (neg << 31));
  const float b[4] = {bv, bv, bv, bv};
  for (uint32_t ma = a_begin; ma < a_end; ma += 4) {
    float a[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = __uint_as_float(0x3f800000u | (ma + j));
    check4(a, b);
  }
}

__device__ __forceinline__ uint32_t xorshift(uint32_t& s) {
  s ^= s << 13; s ^= s >> 17; s ^= s << 5;
  return s;
}

__global__ void k_rand(uint32_t n, uint32_t seed) {
  uint32_t s = seed ^ (0x9E3779B9u * (blockIdx.x * blockDim.x + threadIdx.x + 1));
  for (int i = 0; i < 16; ++i) xorshift(s);
  for (uint32_t it = 0; it < n; ++it) {
    float a[4], b[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t x = xorshift(s), y = xorshift(s);
      // a quarter of the operands get special exponents (0, 255) or zero significands
      const uint32_t sel = xorshift(s);
      if ((sel & 7) == 0) x &= 0x807fffffu;
      if ((sel & 7) == 1) x |= 0x7f800000u;
      if ((sel & 7) == 2) x &= 0xff800000u;
      if (((sel >> 3) & 7) == 0) y &= 0x807fffffu;
      if (((sel >> 3) & 7) == 1) y |= 0x7f800000u;
      if (((sel >> 3) & 7) == 2) y &= 0xff800000u;
      a[j] = __uint_as_float(x);
      b[j] = __uint_as_float(y);
    }
    check4(a, b);
  }
}

// random significands under every exponent pair: block = (ea, eb)
__global__ void k_exps(uint32_t n, uint32_t seed) {
  const uint32_t ea = blockIdx.x, eb = blockIdx.y;
  uint32_t s = seed ^ (0x9E3779B9u * (ea * 256 + eb + 1)) ^ (threadIdx.x * 0x85EBCA6Bu);
  for (int i = 0; i < 8; ++i) xorshift(s);
  for (uint32_t it = 0; it < n; ++it) {
    float a[4], b[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t x = xorshift(s), y = xorshift(s);
      a[j] = __uint_as_float((x & 0x807fffffu) | (ea << 23));
      b[j] = __uint_as_float((y & 0x807fffffu) | (eb << 23));
    }
    check4(a, b);
  }
}

static int finish(const char* what) {
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    printf("%s: CUDA error %s\n", what, cudaGetErrorString(e));
    return 2;
  }
  unsigned long long bad = 0, first[3] = {0, 0, 0};
  cudaMemcpyFromSymbol(&bad, g_bad, sizeof bad);
  cudaMemcpyFromSymbol(first, g_first, sizeof first);
  if (bad) {
    float a, b, q;
    uint32_t ab = (uint32_t)first[0], bb = (uint32_t)first[1], qb = (uint32_t)first[2];
    memcpy(&a, &ab, 4); memcpy(&b, &bb, 4); memcpy(&q, &qb, 4);
    printf("%s: %llu mismatches; first a=%a (0x%08x) b=%a (0x%08x) got %a (0x%08x)\n", what, bad, a, ab, b, bb, q, qb);
    return 1;
  }
  printf("%s: 0 mismatches\n", what);
  return 0;
}

int main(int argc, char** argv) {
  if (argc < 2) {
    fprintf(stderr, "usage: div_check mant <slice> <nslices> | rand <n> <seed> | exps <n> <seed>\n");
    return 3;
  }
  unsigned long long zero = 0;
  cudaMemcpyToSymbol(g_bad, &zero, sizeof zero);
  const char* mode = argv[1];
  if (!strcmp(mode, "mant")) {
    const int slice = atoi(argv[2]), nslices = atoi(argv[3]);
    const uint32_t per = (1u << 23) / (uint32_t)nslices;
    if (per % 4 || per * (uint32_t)nslices != (1u << 23)) { fprintf(stderr, "bad slicing\n"); return 3; }
    for (int s = (slice < 0 ? 0 : slice); s < (slice < 0 ? nslices : slice + 1); ++s) {
      k_mant<<<(1u << 23) / 256, 256>>>(s * per, (s + 1) * per, 0u);
      if (cudaDeviceSynchronize() != cudaSuccess) break;
      k_mant<<<(1u << 23) / 256, 256>>>(s * per, (s + 1) * per, 1u);
      if (cudaDeviceSynchronize() != cudaSuccess) break;
    }
    char what[64];
    snprintf(what, sizeof what, "significand pairs slice %d of %d", slice, nslices);
    return finish(what);
  }
  if (!strcmp(mode, "rand")) {
    k_rand<<<152 * 16, 256>>>((uint32_t)atoi(argv[2]), (uint32_t)atoi(argv[3]));
    return finish("random bit patterns");
  }
  if (!strcmp(mode, "exps")) {
    k_exps<<<dim3(256, 256), 32>>>((uint32_t)atoi(argv[2]), (uint32_t)atoi(argv[3]));
    return finish("all exponent pairs");
  }
  fprintf(stderr, "unknown mode\n");
  return 3;
}
