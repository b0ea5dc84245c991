// eval_bool.cuh -- two-dimensional-stack interpreter for bit-packed Boolean
// programs (Sec. 4.2: 32 fitness cases per 32-bit word, the sub-machine-code
// parallelism the paper uses for the 20-multiplexer).  Each thread holds K
// consecutive words per pass, so one instruction evaluates 32*K cases per
// thread; stack levels are K-word register vectors at static levels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "isa.h"

namespace gpdev {

struct BoolArgs {
  const uint32_t* programs;
  const int64_t* offsets;
  const int32_t* lengths;
  int32_t n_progs;
  const uint32_t* case_bits;  // [n_inputs][n_words]
  int32_t n_inputs;
  int64_t n_cases;
  int64_t n_words;
  const uint32_t* target_bits;      // may be null
  unsigned long long* hits_out;     // may be null; zeroed before the launch
  uint32_t* out_words;              // may be null: [n_progs][n_words]
  int* status;
  int64_t chunk_words;  // multiple of blockDim.x * K
  int32_t n_chunks;
  int32_t aligned;      // case_bits/target_bits/out_words rows 16-byte aligned
};

template <int K>
struct UVec {
  uint32_t w[K];
};

template <int K>
__device__ __forceinline__ void uload(UVec<K>& d, const uint32_t* __restrict__ src, int64_t w0,
                                      int64_t n, bool vec_ok) {
  if (vec_ok && K >= 2) {
    if constexpr (K == 2) {
      uint2 v = __ldg(reinterpret_cast<const uint2*>(src + w0));
      d.w[0] = v.x; d.w[1] = v.y;
    } else if constexpr (K >= 4) {
#pragma unroll
      for (int i = 0; i < K / 4; ++i) {
        uint4 v = __ldg(reinterpret_cast<const uint4*>(src + w0) + i);
        d.w[4 * i] = v.x; d.w[4 * i + 1] = v.y; d.w[4 * i + 2] = v.z; d.w[4 * i + 3] = v.w;
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j) d.w[j] = (w0 + j < n) ? __ldg(src + w0 + j) : 0u;
  }
}

template <int OP, int K>
__device__ __forceinline__ void bop(UVec<K>& d, const UVec<K>& a, const UVec<K>& b) {
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if constexpr (OP == gpisa::B_AND) d.w[j] = a.w[j] & b.w[j];
    else if constexpr (OP == gpisa::B_OR) d.w[j] = a.w[j] | b.w[j];
    else if constexpr (OP == gpisa::B_NAND) d.w[j] = ~(a.w[j] & b.w[j]);
    else d.w[j] = ~(a.w[j] | b.w[j]);
  }
}

template <int K>
struct BSrc {
  const uint32_t* bits;
  int64_t n_words, w0;
  bool vec_ok;
  __device__ __forceinline__ void get(UVec<K>& d, uint32_t v) const {
    uload<K>(d, bits + (int64_t)v * n_words, w0, n_words, vec_ok);
  }
};

template <int BF, int L, int OP, int K>
__device__ __forceinline__ void bool_bin(UVec<K> (&S)[gpisa::R], const BSrc<K>& X, const uint4& in) {
  using namespace gpisa;
  UVec<K> a, b;
  if constexpr (BF == BF_XX) { X.get(a, in.y); X.get(b, in.z); bop<OP, K>(S[L], a, b); }
  else if constexpr (BF == BF_XS) { X.get(a, in.y); bop<OP, K>(S[L], a, S[L]); }
  else if constexpr (BF == BF_SX) { X.get(b, in.z); bop<OP, K>(S[L], S[L], b); }
  else if constexpr (BF == BF_SS) { bop<OP, K>(S[L], S[L], S[(L + 1) % R]); }
  else { bop<OP, K>(S[L], S[(L + 1) % R], S[L]); }
}

// IF(c, a, b) = (c & a) | (~c & b); operand descriptors from the form index
template <int IFORM, int L, int K>
__device__ __forceinline__ void bool_if(UVec<K> (&S)[gpisa::R], const BSrc<K>& X, const uint4& in) {
  using namespace gpisa;
  constexpr int desc = if_form_desc(IFORM);
  constexpr int dc = desc / 16, da = (desc / 4) % 4, db = desc % 4;
  UVec<K> c, a, b;
  if constexpr (dc == 0) X.get(c, in.y); else c = S[(L + dc - 1) % R];
  if constexpr (da == 0) X.get(a, in.z); else a = S[(L + da - 1) % R];
  if constexpr (db == 0) X.get(b, in.w); else b = S[(L + db - 1) % R];
#pragma unroll
  for (int j = 0; j < K; ++j) S[L].w[j] = (c.w[j] & a.w[j]) | (~c.w[j] & b.w[j]);
}

#define GPB_OPS4(M, F, L) M(F, L, 0) M(F, L, 1) M(F, L, 2) M(F, L, 3)
#define GPB_LEVELS(M, F) M(F, 0) M(F, 1) M(F, 2) M(F, 3) M(F, 4) M(F, 5) M(F, 6) M(F, 7)
#define GPB_LEVELS7(M, F) M(F, 0) M(F, 1) M(F, 2) M(F, 3) M(F, 4) M(F, 5) M(F, 6)

template <int K>
__device__ __forceinline__ bool run_bool(const uint4* __restrict__ prog, int n, UVec<K> (&S)[gpisa::R],
                                         const BSrc<K>& X) {
  using namespace gpisa;
  for (int i = 0; i < n; ++i) {
    const uint4 in = prog[i];
    switch (in.x) {
#define B_CASE(F, L, OP) \
  case bool_bin_code(F, L, OP): bool_bin<F, L, OP, K>(S, X, in); continue;
#define B_LEVEL(F, L) GPB_OPS4(B_CASE, F, L)
      GPB_LEVELS(B_LEVEL, BF_XX)
      GPB_LEVELS(B_LEVEL, BF_XS)
      GPB_LEVELS(B_LEVEL, BF_SX)
      GPB_LEVELS7(B_LEVEL, BF_SS)
      GPB_LEVELS7(B_LEVEL, BF_SSR)
#undef B_LEVEL
#undef B_CASE
#define IF_CASE(F, L) case bool_if_code(F, L): bool_if<F, L, K>(S, X, in); continue;
      GPB_LEVELS(IF_CASE, 0)
      GPB_LEVELS(IF_CASE, 1)
      GPB_LEVELS(IF_CASE, 2)
      GPB_LEVELS(IF_CASE, 3)
      GPB_LEVELS(IF_CASE, 4)
      GPB_LEVELS(IF_CASE, 5)
      GPB_LEVELS(IF_CASE, 6)
      GPB_LEVELS(IF_CASE, 7)
      GPB_LEVELS(IF_CASE, 8)
      GPB_LEVELS(IF_CASE, 9)
      GPB_LEVELS(IF_CASE, 10)
      GPB_LEVELS(IF_CASE, 11)
      GPB_LEVELS(IF_CASE, 12)
      GPB_LEVELS(IF_CASE, 13)
      GPB_LEVELS(IF_CASE, 14)
      GPB_LEVELS(IF_CASE, 15)
#undef IF_CASE
      case BOOL_MOVX: X.get(S[0], in.y); continue;
      default: return false;
    }
  }
  return true;
}

__device__ __forceinline__ bool valid_bool_instr(const uint4& in, int n_inputs) {
  using namespace gpisa;
  const uint32_t nin = (uint32_t)n_inputs;
  if (in.x < (uint32_t)BOOL_IF_BASE) {
    const int level = (in.x >> 2) % R, form = (in.x >> 2) / R;
    if ((form == BF_SS || form == BF_SSR) && level + 1 >= R) return false;
    if ((form == BF_XX || form == BF_XS) && in.y >= nin) return false;
    if ((form == BF_XX || form == BF_SX) && in.z >= nin) return false;
    return true;
  }
  if (in.x < (uint32_t)BOOL_MOVX) {
    const int f = (in.x - BOOL_IF_BASE) / R, level = (in.x - BOOL_IF_BASE) % R;
    const int desc = if_form_desc(f);
    const int dc = desc / 16, da = (desc / 4) % 4, db = desc % 4;
    const int m = (dc > 0) + (da > 0) + (db > 0);
    if (level + (m > 0 ? m - 1 : 0) >= R) return false;
    if ((dc == 0 && in.y >= nin) || (da == 0 && in.z >= nin) || (db == 0 && in.w >= nin)) return false;
    return true;
  }
  if (in.x == (uint32_t)BOOL_MOVX) return in.y < nin;
  return false;
}

template <int K>
__global__ void __launch_bounds__(256) eval_bool_kernel(BoolArgs a) {
  using namespace gpisa;
  __shared__ uint4 prog_s[MAX_INSTR];
  __shared__ unsigned long long red_s[32];
  __shared__ int meta_s;

  const int item = blockIdx.x;
  const int p = item / a.n_chunks;
  const int chunk = item - p * a.n_chunks;
  const int tid = threadIdx.x;

  if (tid == 0) {
    int n_instr = -1;
    const int64_t off = a.offsets[p];
    const int32_t len = a.lengths[p];
    if ((off & 3) == 0 && len >= 4) {
      const uint4 h = *reinterpret_cast<const uint4*>(a.programs + off);
      const int n = (int)h.y;
      if ((h.x & 0xffu) == K_BOOL && (h.x >> 16) == VERSION && n >= 1 && n <= MAX_INSTR &&
          4 + 4 * (int64_t)n <= len)
        n_instr = n;
    }
    meta_s = n_instr;
  }
  __syncthreads();
  int n_instr = meta_s;
  bool bad = n_instr < 0;
  if (!bad) {
    const uint4* g = reinterpret_cast<const uint4*>(a.programs + a.offsets[p]) + 1;
    int ok = 1;
    for (int i = tid; i < n_instr; i += blockDim.x) {
      const uint4 in = g[i];
      prog_s[i] = in;
      ok &= valid_bool_instr(in, a.n_inputs) ? 1 : 0;
    }
    bad = !__syncthreads_and(ok);
  }
  if (bad) {
    if (tid == 0) {
      atomicOr(a.status, 2 /* GP_ERR_PROGRAM */);
      if (a.hits_out) atomicExch(&a.hits_out[p], ~0ull);
    }
    return;
  }

  const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
  const int64_t w_begin = (int64_t)chunk * a.chunk_words;
  int64_t w_end = w_begin + a.chunk_words;
  if (w_end > a.n_words) w_end = a.n_words;
  const uint32_t tail = (uint32_t)(a.n_cases & 31);
  const uint32_t last_mask = tail ? ((1u << tail) - 1u) : 0xffffffffu;
  uint32_t* out_row = a.out_words ? a.out_words + (int64_t)p * a.n_words : nullptr;
  unsigned long long hits = 0;

  for (int64_t wb = w_begin + (int64_t)warp * 32 * K; wb < w_end; wb += (int64_t)nwarps * 32 * K) {
    const int64_t w0 = wb + (int64_t)lane * K;
    const bool full = w0 + K <= a.n_words;
    BSrc<K> X{a.case_bits, a.n_words, w0, full && a.aligned};
    UVec<K> S[R];
    run_bool<K>(prog_s, n_instr, S, X);
    if (out_row) {
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (w0 + j < a.n_words) out_row[w0 + j] = S[0].w[j];
    }
    if (a.target_bits) {
      UVec<K> t;
      uload<K>(t, a.target_bits, w0, a.n_words, full && a.aligned);
      uint32_t h = 0;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const int64_t w = w0 + j;
        uint32_t m = (w < a.n_words - 1) ? 0xffffffffu : (w == a.n_words - 1 ? last_mask : 0u);
        h += __popc(~(S[0].w[j] ^ t.w[j]) & m);
      }
      hits += h;
    }
  }
  if (!a.hits_out || !a.target_bits) return;
  // integer sums are exact, so any order gives the same hit count
  hits = __reduce_add_sync(0xffffffffu, (unsigned)hits);
  if (lane == 0) red_s[warp] = hits;
  __syncthreads();
  if (tid == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < nwarps; ++w) t += red_s[w];
    atomicAdd(&a.hits_out[p], t);
  }
}

}  // namespace gpdev
