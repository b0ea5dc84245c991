// eval_float.cuh -- the two-dimensional-stack interpreters for binary32
// programs (prefix S-form trees, postfix RPN trees, register linear GP) with
// the fused fitness reduction.
//
// Paper mapping (Chitty, arXiv:1601.00221):
//   Sec. 3 / Sec. 4.1  one block per (program, chunk of cases); the program is
//                      copied to shared memory once per block, and every warp
//                      reads each instruction with one broadcast load, so the
//                      dispatch jump is warp-uniform and never diverges.
//   Sec. 4             each thread interprets the program once per pass over
//                      K fitness cases (the second dimension of the stack).
//                      Thread t of a warp holds the K consecutive cases
//                      [base + t*K, base + t*K + K): one 16-byte load fetches
//                      four cases and a warp reads 32*K contiguous cases
//                      (the paper strides by the thread count instead; both
//                      keep global loads coalesced).
//   Sec. 5             S-form: only functions are dispatched; operands are an
//                      input, a constant or a stack level.
//   Sec. 6.1 / 6.2     the stack levels are K-wide register vectors; because
//                      the encoder resolves every stack level statically, each
//                      level is a fixed register and no switch on a stack
//                      pointer is needed.
//   Listing 1/2 Sum    per-case |o - y| in binary32, compensated per-thread sums,
//                      block reduction, binary64 sum across blocks.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "isa.h"

namespace gpdev {

using gpisa::R;

// stack depth of the BlockGP-style local-memory interpreter
constexpr int GP_LOCAL_STACK = 64;

struct FloatArgs {
  const uint32_t* programs;
  const int64_t* offsets;
  const int32_t* lengths;
  int32_t n_progs;
  const float* cases;
  int32_t n_inputs;
  int64_t n_cases;
  const float* targets;  // may be null (outputs only)
  double* fitness_out;   // may be null
  float* outputs;        // may be null
  Partial* partials;     // [n_progs * n_chunks] when n_chunks > 1
  unsigned* counters;    // [n_progs] when n_chunks > 1, zero between launches
  int* status;           // program-error status word
  int64_t chunk_cases;   // multiple of blockDim.x * K
  int32_t n_chunks;
  int32_t x_aligned;     // cases + v*n_cases is 16-byte aligned for every v
  int32_t y_aligned;     // targets 16-byte aligned
  int32_t o_aligned;     // outputs + p*n_cases 16-byte aligned for every p
  int32_t want_fitness;  // compute the fitness (targets may be null only if n_cases == 0)
};

// Source of input operands for one pass.  With a single input the K values
// are loaded once per pass into registers; otherwise each input operand is a
// (cached) global load of K consecutive cases.
template <int K, bool XREG>
struct XSrc {
  Vec<K> xv;
  const float* cases;
  int64_t n_cases, c0;
  bool vec_ok;
  __device__ __forceinline__ void get(Vec<K>& d, uint32_t v) const {
    if constexpr (XREG) d = xv;
    else vload<K>(d, cases + (int64_t)v * n_cases, c0, n_cases, vec_ok);
  }
};

// ---------------------------------------------------------------------------
// S-form instruction bodies.
// ---------------------------------------------------------------------------
template <int FORM, int L, int K, bool XREG>
__device__ __forceinline__ void sf_fetch(Vec<K>& a, Vec<K>& b, Vec<K> (&S)[R], const XSrc<K, XREG>& X,
                                         const uint4& in) {
  using namespace gpisa;
  if constexpr (FORM == SF_XX) { X.get(a, in.y); X.get(b, in.z); }
  else if constexpr (FORM == SF_XC) { X.get(a, in.y); vbroadcast<K>(b, __uint_as_float(in.z)); }
  else if constexpr (FORM == SF_CX) { vbroadcast<K>(a, __uint_as_float(in.y)); X.get(b, in.z); }
  else if constexpr (FORM == SF_CC) { vbroadcast<K>(a, __uint_as_float(in.y)); vbroadcast<K>(b, __uint_as_float(in.z)); }
  else if constexpr (FORM == SF_SX) { a = S[L]; X.get(b, in.z); }
  else if constexpr (FORM == SF_XS) { X.get(a, in.y); b = S[L]; }
  else if constexpr (FORM == SF_SC) { a = S[L]; vbroadcast<K>(b, __uint_as_float(in.z)); }
  else if constexpr (FORM == SF_CS) { vbroadcast<K>(a, __uint_as_float(in.y)); b = S[L]; }
  else if constexpr (FORM == SF_SS) { a = S[L]; b = S[(L + 1) % R]; }
  else if constexpr (FORM == SF_SSR) { a = S[(L + 1) % R]; b = S[L]; }
}

template <int FORM, int L, int OP, int K, bool XREG>
__device__ __forceinline__ void sf_exec(Vec<K> (&S)[R], const XSrc<K, XREG>& X, const uint4& in) {
  Vec<K> a, b;
  sf_fetch<FORM, L, K, XREG>(a, b, S, X, in);
  vop<OP, K>(S[L], a, b);
}

// store a division result (or a register-GP result) into level/register `l`
template <int K>
__device__ __forceinline__ void store_level(Vec<K> (&S)[R], int l, const Vec<K>& q) {
  switch (l) {
    case 0: S[0] = q; break;
    case 1: S[1] = q; break;
    case 2: S[2] = q; break;
    case 3: S[3] = q; break;
    case 4: S[4] = q; break;
    case 5: S[5] = q; break;
    case 6: S[6] = q; break;
    default: S[7] = q; break;
  }
}

#define GP_OPS3(M, F, L) M(F, L, 0) M(F, L, 1) M(F, L, 2)
#define GP_LEVELS(M, F) M(F, 0) M(F, 1) M(F, 2) M(F, 3) M(F, 4) M(F, 5) M(F, 6) M(F, 7)
#define GP_LEVELS7(M, F) M(F, 0) M(F, 1) M(F, 2) M(F, 3) M(F, 4) M(F, 5) M(F, 6)

// One pass of an S-form program over K cases per thread.  Returns false on an
// unknown instruction code (validated before the first pass, so unreachable).
template <int K, bool XREG>
__device__ __forceinline__ bool run_sform(const uint4* __restrict__ prog, int n, Vec<K> (&S)[R],
                                          const XSrc<K, XREG>& X) {
  using namespace gpisa;
  Vec<K> ta, tb;
  int dl = 0;
  for (int i = 0; i < n; ++i) {
    const uint4 in = prog[i];
    switch (in.x) {
#define SF_CASE(F, L, OP) \
  case sform_code(F, L, OP): sf_exec<F, L, OP, K, XREG>(S, X, in); continue;
#define SF_DIV(F, L) \
  case sform_code(F, L, F_DIV): sf_fetch<F, L, K, XREG>(ta, tb, S, X, in); dl = L; goto do_div;
#define SF_LEVEL(F, L) GP_OPS3(SF_CASE, F, L) SF_DIV(F, L)
      GP_LEVELS(SF_LEVEL, SF_XX)
      GP_LEVELS(SF_LEVEL, SF_XC)
      GP_LEVELS(SF_LEVEL, SF_CX)
      GP_LEVELS(SF_LEVEL, SF_CC)
      GP_LEVELS(SF_LEVEL, SF_SX)
      GP_LEVELS(SF_LEVEL, SF_XS)
      GP_LEVELS(SF_LEVEL, SF_SC)
      GP_LEVELS(SF_LEVEL, SF_CS)
      GP_LEVELS7(SF_LEVEL, SF_SS)
      GP_LEVELS7(SF_LEVEL, SF_SSR)
#undef SF_LEVEL
#undef SF_DIV
#undef SF_CASE
      case sform_code(SF_MOVX, 0, 0): X.get(S[0], in.y); continue;
      case sform_code(SF_MOVC, 0, 0): vbroadcast<K>(S[0], __uint_as_float(in.y)); continue;
      default: return false;
    }
  do_div:
    vop<F_DIV, K>(ta, ta, tb);
    store_level<K>(S, dl, ta);
  }
  return true;
}

// ---------------------------------------------------------------------------
// RPN (postfix) bodies: push a terminal to level l, or combine l and l+1.
// ---------------------------------------------------------------------------
template <int K, bool XREG>
__device__ __forceinline__ bool run_rpn(const uint4* __restrict__ prog, int n, Vec<K> (&S)[R],
                                        const XSrc<K, XREG>& X) {
  using namespace gpisa;
  Vec<K> ta, tb;
  int dl = 0;
  for (int i = 0; i < n; ++i) {
    const uint4 in = prog[i];
    switch (in.x) {
#define RP_PUSH(F, L) \
  case rpn_code(RF_PUSHX, L, 0): X.get(S[L], in.y); continue; \
  case rpn_code(RF_PUSHC, L, 0): vbroadcast<K>(S[L], __uint_as_float(in.y)); continue;
#define RP_OP(F, L, OP) \
  case rpn_code(RF_OP, L, OP): vop<OP, K>(S[L], S[L], S[L + 1]); continue; \
  case rpn_code(RF_OPR, L, OP): vop<OP, K>(S[L], S[L + 1], S[L]); continue;
#define RP_LEVEL(F, L) GP_OPS3(RP_OP, F, L) \
  case rpn_code(RF_OP, L, F_DIV): ta = S[L]; tb = S[L + 1]; dl = L; goto do_div; \
  case rpn_code(RF_OPR, L, F_DIV): ta = S[L + 1]; tb = S[L]; dl = L; goto do_div;
      GP_LEVELS(RP_PUSH, 0)
      GP_LEVELS7(RP_LEVEL, 0)
#undef RP_LEVEL
#undef RP_OP
#undef RP_PUSH
      default: return false;
    }
  do_div:
    vop<F_DIV, K>(ta, ta, tb);
    store_level<K>(S, dl, ta);
  }
  return true;
}

// ---------------------------------------------------------------------------
// Register linear GP: r[d] = r[a] op r[b]; the code selects (op, a, b), the
// first payload word is d.
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ bool run_linear(const uint4* __restrict__ prog, int n, Vec<K> (&r)[R]) {
  using namespace gpisa;
  Vec<K> t, tb;
  for (int i = 0; i < n; ++i) {
    const uint4 in = prog[i];
    switch (in.x) {
#define LN_CASE(OP, A, B) \
  case lin_code(OP, A, B): vop<OP, K>(t, r[A], r[B]); goto do_store;
#define LN_DIV(A, B) \
  case lin_code(F_DIV, A, B): t = r[A]; tb = r[B]; goto do_div;
#define LN_B(OP, A) LN_CASE(OP, A, 0) LN_CASE(OP, A, 1) LN_CASE(OP, A, 2) LN_CASE(OP, A, 3) \
                    LN_CASE(OP, A, 4) LN_CASE(OP, A, 5) LN_CASE(OP, A, 6) LN_CASE(OP, A, 7)
#define LN_BD(A) LN_DIV(A, 0) LN_DIV(A, 1) LN_DIV(A, 2) LN_DIV(A, 3) LN_DIV(A, 4) LN_DIV(A, 5) \
                 LN_DIV(A, 6) LN_DIV(A, 7)
#define LN_A(OP) LN_B(OP, 0) LN_B(OP, 1) LN_B(OP, 2) LN_B(OP, 3) LN_B(OP, 4) LN_B(OP, 5) \
                 LN_B(OP, 6) LN_B(OP, 7)
      LN_A(F_ADD)
      LN_A(F_SUB)
      LN_A(F_MUL)
      LN_BD(0) LN_BD(1) LN_BD(2) LN_BD(3) LN_BD(4) LN_BD(5) LN_BD(6) LN_BD(7)
#undef LN_A
#undef LN_BD
#undef LN_B
#undef LN_DIV
#undef LN_CASE
      default: return false;
    }
  do_div:
    vop<F_DIV, K>(t, t, tb);
  do_store:
    store_level<K>(r, (int)in.y, t);
  }
  return true;
}

// ---------------------------------------------------------------------------
// Instruction validation (once per block, before the first pass): every code
// known, every input index below n_inputs, every level pair in range.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool valid_instr(uint32_t kind, const uint4& in, int n_inputs) {
  using namespace gpisa;
  const uint32_t nin = (uint32_t)n_inputs;
  if (kind == K_SFORM) {
    if (in.x >= (uint32_t)SF_NCODES) return false;
    const int op = in.x & 3, level = (in.x >> 2) % R, form = (in.x >> 2) / R;
    if ((form == SF_SS || form == SF_SSR) && level + 1 >= R) return false;
    if (form == SF_MOVX || form == SF_MOVC) { if (op != 0 || level != 0) return false; }
    const bool xa = form == SF_XX || form == SF_XC || form == SF_XS || form == SF_MOVX;
    const bool xb = form == SF_XX || form == SF_CX || form == SF_SX;
    if (xa && in.y >= nin) return false;
    if (xb && in.z >= nin) return false;
    return true;
  }
  if (kind == K_RPN) {
    if (in.x >= (uint32_t)RF_NCODES) return false;
    const int op = in.x & 3, level = (in.x >> 2) % R, form = (in.x >> 2) / R;
    if (form == RF_PUSHX || form == RF_PUSHC) { if (op != 0) return false; }
    else if (level + 1 >= R) return false;
    if (form == RF_PUSHX && in.y >= nin) return false;
    return true;
  }
  if (kind == K_LINEAR) return in.x < (uint32_t)LIN_NCODES && in.y < (uint32_t)NREG;
  return false;
}

// ---------------------------------------------------------------------------
// The kernel: block = (program p, chunk of cases).  Shared memory holds the
// program; each warp runs its own sequence of passes.
// ---------------------------------------------------------------------------
template <int K, bool XREG>
__global__ void __launch_bounds__(256) eval_float_kernel(FloatArgs a) {
  using namespace gpisa;
  __shared__ uint4 prog_s[MAX_INSTR];
  __shared__ Partial red_s[32];
  __shared__ int meta_s[2];  // n_instr (or -1 if bad), kind

  const int item = blockIdx.x;
  const int p = item / a.n_chunks;
  const int chunk = item - p * a.n_chunks;
  const int tid = threadIdx.x;

  if (tid == 0) {
    int n_instr = -1, kind = 0;
    const int64_t off = a.offsets[p];
    const int32_t len = a.lengths[p];
    if ((off & 3) == 0 && len >= 4) {
      const uint4 h = *reinterpret_cast<const uint4*>(a.programs + off);
      kind = (int)(h.x & 0xffu);
      const int n = (int)h.y;
      const bool kind_ok = kind == K_SFORM || kind == K_RPN || kind == K_LINEAR;
      const bool ver_ok = (h.x >> 16) == VERSION;
      const bool n_ok = n >= (kind == K_LINEAR ? 0 : 1) && n <= MAX_INSTR && 4 + 4 * (int64_t)n <= len;
      if (kind_ok && ver_ok && n_ok) n_instr = n;
    }
    meta_s[0] = n_instr;
    meta_s[1] = kind;
  }
  __syncthreads();
  int n_instr = meta_s[0];
  const uint32_t kind = (uint32_t)meta_s[1];
  bool bad = n_instr < 0;
  if (!bad) {
    const uint4* g = reinterpret_cast<const uint4*>(a.programs + a.offsets[p]) + 1;
    int ok = 1;
    for (int i = tid; i < n_instr; i += blockDim.x) {
      const uint4 in = g[i];
      prog_s[i] = in;
      ok &= valid_instr(kind, in, a.n_inputs) ? 1 : 0;
    }
    bad = !__syncthreads_and(ok);
  }

  CSum acc = {0.0f, 0.0f};
  uint32_t flags = 0;
  if (bad) {
    flags = FLAG_BAD;
    n_instr = 0;
  }

  const int warp = tid >> 5, lane = tid & 31;
  const int nwarps = blockDim.x >> 5;
  const int64_t c_begin = (int64_t)chunk * a.chunk_cases;
  int64_t c_end = c_begin + a.chunk_cases;
  if (c_end > a.n_cases) c_end = a.n_cases;
  float* out_row = a.outputs ? a.outputs + (int64_t)p * a.n_cases : nullptr;

  if (!bad) {
    for (int64_t wb = c_begin + (int64_t)warp * 32 * K; wb < c_end; wb += (int64_t)nwarps * 32 * K) {
      const int64_t c0 = wb + (int64_t)lane * K;
      const bool full = c0 + K <= a.n_cases;
      XSrc<K, XREG> X;
      X.cases = a.cases;
      X.n_cases = a.n_cases;
      X.c0 = c0;
      X.vec_ok = full && a.x_aligned;
      Vec<K> S[R];
      bool ok;
      if (kind == K_LINEAR) {
#pragma unroll
        for (int v = 0; v < R; ++v) {
          if (v < a.n_inputs) vload<K>(S[v], a.cases + (int64_t)v * a.n_cases, c0, a.n_cases, X.vec_ok);
          else vbroadcast<K>(S[v], 0.0f);
        }
        ok = run_linear<K>(prog_s, n_instr, S);
      } else {
        if constexpr (XREG) vload<K>(X.xv, a.cases, c0, a.n_cases, X.vec_ok);
        ok = (kind == K_SFORM) ? run_sform<K, XREG>(prog_s, n_instr, S, X)
                               : run_rpn<K, XREG>(prog_s, n_instr, S, X);
      }
      if (!ok) flags |= FLAG_BAD;
      if (out_row) vstore<K>(out_row, S[0], c0, a.n_cases, full && a.o_aligned);
      if (a.want_fitness) {
        Vec<K> y;
        vload<K>(y, a.targets, c0, a.n_cases, full && a.y_aligned);
        // pass sum of the K absolute errors, then one compensated add
        float e[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
          float d = fabsf(__fsub_rn(vget<K>(S[0], j), vget<K>(y, j)));
          if (c0 + j >= a.n_cases) d = 0.0f;
          if (!(d <= 3.402823466e38f)) flags |= FLAG_NONFINITE;
          e[j] = d;
        }
#pragma unroll
        for (int w = 1; w < K; w <<= 1)
#pragma unroll
          for (int j = 0; j + w < K; j += 2 * w) e[j] = __fadd_rn(e[j], e[j + w]);
        csum_add(acc, e[0]);
      }
    }
  }

  if (!a.want_fitness && !bad) return;  // outputs only
  block_reduce(acc, flags, red_s, nwarps);
  if (tid == 0) {
    if (flags & FLAG_BAD) atomicOr(a.status, 2 /* GP_ERR_PROGRAM */);
    if (a.want_fitness || bad)
      finish_program(a.partials, a.counters, p, chunk, a.n_chunks, acc, flags, a.fitness_out);
  }
}

// ---------------------------------------------------------------------------
// BlockGP-style one-dimensional stack (Sec. 3, Sec. 4.1 prior art): one case
// per thread per pass, stack array in local memory indexed by a dynamic
// stack pointer.  RPN programs only; the level fields of the codes are
// ignored and the stack pointer is tracked at run time.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) eval_blockgp_kernel(FloatArgs a);

}  // namespace gpdev
