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
#include "gen_interp.h"
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
  int32_t fitness_kind;  // FIT_SUM_ABS, FIT_MSE or FIT_CLASS
  int32_t prog_cap;      // instructions the block's program buffer holds (gp_config.max_instructions)
  const int32_t* order;  // the program of the i-th (program, chunks) group of blocks, longest
                         // first (launch_order_by_size), or null for 0, 1, 2, ...
  int32_t tile_inputs;   // inputs per case the staged tile holds (<= n_inputs)
  const int32_t* order_count;  // with order: the number of its entries to evaluate (a device
                               // count; blocks of later ranks return at once), or null for all
};

// Several populations in one launch (gp_eval_segments, the serving loop's
// merged launches): segment i is programs [prog_begin, prog_begin + n_progs)
// of the launch's program arrays, evaluated on its own cases, split into its
// own chunks (so each program's result is what it would be in a launch of its
// own), blocks [block_begin, block_begin + n_progs * n_chunks).  The table
// travels as a kernel parameter; segments are laid out in block order.
constexpr int kMaxSegments = 64;  // GP_MAX_SEGMENTS
struct SegDesc {
  const void* cases;     // float [n_inputs][n_cases] or uint32 [n_inputs][n_words]
  const void* targets;   // float [n_cases] or uint32 [n_words]
  void* out;             // double fitness or uint64 hits, [n_progs]
  int64_t n_cases;
  int64_t n_units;       // cases (float) or words (Boolean)
  int64_t chunk;         // cases or words per block
  int64_t partial_begin; // first per-block partial of the segment (float, n_chunks > 1)
  int32_t n_inputs;
  int32_t prog_begin;
  int32_t n_progs;
  int32_t n_chunks;
  int32_t block_begin;
  int32_t aligned;       // float: bit 0 cases, bit 1 targets (16-byte rows); Boolean: both
};
struct SegTable {
  int32_t n;
  int32_t pad;
  SegDesc s[kMaxSegments];
};
// the segment of block `item`: the last whose block_begin is <= item
__device__ __forceinline__ int segment_of(const SegTable* t, int item) {
  int lo = 0, hi = t->n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t->s[mid].block_begin <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Trees whose cases have at most GP_COMPACT_MAX_INPUTS inputs stage only the
// inputs the program reads, at most GP_COMPACT_MAX_LIST of them; otherwise
// (and for register programs) the first inputs are staged in order.
constexpr int GP_COMPACT_MAX_INPUTS = 4096;
constexpr int GP_COMPACT_MAX_LIST = 256;

// which payload words of an instruction are input indices: bit 0 = y,
// bit 1 = z, bit 2 = w (codes already validated)
__device__ __forceinline__ uint32_t input_fields(uint32_t kind, uint32_t code) {
  using namespace gpisa;
  auto bin = [](int form) -> uint32_t {
    switch (form) {
      case SF_XX: return 3u;
      case SF_XC: case SF_XS: case SF_MOVX: case SF_XI: return 1u;
      case SF_CX: case SF_SX: return 2u;
      default: return 0u;
    }
  };
  if (kind == K_RPN || kind == K_RPNX)  // extended codes (>= RF_NCODES) read no input
    return (code < (uint32_t)RF_NCODES && ((code >> 2) / R) == RF_PUSHX) ? 1u : 0u;
  if (code < (uint32_t)SF_NCODES) return bin((int)((code >> 2) / R));
  if (code < (uint32_t)SFX_UN_BASE) return bin(((int)code - SFX_BIN_BASE) / XB_NOPS / R);
  if (code < (uint32_t)SFX_IF_BASE) return ((int)code - SFX_UN_BASE) / XU_NOPS / R == UF_X ? 1u : 0u;
  const int desc = xif_form_desc_fast(((int)code - SFX_IF_BASE) / R);
  return (desc / 25 == 0 ? 1u : 0u) | ((desc / 5) % 5 == 0 ? 2u : 0u) | (desc % 5 == 0 ? 4u : 0u);
}

// ---------------------------------------------------------------------------
// The interpreter loops are generated inline PTX (gen_interp.py): one
// brx.idx jump per instruction straight into the body of its (function,
// operand forms, stack level), stack levels in fixed registers, case pairs in
// f32x2 registers.  These wrappers bind the operands of each block.
//   prog  shared-memory address of instruction 0
//   n     instruction count
//   x     the K input values (single-input programs)
//   tile  shared-memory address of this lane's staged inputs (input v at
//         tile + v * 128 * K bytes)
// Each returns true unless an unknown instruction code was met.
// ---------------------------------------------------------------------------
// register unit of the interpreters' stack operands: a pair of binary32
// cases (one value when K == 1)
template <int K>
struct SfxUnit {
  using type = unsigned long long;  // a pair of binary32 cases
};
template <>
struct SfxUnit<1> {
  using type = float;
};

template <int K>
__device__ __forceinline__ void sfx_unpack(const typename SfxUnit<K>::type* u, float (&v)[K]) {
  if constexpr (K == 1) {
    v[0] = u[0];
  } else {
#pragma unroll
    for (int i = 0; i < K / 2; ++i) {
      v[2 * i] = __uint_as_float((unsigned)(u[i] & 0xffffffffull));
      v[2 * i + 1] = __uint_as_float((unsigned)(u[i] >> 32));
    }
  }
}

template <int K>
__device__ __forceinline__ void sfx_pack(const float (&v)[K], typename SfxUnit<K>::type* u) {
  if constexpr (K == 1) {
    u[0] = v[0];
  } else {
#pragma unroll
    for (int i = 0; i < K / 2; ++i)
      u[i] = ((unsigned long long)__float_as_uint(v[2 * i + 1]) << 32) | __float_as_uint(v[2 * i]);
  }
}

// register units of the whole stack (R levels)
template <int K>
__host__ __device__ constexpr int stack_units() { return R * (K == 1 ? 1 : K / 2); }

#define GP_O1(o) "=f"(o[0])
#define GP_O2(o) "=f"(o[0]), "=f"(o[1])
#define GP_O4(o) GP_O2(o), "=f"(o[2]), "=f"(o[3])
#define GP_O8(o) GP_O4(o), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]), "=f"(o[7])
#define GP_I1(x) "f"(x[0])
#define GP_I2(x) "f"(x[0]), "f"(x[1])
#define GP_I4(x) GP_I2(x), "f"(x[2]), "f"(x[3])
#define GP_I8(x) GP_I4(x), "f"(x[4]), "f"(x[5]), "f"(x[6]), "f"(x[7])

// K >= 2: the stack s (stack_units<K>() units, level l at s[l*H .. l*H+H-1])
// is the caller's; it stays in registers between entries and level 0 is the
// output, unpacked into o.  K = 1: the stack is local to the asm block and
// level 0 comes out in o.
#define GP_TREE_REG(MAC, KK) \
  asm volatile(MAC : GP_STACK_K##KK, "=r"(bad) : "r"(prog), "r"(n), GP_I##KK(x) : "memory")
#define GP_TREE_SMEM(MAC, KK) \
  asm volatile(MAC : GP_STACK_K##KK, "=r"(bad) : "r"(prog), "r"(n), "r"(tile) : "memory")
#define GP_LIN(MAC, KK) \
  asm volatile(MAC : GP_STACK_K##KK, "=r"(bad) : "r"(prog), "r"(n), "r"(tile), "r"(nin) : "memory")
#define GP_TREE_REG1(MAC) \
  asm volatile(MAC : GP_O1(o), "=r"(bad) : "r"(prog), "r"(n), GP_I1(x) : "memory")
#define GP_TREE_SMEM1(MAC) \
  asm volatile(MAC : GP_O1(o), "=r"(bad) : "r"(prog), "r"(n), "r"(tile) : "memory")
#define GP_LIN1(MAC) \
  asm volatile(MAC : GP_O1(o), "=r"(bad) : "r"(prog), "r"(n), "r"(tile), "r"(nin) : "memory")

template <int K, bool XREG, bool RPN>
__device__ __forceinline__ bool run_tree(uint32_t prog, uint32_t n, const float (&x)[K], uint32_t tile,
                                         typename SfxUnit<K>::type (&s)[stack_units<K>()], float (&o)[K]) {
  uint32_t bad;
  if constexpr (XREG && !RPN) {
    if constexpr (K == 1) GP_TREE_REG1(GP_PTX_SFORM_K1_REG);
    else if constexpr (K == 2) GP_TREE_REG(GP_PTX_SFORM_K2_REG, 2);
    else if constexpr (K == 4) GP_TREE_REG(GP_PTX_SFORM_K4_REG, 4);
    else GP_TREE_REG(GP_PTX_SFORM_K8_REG, 8);
  } else if constexpr (XREG && RPN) {
    if constexpr (K == 1) GP_TREE_REG1(GP_PTX_RPN_K1_REG);
    else if constexpr (K == 2) GP_TREE_REG(GP_PTX_RPN_K2_REG, 2);
    else if constexpr (K == 4) GP_TREE_REG(GP_PTX_RPN_K4_REG, 4);
    else GP_TREE_REG(GP_PTX_RPN_K8_REG, 8);
  } else if constexpr (!RPN) {
    if constexpr (K == 1) GP_TREE_SMEM1(GP_PTX_SFORM_K1_SMEM);
    else if constexpr (K == 2) GP_TREE_SMEM(GP_PTX_SFORM_K2_SMEM, 2);
    else if constexpr (K == 4) GP_TREE_SMEM(GP_PTX_SFORM_K4_SMEM, 4);
    else GP_TREE_SMEM(GP_PTX_SFORM_K8_SMEM, 8);
  } else {
    if constexpr (K == 1) GP_TREE_SMEM1(GP_PTX_RPN_K1_SMEM);
    else if constexpr (K == 2) GP_TREE_SMEM(GP_PTX_RPN_K2_SMEM, 2);
    else if constexpr (K == 4) GP_TREE_SMEM(GP_PTX_RPN_K4_SMEM, 4);
    else GP_TREE_SMEM(GP_PTX_RPN_K8_SMEM, 8);
  }
  if constexpr (K >= 2) sfx_unpack<K>(s, o);
  return bad == 0;
}

// S-form with stack levels 4..7 in shared memory (K = 8): `sbase` is this
// lane's spill address (per warp [level][16-byte chunk][lane])
#define GP_TREE_REG_SP(MAC, KK) \
  asm volatile(MAC : GP_O##KK(o), "=r"(bad) : "r"(prog), "r"(n), GP_I##KK(x), "r"(sbase) : "memory")
#define GP_TREE_SMEM_SP(MAC, KK) \
  asm volatile(MAC : GP_O##KK(o), "=r"(bad) : "r"(prog), "r"(n), "r"(tile), "r"(sbase) : "memory")

template <bool XREG>
__device__ __forceinline__ bool run_tree_rl4(uint32_t prog, uint32_t n, const float (&x)[8], uint32_t tile,
                                             uint32_t sbase, float (&o)[8]) {
  uint32_t bad;
  if constexpr (XREG) GP_TREE_REG_SP(GP_PTX_SFORM_K8_REG_RL4, 8);
  else GP_TREE_SMEM_SP(GP_PTX_SFORM_K8_SMEM_RL4, 8);
  return bad == 0;
}

// K = 8, input in registers, S-form: `passes` full warp passes (at least
// one) inside one asm block -- each loads the lane's 8 inputs at x, runs the
// program and adds its cases' errors under fitness measure `fit` to `acc`
// (the pass code's own binary32 steps, below), x and y advancing `stride`
// bytes a pass.
static_assert(FLAG_NONFINITE == 1u, "the generated pass loop sets flag bit 1 for a non-finite pass sum");
static_assert(FIT_SUM_ABS == 0 && FIT_MSE == 1 && FIT_CLASS == 2, "the generated pass loop's fitness codes");
__device__ __forceinline__ bool run_tree_passes(uint32_t prog, uint32_t n, const float* x, const float* y,
                                                uint32_t passes, uint64_t stride, int32_t fit,
                                                typename SfxUnit<8>::type (&s)[stack_units<8>()], CSum& acc,
                                                uint32_t& flags) {
  uint32_t bad;
  asm volatile(GP_PTX_SFORM_K8_REG_PASSES
               : GP_STACK_K8, "=r"(bad), "+f"(acc.s), "+f"(acc.c), "+r"(flags)
               : "r"(prog), "r"(n), "l"(x), "l"(y), "r"(passes), "l"(stride), "r"(fit)
               : "memory");
  return bad == 0;
}

// shared-memory bytes of the levels RL.. of one warp
template <int K, int RL>
__host__ __device__ constexpr int spill_bytes_per_warp() { return (gpisa::R - RL) * 4 * K * 32; }

template <int K>
__device__ __forceinline__ bool run_linear(uint32_t prog, uint32_t n, uint32_t tile, uint32_t nin,
                                           typename SfxUnit<K>::type (&s)[stack_units<K>()], float (&o)[K]) {
  uint32_t bad;
  if constexpr (K == 1) GP_LIN1(GP_PTX_LINEAR_K1);
  else if constexpr (K == 2) GP_LIN(GP_PTX_LINEAR_K2, 2);
  else if constexpr (K == 4) GP_LIN(GP_PTX_LINEAR_K4, 4);
  else GP_LIN(GP_PTX_LINEAR_K8, 8);
  if constexpr (K >= 2) sfx_unpack<K>(s, o);
  return bad == 0;
}

// ---------------------------------------------------------------------------
// Extended S-form (the full float function sets of Sec. 4.2).  The generated
// block keeps the stack in asm operands and returns whenever it meets SIN,
// COS, EXP or LOG, with the operand's K values in t; this loop applies CUDA's
// binary32 function (sinf, cosf, expf: 2 ulp; logf: 1 ulp, documented) and
// enters the block again, which stores t into the level and goes on.  The
// program is warp-uniform, so every exit and the function chosen are too.
// ---------------------------------------------------------------------------
constexpr uint32_t SFX_EXIT = 16;  // status >= SFX_EXIT: 16 + fn * 8 + level


// protected log: 0 at a zero operand (either sign), else the log of |a|
__device__ __forceinline__ float protected_logf(float a) { return a == 0.0f ? 0.0f : logf(fabsf(a)); }

template <int K>
__device__ __forceinline__ void sfx_apply(uint32_t fn, typename SfxUnit<K>::type* t) {
  float v[K];
  sfx_unpack<K>(t, v);
  if (fn == gpisa::XU_SIN) {
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = sinf(v[j]);
  } else if (fn == gpisa::XU_COS) {
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = cosf(v[j]);
  } else if (fn == gpisa::XU_EXP) {
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = expf(v[j]);
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = protected_logf(v[j]);
  }
  sfx_pack<K>(v, t);
}

#define GP_SFX(K_, X_) \
  asm volatile(GP_PTX_SFORMX_K##K_##_##X_ : GP_SFX_OUT_K##K_##_##X_ : GP_SFX_IN_K##K_##_##X_ : "memory")
#define GP_RPX(K_, X_) \
  asm volatile(GP_PTX_RPNX_K##K_##_##X_ : GP_SFX_OUT_K##K_##_##X_ : GP_SFX_IN_K##K_##_##X_ : "memory")

// RPN: the (extended) RPN interpreter, else the (extended) S-form one
// The stack s and the operand t are the caller's, defined once and kept
// across passes like the basic interpreters' stack (every program writes a
// level before reading it; t is written before each exit).
template <int K, bool XREG, bool RPN>
__device__ __forceinline__ bool run_tree_ext(uint32_t prog, const float (&x)[K], uint32_t tile,
                                             typename SfxUnit<K>::type (&s)[stack_units<K>()],
                                             typename SfxUnit<K>::type (&t)[K == 1 ? 1 : K / 2], float (&o)[K]) {
  uint32_t adr = prog, st = 0;
#pragma unroll 1
  for (;;) {
    if constexpr (RPN) {
      if constexpr (XREG) {
        if constexpr (K == 1) GP_RPX(1, REG);
        else if constexpr (K == 2) GP_RPX(2, REG);
        else if constexpr (K == 4) GP_RPX(4, REG);
        else GP_RPX(8, REG);
      } else {
        if constexpr (K == 1) GP_RPX(1, SMEM);
        else if constexpr (K == 2) GP_RPX(2, SMEM);
        else if constexpr (K == 4) GP_RPX(4, SMEM);
        else GP_RPX(8, SMEM);
      }
    } else {
      if constexpr (XREG) {
        if constexpr (K == 1) GP_SFX(1, REG);
        else if constexpr (K == 2) GP_SFX(2, REG);
        else if constexpr (K == 4) GP_SFX(4, REG);
        else GP_SFX(8, REG);
      } else {
        if constexpr (K == 1) GP_SFX(1, SMEM);
        else if constexpr (K == 2) GP_SFX(2, SMEM);
        else if constexpr (K == 4) GP_SFX(4, SMEM);
        else GP_SFX(8, SMEM);
      }
    }
    if (st < SFX_EXIT) break;
    sfx_apply<K>((st - SFX_EXIT) >> 3, t);
  }
  sfx_unpack<K>(s, o);
  return st == 0;
}

// payload c of a division by a constant is the divisor's reciprocal rounded
// to nearest.  Out of line: inlined into every kernel's staging code, the
// rounding sequence cost the extended K = 2 interpreter 10% (measured), and
// it runs only for these instructions, once per block.
static __device__ __noinline__ bool reciprocal_payload_ok(uint32_t b, uint32_t y) {
  return y == __float_as_uint(__frcp_rn(__uint_as_float(b)));
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
    if (form == SF_XI || form == SF_SI || form == SF_CI) {
      // division by a constant with its reciprocal: the divisor (and a
      // constant numerator) in the fast range, payload c its reciprocal
      // rounded to nearest even
      if (op != F_DIV || !div_fast_operand(in.z) || (form == SF_CI && !div_fast_operand(in.y)) ||
          !reciprocal_payload_ok(in.z, in.w))
        return false;
    }
    const bool xa = form == SF_XX || form == SF_XC || form == SF_XS || form == SF_MOVX || form == SF_XI;
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

// the extended S-form's or RPN's codes (supersets of the basic ones)
__device__ __forceinline__ bool valid_instr_ext(uint32_t kind, const uint4& in, int n_inputs) {
  using namespace gpisa;
  const uint32_t nin = (uint32_t)n_inputs;
  if (kind == K_RPN || kind == K_RPNX) {
    if (in.x < (uint32_t)RF_NCODES) return valid_instr(K_RPN, in, n_inputs);
    if (in.x >= (uint32_t)RPX_NCODES) return false;
    if (in.x < (uint32_t)RPX_UN_BASE) return ((in.x - RPX_BIN_BASE) / XB_NOPS) % R + 1 < (uint32_t)R;
    if (in.x < (uint32_t)RPX_IF_BASE) return true;
    return (in.x - RPX_IF_BASE) % R + 2 < (uint32_t)R;
  }
  if (in.x < (uint32_t)SF_NCODES) return valid_instr(K_SFORM, in, n_inputs);
  if (in.x >= (uint32_t)SFX_NCODES) return false;
  if (in.x < (uint32_t)SFX_UN_BASE) {
    const int c = (int)in.x - SFX_BIN_BASE;
    const int level = (c / XB_NOPS) % R, form = (c / XB_NOPS) / R;
    if ((form == SF_SS || form == SF_SSR) && level + 1 >= R) return false;
    const bool xa = form == SF_XX || form == SF_XC || form == SF_XS;
    const bool xb = form == SF_XX || form == SF_CX || form == SF_SX;
    return !(xa && in.y >= nin) && !(xb && in.z >= nin);
  }
  if (in.x < (uint32_t)SFX_IF_BASE) {
    const int uform = ((int)in.x - SFX_UN_BASE) / XU_NOPS / R;
    return !(uform == UF_X && in.y >= nin);
  }
  const int c = (int)in.x - SFX_IF_BASE;
  const int level = c % R, desc = xif_form_desc_fast(c / R);
  const int d[3] = {desc / 25, (desc / 5) % 5, desc % 5};
  const uint32_t pay[3] = {in.y, in.z, in.w};
  int m = 0;
  for (int i = 0; i < 3; ++i) {
    if (d[i] >= 2) ++m;
    if (d[i] == 0 && pay[i] >= nin) return false;
  }
  return level + (m > 0 ? m - 1 : 0) < R;
}

// ---------------------------------------------------------------------------
// The kernel: block = (program p, chunk of cases).  Shared memory holds the
// program; each warp runs its own sequence of passes.
// ---------------------------------------------------------------------------
// EXT: 0 the basic interpreters (S-form, RPN, register GP); 1 the extended
// S-form (K_SFORM, K_SFORMX programs); 2 the extended RPN (K_RPN, K_RPNX).
// One form per kernel: the two extended interpreters in one kernel cost the
// S-form one 6-9% (measured).
// RL < R: stack levels RL.. in shared memory (K = 8, RL = 4; K_SFORM only).
// Up to 512 threads per block at 128 registers: the warps of an SM interpret
// as few distinct programs as possible (every block holds one program).
// SEG: the block's population, cases and outputs come from segment table t
// (the basic interpreters only); otherwise from a.
template <int K, bool XREG, int EXT, int RL, bool SEG>
__device__ __forceinline__ void eval_float_block(const FloatArgs& a, const SegTable* t) {
  using namespace gpisa;
  // dynamic: the program (prog_cap instructions + the end sentinel), then the
  // tiles [warp][slot][32 lanes][K] when staged
  extern __shared__ uint4 dyn_s[];
  uint4* prog_s = dyn_s;
  float4* tile_s = reinterpret_cast<float4*>(dyn_s + a.prog_cap + 1);
  __shared__ Partial red_s[32];
  __shared__ int meta_s[2];  // n_instr (or -1 if bad), kind
  __shared__ uint32_t list_s[GP_COMPACT_MAX_LIST];  // input of each staged slot
  __shared__ uint32_t used_s[GP_COMPACT_MAX_INPUTS / 32];  // bitmap of the inputs read
  __shared__ uint32_t before_s[GP_COMPACT_MAX_INPUTS / 32];  // set bits in earlier words
  __shared__ int n_stage_s;

  const int item = blockIdx.x;
  const int seg = SEG ? segment_of(t, item) : 0;
  // the block's population: the launch's, or its segment's
#define GP_SEG(field, seg_expr) (SEG ? (seg_expr) : a.field)
  // (expressions, not locals: without segments each use reads the kernel
  // parameter, as the single-population kernels always have; locals moved
  // the extended K = 2 staged kernel's code enough to cost it 11%, measured)
#define a_n_cases GP_SEG(n_cases, t->s[seg].n_cases)
#define a_n_inputs GP_SEG(n_inputs, t->s[seg].n_inputs)
#define a_chunk_cases GP_SEG(chunk_cases, t->s[seg].chunk)
#define a_n_chunks GP_SEG(n_chunks, t->s[seg].n_chunks)
#define a_cases GP_SEG(cases, static_cast<const float*>(t->s[seg].cases))
#define a_targets GP_SEG(targets, static_cast<const float*>(t->s[seg].targets))
#define a_x_aligned GP_SEG(x_aligned, (t->s[seg].aligned & 1) != 0)
#define a_y_aligned GP_SEG(y_aligned, (t->s[seg].aligned & 2) != 0)
  const int prog_base = SEG ? t->s[seg].prog_begin : 0;
  const int local = SEG ? item - t->s[seg].block_begin : item;
  const int rank = local / a_n_chunks;
  if (!SEG && a.order_count && rank >= *a.order_count) return;  // (uniform over the block)
  const int p = a.order ? a.order[prog_base + rank] : prog_base + rank;
  const int chunk = local - rank * a_n_chunks;
  const int tid = threadIdx.x;

  if (tid == 0) {
    int n_instr = -1, kind = 0;
    const int64_t off = a.offsets[p];
    const int32_t len = a.lengths[p];
    if ((off & 3) == 0 && len >= 4) {
      const uint4 h = *reinterpret_cast<const uint4*>(a.programs + off);
      kind = (int)(h.x & 0xffu);
      const int n = (int)h.y;
      const bool kind_ok = EXT == 1    ? (kind == K_SFORM || kind == K_SFORMX)
                           : EXT == 2  ? (kind == K_RPN || kind == K_RPNX)
                           : RL < R    ? kind == K_SFORM
                                       : (kind == K_SFORM || kind == K_RPN || kind == K_LINEAR);
      const bool ver_ok = (h.x >> 16) == VERSION;
      const bool n_ok = n >= (kind == K_LINEAR ? 0 : 1) && n <= a.prog_cap && 4 + 4 * (int64_t)n <= len;
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
      if constexpr (EXT) ok &= valid_instr_ext(kind, in, a_n_inputs) ? 1 : 0;
      else ok &= valid_instr(kind, in, a_n_inputs) ? 1 : 0;
    }
    // the interpreters leave through the table entry one past the last code
    if (tid == 0)
      prog_s[n_instr] = make_uint4(EXT == 2 ? RPX_NCODES : EXT == 1 ? SFX_NCODES
                                       : kind == K_SFORM ? SF_NCODES
                                       : kind == K_RPN   ? RF_NCODES
                                                         : LIN_NCODES,
                                   0u, 0u, 0u);
    bad = !__syncthreads_and(ok);
  }

  // Inputs to stage.  A tree stages only the inputs it reads: they are listed
  // in increasing order (slot s holds input list_s[s]) and the program's
  // input payloads, in shared memory, become slots.  Register programs stage
  // their first min(n_inputs, 8) inputs.
  const bool staged = !XREG || (!EXT && kind == K_LINEAR);
  // (the count is read back from shared memory where it is used, so no
  // register holds it across the interpreter loop)
  if (!bad && staged) {
    int n_stage;
    if (XREG || kind == K_LINEAR || a_n_inputs > GP_COMPACT_MAX_INPUTS) {
      // (a kernel with the input in registers stages register programs only)
      n_stage = kind == K_LINEAR ? (a_n_inputs < R ? a_n_inputs : R) : a_n_inputs;
      if (tid == 0) n_stage_s = n_stage;
    } else if constexpr (!XREG) {
      const int nw = (a_n_inputs + 31) >> 5;
      for (int i = tid; i < nw; i += blockDim.x) used_s[i] = 0u;
      __syncthreads();
      for (int i = tid; i < n_instr; i += blockDim.x) {
        const uint4 in = prog_s[i];
        const uint32_t f = input_fields(kind, in.x);
        if (f & 1u) atomicOr(&used_s[in.y >> 5], 1u << (in.y & 31));
        if (f & 2u) atomicOr(&used_s[in.z >> 5], 1u << (in.z & 31));
        if (f & 4u) atomicOr(&used_s[in.w >> 5], 1u << (in.w & 31));
      }
      __syncthreads();
      if (tid == 0) {
        uint32_t c = 0;
        for (int i = 0; i < nw; ++i) {
          before_s[i] = c;
          c += (uint32_t)__popc(used_s[i]);
        }
        n_stage_s = (int)c;
      }
      __syncthreads();
      n_stage = n_stage_s;
      auto slot = [&](uint32_t v) {
        return before_s[v >> 5] + (uint32_t)__popc(used_s[v >> 5] & ((1u << (v & 31)) - 1u));
      };
      if (n_stage > GP_COMPACT_MAX_LIST) {  // too many to list: stage every input in order
        n_stage = a_n_inputs;
        __syncthreads();
        if (tid == 0) n_stage_s = n_stage;
      } else if (n_stage <= a.tile_inputs) {
        for (int i = tid; i < n_instr; i += blockDim.x) {
          uint4 in = prog_s[i];
          const uint32_t f = input_fields(kind, in.x);
          if (f & 1u) in.y = slot(in.y);
          if (f & 2u) in.z = slot(in.z);
          if (f & 4u) in.w = slot(in.w);
          prog_s[i] = in;
        }
        for (int i = tid; i < nw; i += blockDim.x) {
          uint32_t m = used_s[i];
          uint32_t s0 = before_s[i];
          while (m) {
            const int b = __ffs(m) - 1;
            list_s[s0++] = (uint32_t)(i * 32 + b);
            m &= m - 1u;
          }
        }
      }
    }
    __syncthreads();
    if (n_stage > a.tile_inputs) bad = true;  // the tile was sized too small
  }

  CSum acc = {0.0f, 0.0f};
  uint32_t flags = 0;
  if (bad) {
    flags = FLAG_BAD;
    n_instr = 0;
  }

  const int warp = tid >> 5, lane = tid & 31;
  const int nwarps = blockDim.x >> 5;
  const int64_t c_begin = (int64_t)chunk * a_chunk_cases;
  int64_t c_end = c_begin + a_chunk_cases;
  if (c_end > a_n_cases) c_end = a_n_cases;
  float* out_row = (!SEG && a.outputs) ? a.outputs + (int64_t)p * a_n_cases : nullptr;
  const uint32_t prog_addr = (uint32_t)__cvta_generic_to_shared(prog_s);
  // this lane's K staged values of slot v live at tile + v * 32 * K floats
  float* tile = reinterpret_cast<float*>(tile_s) + (size_t)warp * a.tile_inputs * 32 * K + lane * K;
  const uint32_t tile_addr = (uint32_t)__cvta_generic_to_shared(tile);
  // levels RL.. of this lane, after the staged tiles
  uint32_t sbase = 0;
  if constexpr (RL < R)
    sbase = (uint32_t)__cvta_generic_to_shared(tile_s) +
            (uint32_t)(sizeof(float) * (size_t)nwarps * a.tile_inputs * 32 * K) +
            (uint32_t)(warp * spill_bytes_per_warp<K, RL>() + lane * 16);

  // the basic interpreters' stack (K >= 2): defined once here, kept in
  // registers across the passes (every program writes a level before reading
  // it); unused at K = 1
  typename SfxUnit<K>::type stk[stack_units<K>()];
#pragma unroll
  for (int i = 0; i < stack_units<K>(); ++i) stk[i] = 0;
  // the extended interpreters' unary-function operand (unused otherwise)
  typename SfxUnit<K>::type tfn[K == 1 ? 1 : K / 2];
#pragma unroll
  for (int i = 0; i < (K == 1 ? 1 : K / 2); ++i) tfn[i] = 0;

  if (!bad) {
    int64_t wb_first = c_begin + (int64_t)warp * 32 * K;
    if constexpr (XREG && EXT == 0 && RL == R && K == 8) {
      // the warp's full passes (all 32 lanes' cases inside the population)
      // in one interpreter call that loops over them itself; the rest below
      if (kind == K_SFORM && a.want_fitness && !out_row && a_x_aligned && a_y_aligned &&
          (a.fitness_kind == FIT_SUM_ABS || a.fitness_kind == FIT_MSE || a.fitness_kind == FIT_CLASS)) {
        const int64_t stride = (int64_t)nwarps * 32 * K;
        const int64_t last = min(c_end - 1, a_n_cases - (int64_t)32 * K);  // last start of a full pass
        if (last >= wb_first) {
          const int64_t passes = (last - wb_first) / stride + 1;
          const int64_t c0 = wb_first + (int64_t)lane * K;
          if (!run_tree_passes(prog_addr, (uint32_t)n_instr, a_cases + c0, a_targets + c0, (uint32_t)passes,
                               (uint64_t)stride * sizeof(float), a.fitness_kind, stk, acc, flags))
            flags |= FLAG_BAD;
          wb_first += passes * stride;
        }
      }
    }
#pragma unroll 1
    for (int64_t wb = wb_first; wb < c_end; wb += (int64_t)nwarps * 32 * K) {
      const int64_t c0 = wb + (int64_t)lane * K;
      const bool full = c0 + K <= a_n_cases;
      const bool vec_ok = full && a_x_aligned;
      float x[K];
      float o[K];
      if (staged) {
        // a kernel with the input in registers has one input (register programs)
        const int n_stage = XREG ? a_n_inputs : n_stage_s;
        const bool listed = !XREG && kind != K_LINEAR && a_n_inputs <= GP_COMPACT_MAX_INPUTS &&
                            n_stage <= GP_COMPACT_MAX_LIST;
        int v = 0;
        if (vec_ok) {
          // G inputs per step, their loads issued before their stores, so
          // that G global round trips overlap instead of following each other
          constexpr int G = K >= 8 ? 2 : 4;
          for (; v + G <= n_stage; v += G) {
            Vec<K> tv[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
              const int64_t src = listed ? (int64_t)list_s[v + g] : (int64_t)(v + g);
              vload<K>(tv[g], a_cases + src * a_n_cases, c0, a_n_cases, true);
            }
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
              for (int j = 0; j < K; ++j) tile[(v + g) * 32 * K + j] = vget<K>(tv[g], j);
          }
        }
        for (; v < n_stage; ++v) {
          Vec<K> tv;
          const int64_t src = listed ? (int64_t)list_s[v] : (int64_t)v;
          vload<K>(tv, a_cases + src * a_n_cases, c0, a_n_cases, vec_ok);
#pragma unroll
          for (int j = 0; j < K; ++j) tile[v * 32 * K + j] = vget<K>(tv, j);
        }
      }
      if constexpr (XREG) {
        Vec<K> tv;
        vload<K>(tv, a_cases, c0, a_n_cases, vec_ok);
#pragma unroll
        for (int j = 0; j < K; ++j) x[j] = vget<K>(tv, j);
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) x[j] = 0.0f;
      }
      bool ok;
      if constexpr (EXT) {
        ok = run_tree_ext<K, XREG, EXT == 2>(prog_addr, x, tile_addr, stk, tfn, o);
      } else if constexpr (RL < R) {
        static_assert(K == 8 && RL == 4, "shared-memory levels are generated for K = 8, RL = 4");
        ok = run_tree_rl4<XREG>(prog_addr, (uint32_t)n_instr, x, tile_addr, sbase, o);
      } else if (kind == K_LINEAR) {
        ok = run_linear<K>(prog_addr, (uint32_t)n_instr, tile_addr,
                           (uint32_t)(a_n_inputs < R ? a_n_inputs : R), stk, o);
      } else if (kind == K_SFORM) {
        ok = run_tree<K, XREG, false>(prog_addr, (uint32_t)n_instr, x, tile_addr, stk, o);
      } else {
        ok = run_tree<K, XREG, true>(prog_addr, (uint32_t)n_instr, x, tile_addr, stk, o);
      }
      if (!ok) flags |= FLAG_BAD;
      Vec<K> ov;
#pragma unroll
      for (int j = 0; j < K; ++j) vset<K>(ov, j, o[j]);
      if (out_row) vstore<K>(out_row, ov, c0, a_n_cases, full && a.o_aligned);
      if (a.want_fitness) {
        Vec<K> y;
        vload<K>(y, a_targets, c0, a_n_cases, full && a_y_aligned);
        // the K errors (the measure chosen once per pass), the cases past the
        // end masked on the last pass only; then their pass sum and one
        // compensated add
        float e[K];
        if (a.fitness_kind == FIT_SUM_ABS) {
#pragma unroll
          for (int j = 0; j < K; ++j) e[j] = fabsf(__fsub_rn(o[j], vget<K>(y, j)));
        } else if (a.fitness_kind == FIT_MSE) {
#pragma unroll
          for (int j = 0; j < K; ++j) {
            const float d = __fsub_rn(o[j], vget<K>(y, j));
            e[j] = __fmul_rn(d, d);
          }
        } else {
#pragma unroll
          for (int j = 0; j < K; ++j) e[j] = (rintf(o[j]) == vget<K>(y, j)) ? 0.0f : 1.0f;
        }
        if (!full) {
#pragma unroll
          for (int j = 0; j < K; ++j)
            if (c0 + j >= a_n_cases) e[j] = 0.0f;
        }
#pragma unroll
        for (int w = 1; w < K; w <<= 1)
#pragma unroll
          for (int j = 0; j + w < K; j += 2 * w) e[j] = __fadd_rn(e[j], e[j + w]);
        // errors are >= 0: the pass sum is non-finite exactly when an error
        // is, or when finite errors overflow binary32 (the fitness is then
        // +inf as well, not the NaN the compensation term would give)
        if (!(e[0] <= 3.402823466e38f)) flags |= FLAG_NONFINITE;
        csum_add(acc, e[0]);
      }
    }
  }

  if (!a.want_fitness && !bad) return;  // outputs only
  block_reduce(acc, flags, red_s, nwarps);
  if (tid == 0) {
    if (flags & FLAG_BAD) atomicOr(a.status, 2 /* GP_ERR_PROGRAM */);
    if (a.want_fitness || bad) {
      if constexpr (SEG) {  // the segment's partials, counters and outputs
        const SegDesc& d = t->s[seg];
        finish_program(a.partials + d.partial_begin, a.counters + d.prog_begin, p - d.prog_begin, chunk,
                       d.n_chunks, acc, flags, static_cast<double*>(d.out),
                       fitness_divisor(a.fitness_kind, d.n_cases));
      } else {
        finish_program(a.partials, a.counters, p, chunk, a.n_chunks, acc, flags, a.fitness_out,
                       fitness_divisor(a.fitness_kind, a.n_cases));
      }
    }
  }
#undef a_n_cases
#undef a_n_inputs
#undef a_chunk_cases
#undef a_n_chunks
#undef a_cases
#undef a_targets
#undef a_x_aligned
#undef a_y_aligned
#undef GP_SEG
}

// Registers per thread of an interpreter kernel.  Each dispatch waits on an
// indirect jump and its body's dependent arithmetic, so more resident warps
// hide more of that latency: the basic interpreters at K = 4 fit 80 registers
// (24 warps per SM in blocks of 256) and at K = 1, 2 fit 64 (32 warps) with
// no spills, where the compiler's own choice under a 512-thread bound was 121
// to 124 registers (16 warps).  K = 8 needs all 128 (its stack alone is 64)
// and so do the shared-memory stack levels; the extended interpreters keep the
// compiler's choice (their many-input tiles limit residency by shared memory).
// (The 128-register kernels keep the bound of one 512-thread block per SM,
// under which the compiler lays them out as before; a capped kernel takes no
// block minimum, which is what lets K = 4 fit 80 registers without spills.)
template <int K, int EXT, int RL>
__host__ __device__ constexpr int float_reg_cap() {
  return (K == 8 || EXT != 0 || RL < gpisa::R) ? 128 : K == 4 ? 80 : 64;
}
template <int K, int EXT, int RL>
__host__ __device__ constexpr int float_min_blocks() {
  return float_reg_cap<K, EXT, RL>() == 128 ? 1 : 0;
}

template <int K, bool XREG, int EXT = 0, int RL = gpisa::R>
__global__ void __launch_bounds__(512, (float_min_blocks<K, EXT, RL>())) __maxnreg__((float_reg_cap<K, EXT, RL>()))
    eval_float_kernel(FloatArgs a) {
  eval_float_block<K, XREG, EXT, RL, false>(a, nullptr);
}

// several populations in one launch (basic interpreters, all stack levels in
// registers); a.partials / a.counters span every segment
template <int K, bool XREG>
__global__ void __launch_bounds__(512, (float_min_blocks<K, 0, gpisa::R>())) __maxnreg__((float_reg_cap<K, 0, gpisa::R>()))
    eval_float_seg_kernel(FloatArgs a, const __grid_constant__ SegTable t) {
  eval_float_block<K, XREG, 0, gpisa::R, true>(a, &t);
}

// dynamic shared memory of eval_float_kernel: the staged input tiles, for
// tile_inputs inputs per case (the program buffer comes on top of it)
inline size_t float_tile_bytes(int k, int block, int tile_inputs) {
  return sizeof(float) * (size_t)(block / 32) * (size_t)tile_inputs * 32u * (size_t)k;
}
// the program buffer at the start of the dynamic shared memory: prog_cap
// instructions and the end sentinel
inline size_t prog_buffer_bytes(int prog_cap) { return 16u * (size_t)(prog_cap + 1); }

// ---------------------------------------------------------------------------
// BlockGP-style one-dimensional stack (Sec. 3, Sec. 4.1 prior art): one case
// per thread per pass, stack array in local memory indexed by a dynamic
// stack pointer.  RPN programs only; the level fields of the codes are
// ignored and the stack pointer is tracked at run time.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) eval_blockgp_kernel(FloatArgs a);

}  // namespace gpdev
