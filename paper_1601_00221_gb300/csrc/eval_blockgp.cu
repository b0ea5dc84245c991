// eval_blockgp.cu -- BlockGP-style one-dimensional-stack interpreter
// (Sec. 3 and Sec. 4.1 prior art, Robilliard et al.): one block per program,
// the program in shared memory, one fitness case per thread per pass, and a
// per-thread stack array in local memory addressed by a run-time stack
// pointer.  It interprets GP_KIND_RPN programs, basic or with the extended
// functions of Sec. 4.2 (GP_KIND_RPN_EXT), and ignores the static level fields
// of their codes.  Kept as the paper's baseline design.
#include "launch.h"

namespace gpdev {

__global__ void __launch_bounds__(256) eval_blockgp_kernel(FloatArgs a) {
  using namespace gpisa;
  extern __shared__ uint4 prog_s[];  // prog_cap instructions (dynamic)
  __shared__ Partial red_s[32];
  __shared__ int meta_s;
  const int item = blockIdx.x;
  const int rank = item / a.n_chunks;
  if (a.order_count && rank >= *a.order_count) return;  // (uniform over the block)
  const int p = a.order ? a.order[rank] : rank;
  const int chunk = item - rank * a.n_chunks;
  const int tid = threadIdx.x;
  if (tid == 0) {
    int n_instr = -1;
    const int64_t off = a.offsets[p];
    const int32_t len = a.lengths[p];
    if ((off & 3) == 0 && len >= 4) {
      const uint4 h = *reinterpret_cast<const uint4*>(a.programs + off);
      const int n = (int)h.y;
      if (((h.x & 0xffu) == K_RPN || (h.x & 0xffu) == K_RPNX) && (h.x >> 16) == VERSION && n >= 1 &&
          n <= a.prog_cap &&
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
      ok &= valid_instr_ext(K_RPNX, in, a.n_inputs) ? 1 : 0;
    }
    bad = !__syncthreads_and(ok);
  }
  CSum acc = {0.0f, 0.0f};
  uint32_t flags = bad ? FLAG_BAD : 0u;
  const int64_t c_begin = (int64_t)chunk * a.chunk_cases;
  int64_t c_end = c_begin + a.chunk_cases;
  if (c_end > a.n_cases) c_end = a.n_cases;
  float* out_row = a.outputs ? a.outputs + (int64_t)p * a.n_cases : nullptr;
  if (!bad) {
    float stack[GP_LOCAL_STACK];
    for (int64_t c = c_begin + tid; c < c_end; c += blockDim.x) {
      int sp = 0;
      for (int i = 0; i < n_instr && !bad; ++i) {
        const uint4 in = prog_s[i];
        if (in.x >= (uint32_t)RF_NCODES) {  // the extended functions
          if (in.x >= (uint32_t)RPX_IF_BASE) {  // IF: operands on the three top slots
            if (sp < 3) { bad = true; break; }
            const int perm = (int)(in.x - RPX_IF_BASE) / R;
            const int lc = perm / 2, rest0 = (lc == 0) ? 1 : 0, rest1 = (lc == 2) ? 1 : 2;
            const int la = (perm & 1) ? rest1 : rest0, lb = (perm & 1) ? rest0 : rest1;
            const int base = sp - 3;
            const float cv = stack[base + lc];
            stack[base] = (cv != 0.0f) ? stack[base + la] : stack[base + lb];
            sp -= 2;
          } else if (in.x >= (uint32_t)RPX_UN_BASE) {
            if (sp < 1) { bad = true; break; }
            const int fn = (int)(in.x - RPX_UN_BASE) % XU_NOPS;
            const float v = stack[sp - 1];
            stack[sp - 1] = fn == XU_SIN ? sinf(v) : fn == XU_COS ? cosf(v) : fn == XU_EXP ? expf(v)
                                                                              : protected_logf(v);
          } else {
            if (sp < 2) { bad = true; break; }
            const int c = (int)(in.x - RPX_BIN_BASE), op = c % XB_NOPS, opr = (c / XB_NOPS) / R;
            const float top = stack[--sp];
            const float below = stack[sp - 1];
            const float x = opr == 0 ? below : top;
            const float y = opr == 0 ? top : below;
            bool r;
            switch (op) {
              case XB_GT: r = x > y; break;
              case XB_LT: r = x < y; break;
              case XB_EQ: r = x == y; break;
              case XB_AND: r = x != 0.0f && y != 0.0f; break;
              default: r = x != 0.0f || y != 0.0f; break;
            }
            stack[sp - 1] = r ? 1.0f : 0.0f;
          }
          continue;
        }
        const int form = (in.x >> 2) / R, op = in.x & 3;
        if (form == RF_PUSHX || form == RF_PUSHC) {
          if (sp >= GP_LOCAL_STACK) { bad = true; break; }
          stack[sp++] = (form == RF_PUSHX) ? __ldg(a.cases + (int64_t)in.y * a.n_cases + c)
                                           : __uint_as_float(in.y);
        } else {
          if (sp < 2) { bad = true; break; }
          const float top = stack[--sp];
          const float below = stack[sp - 1];
          const float x = (form == RF_OP) ? below : top;
          const float y = (form == RF_OP) ? top : below;
          float r;
          switch (op) {
            case F_ADD: r = __fadd_rn(x, y); break;
            case F_SUB: r = __fsub_rn(x, y); break;
            case F_MUL: r = __fmul_rn(x, y); break;
            default: r = pdiv(x, y); break;
          }
          stack[sp - 1] = r;
        }
      }
      if (bad || sp != 1) { flags |= FLAG_BAD; break; }
      const float o = stack[0];
      if (out_row) out_row[c] = o;
      if (a.want_fitness) {
        const float d = case_error(o, __ldg(a.targets + c), a.fitness_kind);
        if (!(d <= 3.402823466e38f)) flags |= FLAG_NONFINITE;
        csum_add(acc, d);
      }
    }
  }
  block_reduce(acc, flags, red_s, blockDim.x >> 5);
  if (tid == 0) {
    if (flags & FLAG_BAD) atomicOr(a.status, 2 /* GP_ERR_PROGRAM */);
    if (a.want_fitness || (flags & FLAG_BAD))
      finish_program(a.partials, a.counters, p, chunk, a.n_chunks, acc, flags, a.fitness_out,
                     fitness_divisor(a.fitness_kind, a.n_cases));
  }
}

cudaError_t launch_blockgp(const FloatArgs& a, int block, int grid, cudaStream_t s) {
  static std::atomic<size_t> set{0};
  const size_t smem = 16u * (size_t)a.prog_cap;  // the program (no sentinel: the loop counts)
  ensure_dynamic_smem(eval_blockgp_kernel, smem, set);
  eval_blockgp_kernel<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace gpdev
