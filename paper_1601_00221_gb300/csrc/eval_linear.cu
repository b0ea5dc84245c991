// eval_linear.cu -- register linear GP with the register file in shared
// memory (GP_VARIANT_REGISTER_FILE).
//
// The register-variant interpreter keeps the eight registers of a register
// program in machine registers: every instruction then needs one jump on
// (function, a, b) and a second on the destination, and the 64 registers of
// the file at K = 8 hold the kernel at 16 warps per multiprocessor.  Here the
// file lives in shared memory, [register][chunk][lane][chunk bytes] per warp
// (a warp's access to one chunk of one register is conflict-free), and an
// instruction is one jump on its function and flags: its operand and
// destination registers are byte offsets in the warp's file, which the block
// writes into its staged copy of the program.  Two values
// stay in machine registers, A (the previous result) and B (a value loaded
// earlier), and the encoder's flags take an operand from either instead of
// the file and skip the store of a result no later instruction reads from
// the file.  Each pass stages the lane's K cases of the first
// min(n_inputs, 8) inputs straight into registers 0.. by asynchronous copies
// (the initial register values of the register machine: r[i] = input i, the
// rest 0), runs the program and reads register 0.  The kernel needs few registers, so shared memory alone
// bounds its warps per multiprocessor.  Fitness is formed and reduced as in
// the other float kernels (per-case error in binary32, compensated per-thread
// sums, warp, block, binary64 across blocks).
#include <cuda_pipeline_primitives.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"

namespace gpdev {
namespace {

template <int K>
struct RF {
  static constexpr int CB = K >= 4 ? 16 : 4 * K;     // bytes per chunk
  static constexpr int NCHUNK = 4 * K / CB;          // chunks per lane per register
  static constexpr int RSTRIDE = NCHUNK * 32 * CB;   // bytes between registers of a warp's file
  static constexpr int WARP_BYTES = gpisa::NREG * RSTRIDE;
};

template <int K>
__device__ __forceinline__ bool run_linear_rf(uint32_t prog, uint32_t base) {
  uint32_t bad;
  if constexpr (K == 1) asm volatile(GP_PTX_LINEAR_RF_K1 : "=r"(bad) : "r"(prog), "r"(base) : "memory");
  else if constexpr (K == 2) asm volatile(GP_PTX_LINEAR_RF_K2 : "=r"(bad) : "r"(prog), "r"(base) : "memory");
  else if constexpr (K == 4) asm volatile(GP_PTX_LINEAR_RF_K4 : "=r"(bad) : "r"(prog), "r"(base) : "memory");
  else asm volatile(GP_PTX_LINEAR_RF_K8 : "=r"(bad) : "r"(prog), "r"(base) : "memory");
  return bad == 0;
}

// blocks of 256 threads per multiprocessor the register budget is sized for:
// the register files (4 K KB per warp) and a program buffer sized to the
// population leave room for 24 warps at K = 8 and 48 at K = 4 or less (78
// registers at K = 8, 40 below; at K = 4 and 2 ptxas spills 16 and 12 bytes,
// and the 48 warps still beat 40 without spills: C4 3106 -> 3176 GPop/s at
// K = 4, measured)
template <int K>
constexpr int rf_min_blocks() { return K == 8 ? 3 : 6; }

template <int K>
__global__ void __launch_bounds__(256, rf_min_blocks<K>()) eval_linear_rf_kernel(FloatArgs a) {
  using namespace gpisa;
  using L = RF<K>;
  extern __shared__ uint4 dyn_s[];
  uint4* prog_s = dyn_s;
  unsigned char* rf_s = reinterpret_cast<unsigned char*>(dyn_s + a.prog_cap + 1);
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
      if ((h.x & 0xffu) == K_LINEAR && (h.x >> 16) == VERSION && n >= 0 && n <= a.prog_cap &&
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
      ok &= valid_instr(K_LINEAR, in, a.n_inputs) ? 1 : 0;
      ok &= in.z < 32u ? 1 : 0;  // the flags (payload b): bits 0..4
    }
    if (tid == 0) prog_s[n_instr] = make_uint4(LIN_NCODES, 0u, 32u, 0u);  // the sentinel: dispatch index 128
    bad = !__syncthreads_and(ok);
    if (!bad) {
      // an operand taken from A or B must be the register that A or B holds:
      // one thread replays the encoder's forward pass on the flags as given
      // (the body's load rules decide what B holds next)
      if (tid == 0) {
        int a_reg = -1, b_reg = -1, good = 1;
        for (int i = 0; i < n_instr; ++i) {
          const uint4 in = prog_s[i];
          const int ra = (int)((in.x >> 3) & 7u), rb = (int)(in.x & 7u), d = (int)in.y;
          const uint32_t sa = in.z & 3u, sb = (in.z >> 2) & 3u;
          good &= (sa == 0u || (sa == 1u && ra == a_reg) || (sa == 2u && ra == b_reg)) ? 1 : 0;
          good &= (sb == 0u || (sb == 1u && rb == a_reg) || (sb == 2u && rb == b_reg)) ? 1 : 0;
          good &= (sa == 0u || sb == 0u) ? 1 : 0;  // (at most one operand held)
          int nb = b_reg;
          if (sa == 0u && sb == 0u) nb = rb;
          else if (sa == 0u && sb == 1u) nb = ra;
          else if (sa == 1u && sb == 0u) nb = rb;
          a_reg = d;
          b_reg = nb == d ? -1 : nb;
        }
        meta_s = good;
      }
      __syncthreads();
      bad = meta_s == 0;
    }
    if (!bad) {
      // the staged program in the interpreter's form: (dispatch index = flags
      // * 4 + function, and the byte offsets in this warp's register file of
      // the destination, operand a and operand b), so that a dispatch needs
      // no decoding; the sentinel's index is 128
      for (int i = tid; i < n_instr; i += blockDim.x) {
        const uint4 in = prog_s[i];
        prog_s[i] = make_uint4((in.z << 2) | ((in.x >> 6) & 3u), in.y * (uint32_t)L::RSTRIDE,
                               ((in.x >> 3) & 7u) * (uint32_t)L::RSTRIDE, (in.x & 7u) * (uint32_t)L::RSTRIDE);
      }
      if (tid == 0) prog_s[n_instr] = make_uint4(128u, 0u, 0u, 0u);
      __syncthreads();
    }
  }

  CSum acc = {0.0f, 0.0f};
  uint32_t flags = bad ? FLAG_BAD : 0u;
  const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
  const int nin = a.n_inputs < NREG ? a.n_inputs : NREG;
  unsigned char* mine = rf_s + (size_t)warp * L::WARP_BYTES + lane * L::CB;
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(mine);
  const uint32_t prog_addr = (uint32_t)__cvta_generic_to_shared(prog_s);
  const int64_t c_begin = (int64_t)chunk * a.chunk_cases;
  int64_t c_end = c_begin + a.chunk_cases;
  if (c_end > a.n_cases) c_end = a.n_cases;
  float* out_row = a.outputs ? a.outputs + (int64_t)p * a.n_cases : nullptr;

  if (!bad) {
#pragma unroll 1
    for (int64_t wb = c_begin + (int64_t)warp * 32 * K; wb < c_end; wb += (int64_t)nwarps * 32 * K) {
      const int64_t c0 = wb + (int64_t)lane * K;
      const bool full = c0 + K <= a.n_cases;
      // registers 0 .. nin-1 <- inputs, the rest 0 (this lane's chunks only)
      if (full && a.x_aligned) {
        for (int v = 0; v < nin; ++v) {
          const float* src = a.cases + (int64_t)v * a.n_cases + c0;
#pragma unroll
          for (int q = 0; q < L::NCHUNK; ++q)
            __pipeline_memcpy_async(mine + v * L::RSTRIDE + q * 32 * L::CB, src + q * (L::CB / 4), L::CB);
        }
        __pipeline_commit();
      } else {
        for (int v = 0; v < nin; ++v)
#pragma unroll
          for (int j = 0; j < K; ++j) {
            const int64_t c = c0 + j;
            const float x = c < a.n_cases ? __ldg(a.cases + (int64_t)v * a.n_cases + c) : 0.0f;
            *reinterpret_cast<float*>(mine + v * L::RSTRIDE + (j / (L::CB / 4)) * 32 * L::CB +
                                      (j % (L::CB / 4)) * 4) = x;
          }
      }
      for (int v = nin; v < NREG; ++v)
#pragma unroll
        for (int q = 0; q < L::NCHUNK; ++q)
          for (int w = 0; w < L::CB / 4; ++w)
            reinterpret_cast<float*>(mine + v * L::RSTRIDE + q * 32 * L::CB)[w] = 0.0f;
      if (full && a.x_aligned) __pipeline_wait_prior(0);
      if (!run_linear_rf<K>(prog_addr, base)) flags |= FLAG_BAD;
      float o[K];  // register 0, one vector load per chunk
      if constexpr (K >= 4) {
#pragma unroll
        for (int q = 0; q < L::NCHUNK; ++q) {
          const float4 v = *reinterpret_cast<const float4*>(mine + q * 32 * L::CB);
          o[4 * q] = v.x; o[4 * q + 1] = v.y; o[4 * q + 2] = v.z; o[4 * q + 3] = v.w;
        }
      } else if constexpr (K == 2) {
        const float2 v = *reinterpret_cast<const float2*>(mine);
        o[0] = v.x; o[1] = v.y;
      } else {
        o[0] = *reinterpret_cast<const float*>(mine);
      }
      if (out_row) {
        Vec<K> ov;
#pragma unroll
        for (int j = 0; j < K; ++j) vset<K>(ov, j, o[j]);
        vstore<K>(out_row, ov, c0, a.n_cases, full && a.o_aligned);
      }
      if (a.want_fitness) {
        Vec<K> y;
        vload<K>(y, a.targets, c0, a.n_cases, full && a.y_aligned);
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
            if (c0 + j >= a.n_cases) e[j] = 0.0f;
        }
#pragma unroll
        for (int w = 1; w < K; w <<= 1)
#pragma unroll
          for (int j = 0; j + w < K; j += 2 * w) e[j] = __fadd_rn(e[j], e[j + w]);
        if (!(e[0] <= 3.402823466e38f)) flags |= FLAG_NONFINITE;
        csum_add(acc, e[0]);
      }
    }
  }
  if (!a.want_fitness && !bad) return;  // outputs only
  block_reduce(acc, flags, red_s, nwarps);
  if (tid == 0) {
    if (flags & FLAG_BAD) atomicOr(a.status, 2 /* GP_ERR_PROGRAM */);
    if (a.want_fitness || bad)
      finish_program(a.partials, a.counters, p, chunk, a.n_chunks, acc, flags, a.fitness_out,
                     fitness_divisor(a.fitness_kind, a.n_cases));
  }
}

template <int K>
cudaError_t launch_k(const FloatArgs& a, int block, int grid, size_t smem, cudaStream_t s) {
  static std::atomic<size_t> configured{0};
  ensure_dynamic_smem(eval_linear_rf_kernel<K>, smem, configured);
  eval_linear_rf_kernel<K><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t linear_rf_bytes(int k, int block) {
  return (size_t)(block / 32) * gpisa::NREG * 32u * 4u * (size_t)k;
}

cudaError_t launch_linear_rf(const FloatArgs& a, int k, int block, int grid, size_t smem, cudaStream_t s) {
  switch (k) {
    case 1: return launch_k<1>(a, block, grid, smem, s);
    case 2: return launch_k<2>(a, block, grid, smem, s);
    case 4: return launch_k<4>(a, block, grid, smem, s);
    default: return launch_k<8>(a, block, grid, smem, s);
  }
}

}  // namespace gpdev
