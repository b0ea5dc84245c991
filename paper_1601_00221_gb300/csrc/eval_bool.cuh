// eval_bool.cuh -- two-dimensional-stack interpreter for bit-packed Boolean
// programs (Sec. 4.2: 32 fitness cases per 32-bit word, the sub-machine-code
// parallelism the paper uses for the 20-multiplexer).  Each thread holds K
// consecutive words per pass, so one instruction evaluates 32*K cases per
// thread; stack levels are K-word register vectors at static levels.
#pragma once
#include <cuda_pipeline_primitives.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "eval_float.cuh"
#include "gen_interp.h"
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
  const int32_t* order;  // programs longest first (launch_order_by_size), or null
  int32_t prog_cap;      // instructions the block's program buffer holds (gp_config.max_instructions)
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

// The interpreter loop is generated inline PTX (gen_interp.py): stack levels
// are K-word registers at static levels, every function is one lop3 per word.
#define GP_BO1(o) "=r"(o[0])
#define GP_BO2(o) "=r"(o[0]), "=r"(o[1])
#define GP_BO4(o) GP_BO2(o), "=r"(o[2]), "=r"(o[3])
#define GP_BO8(o) GP_BO4(o), "=r"(o[4]), "=r"(o[5]), "=r"(o[6]), "=r"(o[7])
#define GP_BOOL_ASM(MAC, KK) \
  asm volatile(MAC : GP_BO##KK(o), "=r"(bad) : "r"(prog), "r"(n), "r"(tile) : "memory")

template <int K>
__device__ __forceinline__ bool run_bool(uint32_t prog, uint32_t n, uint32_t tile, uint32_t (&o)[K]) {
  uint32_t bad;
  if constexpr (K == 1) GP_BOOL_ASM(GP_PTX_BOOL_K1, 1);
  else if constexpr (K == 2) GP_BOOL_ASM(GP_PTX_BOOL_K2, 2);
  else if constexpr (K == 4) GP_BOOL_ASM(GP_PTX_BOOL_K4, 4);
  else GP_BOOL_ASM(GP_PTX_BOOL_K8, 8);
  return bad == 0;
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
    const int desc = if_form_desc_fast(f);
    const int dc = desc / 16, da = (desc / 4) % 4, db = desc % 4;
    const int m = (dc > 0) + (da > 0) + (db > 0);
    if (level + (m > 0 ? m - 1 : 0) >= R) return false;
    if ((dc == 0 && in.y >= nin) || (da == 0 && in.z >= nin) || (db == 0 && in.w >= nin)) return false;
    return true;
  }
  if (in.x == (uint32_t)BOOL_MOVX) return in.y < nin;
  return false;
}

// which payload words of a (validated) Boolean instruction are input
// indices: bit 0 = y, bit 1 = z, bit 2 = w
__device__ __forceinline__ uint32_t bool_input_fields(uint32_t code) {
  using namespace gpisa;
  if (code < (uint32_t)BOOL_IF_BASE) {
    const int form = (int)(code >> 2) / R;
    return (form == BF_XX ? 3u : 0u) | (form == BF_XS ? 1u : 0u) | (form == BF_SX ? 2u : 0u);
  }
  if (code < (uint32_t)BOOL_MOVX) {
    const int desc = if_form_desc_fast((int)(code - BOOL_IF_BASE) / R);
    return (desc / 16 == 0 ? 1u : 0u) | ((desc / 4) % 4 == 0 ? 2u : 0u) | (desc % 4 == 0 ? 4u : 0u);
  }
  return 1u;  // MOVX
}

// SEG: the block's population, cases and hit counts come from segment table
// t (eval_float.cuh's SegTable: Boolean segments hold words); otherwise from a.
// COMPACT: a block of at least four passes stages only the inputs its
// program reads (the listing's shared arrays exist in these kernels only).
template <int K, bool SEG, bool COMPACT>
__device__ __forceinline__ void eval_bool_block(const BoolArgs& a, const SegTable* t) {
  using namespace gpisa;
  // dynamic: the program (prog_cap instructions + the end sentinel), then the
  // staged inputs [warp][input][32 lanes][K words]
  extern __shared__ uint4 dyn_s[];
  uint4* prog_s = dyn_s;
  uint4* btile_s = dyn_s + a.prog_cap + 1;
  __shared__ unsigned long long red_s[32];
  __shared__ int meta_s;

  const int item = blockIdx.x;
  const int seg = SEG ? segment_of(t, item) : 0;
#define GP_SEG(field, seg_expr) (SEG ? (seg_expr) : a.field)
  const int32_t a_n_chunks = GP_SEG(n_chunks, t->s[seg].n_chunks);
  const int prog_base = SEG ? t->s[seg].prog_begin : 0;
  const int local = SEG ? item - t->s[seg].block_begin : item;
  const int rank = local / a_n_chunks;
  const int p = a.order ? a.order[prog_base + rank] : prog_base + rank;
  const int chunk = local - rank * a_n_chunks;
  const int tid = threadIdx.x;
  const int32_t a_n_inputs = GP_SEG(n_inputs, t->s[seg].n_inputs);
  const int64_t a_n_cases = GP_SEG(n_cases, t->s[seg].n_cases);
  const int64_t a_n_words = GP_SEG(n_words, t->s[seg].n_units);
  const int64_t a_chunk_words = GP_SEG(chunk_words, t->s[seg].chunk);
  const uint32_t* a_case_bits = GP_SEG(case_bits, static_cast<const uint32_t*>(t->s[seg].cases));
  const uint32_t* a_target_bits = GP_SEG(target_bits, static_cast<const uint32_t*>(t->s[seg].targets));
  const bool a_aligned = GP_SEG(aligned, t->s[seg].aligned != 0);
  // hit counts: indexed by the segment's own program numbers
  unsigned long long* hits_row =
      SEG ? static_cast<unsigned long long*>(t->s[seg].out) + (p - prog_base) : (a.hits_out ? a.hits_out + p : nullptr);

  if (tid == 0) {
    int n_instr = -1;
    const int64_t off = a.offsets[p];
    const int32_t len = a.lengths[p];
    if ((off & 3) == 0 && len >= 4) {
      const uint4 h = *reinterpret_cast<const uint4*>(a.programs + off);
      const int n = (int)h.y;
      if ((h.x & 0xffu) == K_BOOL && (h.x >> 16) == VERSION && n >= 1 && n <= a.prog_cap &&
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
      ok &= valid_bool_instr(in, a_n_inputs) ? 1 : 0;
    }
    if (tid == 0) prog_s[n_instr] = make_uint4(BOOL_NCODES, 0u, 0u, 0u);  // end sentinel
    bad = !__syncthreads_and(ok);
  }
  if (bad) {
    if (tid == 0) {
      atomicOr(a.status, 2 /* GP_ERR_PROGRAM */);
      if (hits_row) atomicExch(hits_row, ~0ull);
    }
    return;
  }

  // Inputs to stage: only those the program reads, in increasing order (slot
  // s holds input list_s[s]), its input payloads rewritten to slots -- as the
  // float kernels do.  Every pass stages its words of each listed input only.
  // Blocks of fewer than four passes stage every input: the listing's
  // barriers and atomics cost them more than the copies they save (measured:
  // one pass per block, 11- and 13-input sets 11-15% slower listed; sixteen,
  // the 20-multiplexer 8% faster), and launches whose chunks are that short
  // take the kernel without the listing (its shared arrays and code cost
  // those sets 6% even unused, measured).
  int n_stage = a_n_inputs;
  bool listed = false;
  const uint32_t* list_p = nullptr;  // input of each staged slot when listed
  if constexpr (COMPACT) {
    __shared__ uint32_t used_s[GP_COMPACT_MAX_INPUTS / 32];    // bitmap of the inputs the program reads
    __shared__ uint32_t before_s[GP_COMPACT_MAX_INPUTS / 32];  // set bits in earlier words
    __shared__ uint32_t list_s[GP_COMPACT_MAX_LIST];
    __shared__ int n_stage_s;
    list_p = list_s;
    if (a_n_inputs <= GP_COMPACT_MAX_INPUTS && a_chunk_words >= 4 * (int64_t)blockDim.x * K) {
      const int nw = (a_n_inputs + 31) >> 5;
      for (int i = tid; i < nw; i += blockDim.x) used_s[i] = 0u;
      __syncthreads();
      for (int i = tid; i < n_instr; i += blockDim.x) {
        const uint4 in = prog_s[i];
        const uint32_t f = bool_input_fields(in.x);
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
      if (n_stage_s <= GP_COMPACT_MAX_LIST) {  // (block-uniform)
        n_stage = n_stage_s;
        listed = true;
        auto slot = [&](uint32_t v) {
          return before_s[v >> 5] + (uint32_t)__popc(used_s[v >> 5] & ((1u << (v & 31)) - 1u));
        };
        for (int i = tid; i < n_instr; i += blockDim.x) {
          uint4 in = prog_s[i];
          const uint32_t f = bool_input_fields(in.x);
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
        __syncthreads();
      }
    }
  }

  const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
  const int64_t w_begin = (int64_t)chunk * a_chunk_words;
  int64_t w_end = w_begin + a_chunk_words;
  if (w_end > a_n_words) w_end = a_n_words;
  const uint32_t tail = (uint32_t)(a_n_cases & 31);
  const uint32_t last_mask = tail ? ((1u << tail) - 1u) : 0xffffffffu;
  uint32_t* out_row = (!SEG && a.out_words) ? a.out_words + (int64_t)p * a_n_words : nullptr;
  unsigned long long hits = 0;
  bool bad_pass = false;

  const uint32_t prog_addr = (uint32_t)__cvta_generic_to_shared(prog_s);
  uint32_t* tile = reinterpret_cast<uint32_t*>(btile_s) + (size_t)warp * a_n_inputs * 32 * K + lane * K;
  const uint32_t tile_addr = (uint32_t)__cvta_generic_to_shared(tile);
#pragma unroll 1
  for (int64_t wb = w_begin + (int64_t)warp * 32 * K; wb < w_end; wb += (int64_t)nwarps * 32 * K) {
    const int64_t w0 = wb + (int64_t)lane * K;
    const bool full = w0 + K <= a_n_words;
    int v = 0;
    if (full && a_aligned) {
      // every input's K words as asynchronous copies straight into the tile
      // (16-, 8- or 4-byte aligned: rows aligned, w0 a multiple of K): all
      // inputs in one global round trip, no registers held.  A lane reads
      // back only its own words, so its own wait suffices.
      for (; v < n_stage; ++v) {
        const uint32_t* src = a_case_bits + (int64_t)(listed ? list_p[v] : (uint32_t)v) * a_n_words + w0;
        uint32_t* dst = tile + v * 32 * K;
        if constexpr (K == 8) {
          __pipeline_memcpy_async(dst, src, 16);
          __pipeline_memcpy_async(dst + 4, src + 4, 16);
        } else {
          __pipeline_memcpy_async(dst, src, 4 * K);
        }
      }
      __pipeline_commit();
      __pipeline_wait_prior(0);
    }
    for (; v < n_stage; ++v) {
      UVec<K> tv;
      uload<K>(tv, a_case_bits + (int64_t)(listed ? list_p[v] : (uint32_t)v) * a_n_words, w0, a_n_words,
               full && a_aligned);
#pragma unroll
      for (int j = 0; j < K; ++j) tile[v * 32 * K + j] = tv.w[j];
    }
    uint32_t o[K];
    if (!run_bool<K>(prog_addr, (uint32_t)n_instr, tile_addr, o)) bad_pass = true;
    if (out_row) {
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (w0 + j < a_n_words) out_row[w0 + j] = o[j];
    }
    if (a_target_bits) {
      UVec<K> tv;
      uload<K>(tv, a_target_bits, w0, a_n_words, full && a_aligned);
      uint32_t h = 0;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const int64_t w = w0 + j;
        uint32_t m = (w < a_n_words - 1) ? 0xffffffffu : (w == a_n_words - 1 ? last_mask : 0u);
        h += __popc(~(o[j] ^ tv.w[j]) & m);
      }
      hits += h;
    }
  }
  if (__syncthreads_or(bad_pass ? 1 : 0)) {
    if (tid == 0) {
      atomicOr(a.status, 2 /* GP_ERR_PROGRAM */);
      if (hits_row) atomicExch(hits_row, ~0ull);
    }
    return;
  }
  if (!hits_row || !a_target_bits) return;
  // integer sums are exact, so any order gives the same hit count
  hits = __reduce_add_sync(0xffffffffu, (unsigned)hits);
  if (lane == 0) red_s[warp] = hits;
  __syncthreads();
  if (tid == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < nwarps; ++w) t += red_s[w];
    atomicAdd(hits_row, t);
  }
#undef GP_SEG
}

template <int K, bool COMPACT>
__global__ void __launch_bounds__(256) eval_bool_kernel(BoolArgs a) {
  eval_bool_block<K, false, COMPACT>(a, nullptr);
}

// several populations in one launch; each segment's hits are zero before it
template <int K>
__global__ void __launch_bounds__(256) eval_bool_seg_kernel(BoolArgs a, const __grid_constant__ SegTable t) {
  eval_bool_block<K, true, true>(a, &t);
}

}  // namespace gpdev

namespace gpdev {
inline size_t bool_tile_bytes(int k, int block, int n_inputs) {
  return (size_t)(block / 32) * (size_t)n_inputs * 32u * (size_t)k * sizeof(uint32_t);
}
}  // namespace gpdev

namespace gpdev {

// ---------------------------------------------------------------------------
// Program per lane, for tiny case sets (at most 4 words = 128 cases per
// input; the 6-input problems have 2 words).  A warp per program would leave
// most lanes idle; here each lane runs its own program over all W words
// (the paper's ThreadGP layout, Sec. 3), and branch-free decoding keeps the
// lanes of a warp on one instruction stream even though their programs
// differ: operand slots are computed, AND / OR / IF are all computed and one
// is selected, NAND / NOR are a negation mask.  Stack levels live in shared
// memory [level][lane][W], the staged inputs [input][W] are shared by the
// block.  Instructions are read per lane from global memory (L1-cached), one
// ahead of the one being computed.  One warp per block, so that small
// populations still spread over every SM.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(32) eval_bool_lanes_kernel(BoolArgs a) {
  using namespace gpisa;
  extern __shared__ uint32_t lane_smem[];
  __shared__ uint32_t if_desc_s[BOOL_IF_FORMS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t* inp_s = lane_smem;  // [n_inputs][W]; then each warp's levels [R][32][W] (lv_addr)
  if (tid < BOOL_IF_FORMS) if_desc_s[tid] = (uint32_t)if_form_desc(tid);
  for (int i = tid; i < a.n_inputs * W; i += blockDim.x) {
    const int v = i / W, w = i % W;
    inp_s[i] = (w < a.n_words) ? a.case_bits[(int64_t)v * a.n_words + w] : 0u;
  }
  __syncthreads();
  const int rank = blockIdx.x * blockDim.x + tid;
  if (rank >= a.n_progs) return;
  const int p = a.order ? a.order[rank] : rank;  // (the launch passes no order)

  int n = -1;
  const uint4* prog = nullptr;
  {
    const int64_t off = a.offsets[p];
    const int32_t len = a.lengths[p];
    if ((off & 3) == 0 && len >= 4) {
      prog = reinterpret_cast<const uint4*>(a.programs + off);
      const uint4 h = __ldg(prog);
      const int cnt = (int)h.y;
      if ((h.x & 0xffu) == K_BOOL && (h.x >> 16) == VERSION && cnt >= 1 && cnt <= MAX_INSTR &&
          4 + 4 * (int64_t)cnt <= len)
        n = cnt;
    }
  }
  bool bad = n < 0;
  const uint32_t nin = (uint32_t)a.n_inputs;
  // address (in words) of a slot: input v, or stack level l of this lane
  auto in_addr = [&](uint32_t v, bool& b) -> uint32_t {
    if (v >= nin) { b = true; v = 0; }
    return v * W;
  };
  auto lv_addr = [&](uint32_t l, bool& b) -> uint32_t {
    if (l >= (uint32_t)R) { b = true; l = 0; }
    return (uint32_t)(a.n_inputs * W + warp * (R * 32 * W)) + (l * 32 + (uint32_t)lane) * W;
  };
  // the next instruction is loaded while the current one is computed
  uint4 next = bad ? make_uint4(0, 0, 0, 0) : __ldg(prog + 1);
  for (int i = 0; i < (bad ? 0 : n); ++i) {
    const uint4 in = next;
    if (i + 1 < n) next = __ldg(prog + 2 + i);
    const uint32_t code = in.x;
    uint32_t sa, sb, sc, dst;
    uint32_t is_or = 0, is_if = 0, neg = 0;
    if (code < (uint32_t)BOOL_IF_BASE) {
      const uint32_t op = code & 3u, l = (code >> 2) & 7u, form = code >> 5;
      dst = l;
      // XX, XS, SX, SS, SSR
      sa = (form == BF_XX || form == BF_XS) ? in_addr(in.y, bad)
                                            : lv_addr(form == BF_SSR ? l + 1 : l, bad);
      sb = (form == BF_XX || form == BF_SX) ? in_addr(in.z, bad)
                                            : lv_addr(form == BF_SS ? l + 1 : l, bad);
      sc = sb;
      is_or = (op == B_OR || op == B_NOR) ? 1u : 0u;
      neg = (op == B_NAND || op == B_NOR) ? 0xffffffffu : 0u;
    } else if (code < (uint32_t)BOOL_MOVX) {
      const uint32_t f = (code - BOOL_IF_BASE) >> 3, l = (code - BOOL_IF_BASE) & 7u;
      const uint32_t d = if_desc_s[f & 15u];
      const uint32_t dc = d >> 4, da = (d >> 2) & 3u, db = d & 3u;
      dst = l;
      sa = dc ? lv_addr(l + dc - 1, bad) : in_addr(in.y, bad);
      sb = da ? lv_addr(l + da - 1, bad) : in_addr(in.z, bad);
      sc = db ? lv_addr(l + db - 1, bad) : in_addr(in.w, bad);
      is_if = 1u;
    } else {
      if (code != (uint32_t)BOOL_MOVX) bad = true;
      dst = 0;
      sa = in_addr(in.y, bad);
      sb = sa;  // AND(a, a) = a
      sc = sa;
    }
    const uint32_t da_ = lv_addr(dst, bad);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t x = lane_smem[sa + w], y = lane_smem[sb + w], z = lane_smem[sc + w];
      uint32_t r = is_or ? (x | y) : (x & y);
      r ^= neg;
      const uint32_t f3 = (x & y) | (~x & z);
      lane_smem[da_ + w] = is_if ? f3 : r;
    }
  }
  uint32_t out[W];
  const uint32_t base0 = (uint32_t)(a.n_inputs * W + warp * (R * 32 * W)) + (uint32_t)lane * W;
#pragma unroll
  for (int w = 0; w < W; ++w) out[w] = lane_smem[base0 + w];
  if (bad) {
    atomicOr(a.status, 2 /* GP_ERR_PROGRAM */);
    if (a.hits_out) a.hits_out[p] = ~0ull;
    return;
  }
  if (a.out_words) {
#pragma unroll
    for (int w = 0; w < W; ++w)
      if (w < a.n_words) a.out_words[(int64_t)p * a.n_words + w] = out[w];
  }
  if (a.hits_out && a.target_bits) {
    const uint32_t tail = (uint32_t)(a.n_cases & 31);
    const uint32_t last_mask = tail ? ((1u << tail) - 1u) : 0xffffffffu;
    unsigned long long h = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      if (w >= a.n_words) break;
      const uint32_t m = (w < a.n_words - 1) ? 0xffffffffu : last_mask;
      h += __popc(~(out[w] ^ __ldg(a.target_bits + w)) & m);
    }
    a.hits_out[p] = h;
  }
}

inline size_t bool_lanes_smem(int w, int block, int n_inputs) {
  return sizeof(uint32_t) * ((size_t)n_inputs * w + (size_t)(block / 32) * gpisa::R * 32 * w);
}

// ---------------------------------------------------------------------------
// Warp per program, several programs per block, for case sets of a few
// hundred words (the 11-input problems: 64 words).  The block kernel above
// gives every program blocks of its own, each staging the inputs again and
// reducing across its warps; with 64 words a program is one pass of one warp,
// so those fixed costs dominate.  Here the block stages the whole case set
// once, as pass tiles [pass][input][32 lanes][K words] (the generated
// interpreter's tile layout, so every pass of every warp reads its inputs
// from the same place), and each warp stages its own program, interprets it
// over every pass and writes its hit count: no barrier after the staging, no
// cross-warp reduction.  The block's warps take consecutive ranks of the
// order (longest first), so they finish together.
// dynamic shared memory: the pass tiles (n_pass * n_inputs * 32 * K words),
// then one program buffer (prog_cap + 1 instructions) per warp.
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(256) eval_bool_warps_kernel(BoolArgs a) {
  using namespace gpisa;
  extern __shared__ uint4 dyn_s[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
  constexpr int kPassWords = 32 * K;
  const int64_t n_words = a.n_words;
  const int n_pass = (int)((n_words + kPassWords - 1) / kPassWords);
  const int nin = a.n_inputs;
  const size_t tile_words = (size_t)n_pass * nin * kPassWords;  // a multiple of 32
  uint32_t* tile_s = reinterpret_cast<uint32_t*>(dyn_s);
  uint4* prog_s = dyn_s + tile_words / 4 + (size_t)warp * (a.prog_cap + 1);

  // the case set, four words at a time (a group never straddles a pass tile:
  // tiles hold a multiple of 32 words); words past the end are 0
  const int64_t row = (int64_t)n_pass * kPassWords;  // padded words per input
  const bool vec = a.aligned && (n_words & 3) == 0;
  for (int64_t q = tid; q < (int64_t)nin * row / 4; q += blockDim.x) {
    const int64_t e = q * 4;
    const int v = (int)(e / row);
    const int64_t w = e - (int64_t)v * row;
    const int pass = (int)(w / kPassWords);
    const int r = (int)(w - (int64_t)pass * kPassWords);
    const uint32_t* src = a.case_bits + (int64_t)v * n_words + w;
    uint4 val;
    if (vec && w + 4 <= n_words) {
      val = __ldg(reinterpret_cast<const uint4*>(src));
    } else {
      val.x = w < n_words ? __ldg(src) : 0u;
      val.y = w + 1 < n_words ? __ldg(src + 1) : 0u;
      val.z = w + 2 < n_words ? __ldg(src + 2) : 0u;
      val.w = w + 3 < n_words ? __ldg(src + 3) : 0u;
    }
    *reinterpret_cast<uint4*>(tile_s + ((size_t)pass * nin + v) * kPassWords + r) = val;
  }

  // this warp's program (ranks past the population stage nothing)
  const int rank = blockIdx.x * nwarps + warp;
  const bool active = rank < a.n_progs;
  const int p = !active ? 0 : (a.order ? a.order[rank] : rank);
  int n_instr = -1;
  if (active) {
    if (lane == 0) {
      const int64_t off = a.offsets[p];
      const int32_t len = a.lengths[p];
      if ((off & 3) == 0 && len >= 4) {
        const uint4 h = *reinterpret_cast<const uint4*>(a.programs + off);
        const int n = (int)h.y;
        if ((h.x & 0xffu) == K_BOOL && (h.x >> 16) == VERSION && n >= 1 && n <= a.prog_cap &&
            4 + 4 * (int64_t)n <= len)
          n_instr = n;
      }
    }
    n_instr = __shfl_sync(0xffffffffu, n_instr, 0);
    if (n_instr >= 0) {
      const uint4* g = reinterpret_cast<const uint4*>(a.programs + a.offsets[p]) + 1;
      bool ok = true;
      for (int i = lane; i < n_instr; i += 32) {
        const uint4 in = g[i];
        prog_s[i] = in;
        ok &= valid_bool_instr(in, nin);
      }
      if (lane == 0) prog_s[n_instr] = make_uint4(BOOL_NCODES, 0u, 0u, 0u);  // end sentinel
      if (!__all_sync(0xffffffffu, ok)) n_instr = -1;
    }
  }
  __syncthreads();  // the case set is staged (each warp's program: its own lanes, ordered by the barrier)
  if (!active) return;
  unsigned long long* hits_row = a.hits_out ? a.hits_out + p : nullptr;
  if (n_instr < 0) {
    if (lane == 0) {
      atomicOr(a.status, 2 /* GP_ERR_PROGRAM */);
      if (hits_row) *hits_row = ~0ull;
    }
    return;
  }

  const uint32_t tail = (uint32_t)(a.n_cases & 31);
  const uint32_t last_mask = tail ? ((1u << tail) - 1u) : 0xffffffffu;
  uint32_t* out_row = a.out_words ? a.out_words + (int64_t)p * n_words : nullptr;
  const uint32_t prog_addr = (uint32_t)__cvta_generic_to_shared(prog_s);
  const uint32_t tile_addr0 = (uint32_t)__cvta_generic_to_shared(tile_s) + (uint32_t)(lane * K * 4);
  unsigned hits = 0;  // at most n_words * 32 / 32 lanes per lane, below 2^32
  bool bad = false;
#pragma unroll 1
  for (int pass = 0; pass < n_pass; ++pass) {
    const int64_t w0 = (int64_t)pass * kPassWords + lane * K;
    uint32_t o[K];
    if (!run_bool<K>(prog_addr, (uint32_t)n_instr,
                     tile_addr0 + (uint32_t)((size_t)pass * nin * kPassWords * 4), o))
      bad = true;
    if (out_row) {
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (w0 + j < n_words) out_row[w0 + j] = o[j];
    }
    if (a.target_bits) {
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const int64_t w = w0 + j;
        if (w < n_words) {
          const uint32_t m = w < n_words - 1 ? 0xffffffffu : last_mask;
          hits += __popc(~(o[j] ^ __ldg(a.target_bits + w)) & m);
        }
      }
    }
  }
  // (an unknown code stops every lane of the warp: the program is warp-uniform)
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0) {
      atomicOr(a.status, 2 /* GP_ERR_PROGRAM */);
      if (hits_row) *hits_row = ~0ull;
    }
    return;
  }
  if (!hits_row || !a.target_bits) return;
  hits = __reduce_add_sync(0xffffffffu, hits);  // integer sums: any order gives the same count
  if (lane == 0) *hits_row = hits;
}

// dynamic shared memory of eval_bool_warps_kernel
inline size_t bool_warps_smem(int k, int block, int n_inputs, int64_t n_words, int prog_cap) {
  const int64_t pass_words = 32 * (int64_t)k;
  const int64_t n_pass = (n_words + pass_words - 1) / pass_words;
  return sizeof(uint32_t) * (size_t)(n_pass * n_inputs * pass_words) +
         (size_t)(block / 32) * (size_t)(prog_cap + 1) * sizeof(uint4);
}

}  // namespace gpdev
