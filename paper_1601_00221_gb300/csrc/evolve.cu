// evolve.cu -- the device-side encoder and the on-device generation loop
// (include/gpeval.h: gp_encode_population_device, gp_evolve_*).
//
// Sec. 5 of the paper converts each tree to its linear form on the host every
// generation; Sec. 4.2 runs tournament selection, crossover and mutation
// around the evaluation.  Here all three steps of a generation -- variation,
// encoding and evaluation -- are kernels, captured once as a CUDA graph per
// direction of the population's double buffer and replayed, so a run needs
// the host only to start it and to read the result.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "../../include/gpeval.h"
#include "isa.h"
#include "launch.h"
#include "status.h"

using namespace gpisa;

namespace gpdev {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// the draws of one offspring: blocks (i, g, j, 0), j = 0, 1, ..., words in order
struct Draws {
  uint2 key;
  uint32_t i, g, j, n;
  uint4 blk;
  __device__ uint32_t next() {
    if (n == 0) {
      blk = philox4x32_10(make_uint4(i, g, j, 0u), key);
      ++j;
      n = 4;
    }
    const uint32_t w = n == 4 ? blk.x : n == 3 ? blk.y : n == 2 ? blk.z : blk.w;
    --n;
    return w;
  }
  __device__ uint32_t uniform(uint32_t m) { return (uint32_t)(((uint64_t)next() * m) >> 32); }
};

__host__ __device__ inline int fn_arity(uint32_t op) {
  if (op >= GP_OP_ADD && op <= GP_OP_DIV) return 2;
  if (op >= GP_OP_SIN && op <= GP_OP_LOG) return 1;
  if ((op >= GP_OP_GT && op <= GP_OP_EQ) || op == GP_OP_AND || op == GP_OP_OR) return 2;
  if (op == GP_OP_IF) return 3;
  return -1;  // terminal or unknown
}

// ---------------------------------------------------------------------------
// prefix-tree walks over a tree in (global) memory
// ---------------------------------------------------------------------------
// word position of node `idx` (prefix order) and the number of nodes
__device__ uint32_t node_start(const uint32_t* t, uint32_t idx) {
  uint32_t pos = 0;
  for (uint32_t k = 0; k < idx; ++k) pos += ((t[pos] & 0xffu) == GP_OP_CONST) ? 2u : 1u;
  return pos;
}
__device__ uint32_t count_nodes(const uint32_t* t, uint32_t len) {
  uint32_t pos = 0, n = 0;
  while (pos < len) {
    pos += ((t[pos] & 0xffu) == GP_OP_CONST) ? 2u : 1u;
    ++n;
  }
  return n;
}
// one past the subtree at `start`; *nodes receives its node count
__device__ uint32_t subtree_end(const uint32_t* t, uint32_t start, uint32_t* nodes) {
  uint32_t owed = 1, pos = start, n = 0;
  while (owed) {
    const uint32_t op = t[pos] & 0xffu;
    --owed;
    ++n;
    if (op == GP_OP_CONST) { pos += 2; continue; }
    if (op != GP_OP_VAR) owed += (uint32_t)fn_arity(op);
    ++pos;
  }
  *nodes = n;
  return pos;
}

// ---------------------------------------------------------------------------
// variation: one thread per offspring
// ---------------------------------------------------------------------------
struct VaryArgs {
  const uint32_t* cur;      // [n][slot] parents
  const int32_t* cur_len;
  const double* fitness;    // of the parents
  uint32_t* next;           // [n][slot] offspring
  int32_t* next_len;
  const int32_t* generation;  // index of the parents' generation
  int32_t n, slot, max_nodes, tournament, mutation_depth, n_funcs, n_inputs;
  int32_t funcs[16];
  uint32_t thr_cross, thr_mut, thr_const;
  float const_lo, const_hi;
  uint2 key;
};

constexpr int kGrowWords = 96;  // a grown subtree of depth <= 4: at most 40 nodes, 80 words

__device__ __forceinline__ bool worse_or_equal(double a, double b) {  // a not strictly better than b
  const double ka = isnan(a) ? INFINITY : a, kb = isnan(b) ? INFINITY : b;
  return !(ka < kb);
}

__device__ uint32_t tournament(Draws& d, const VaryArgs& a) {
  uint32_t best = d.uniform((uint32_t)a.n);
  for (int t = 1; t < a.tournament; ++t) {
    const uint32_t c = d.uniform((uint32_t)a.n);
    if (!worse_or_equal(a.fitness[c], a.fitness[best])) best = c;
  }
  return best;
}

// grows a subtree into buf (prefix order); returns its word count, *nodes its nodes
__device__ uint32_t grow(Draws& d, const VaryArgs& a, uint32_t* buf, uint32_t* nodes) {
  int pending[24];  // depths of the nodes still to draw (LIFO keeps prefix order)
  int np = 0;
  pending[np++] = 1;
  uint32_t w = 0, n = 0;
  while (np) {
    const int dep = pending[--np];
    ++n;
    bool term = dep >= a.mutation_depth;
    if (!term && dep > 1) term = d.next() < 0x80000000u;
    if (term) {
      if (d.next() < a.thr_const) {
        const uint32_t u = d.next();
        const float t = __fmul_rn((float)(u >> 8), 5.9604644775390625e-08f);  // 2^-24
        const float v = __fadd_rn(a.const_lo, __fmul_rn(__fsub_rn(a.const_hi, a.const_lo), t));
        buf[w++] = GP_OP_CONST;
        buf[w++] = __float_as_uint(v);
      } else {
        buf[w++] = (uint32_t)GP_OP_VAR | (d.uniform((uint32_t)a.n_inputs) << 8);
      }
      continue;
    }
    const uint32_t f = (uint32_t)a.funcs[d.uniform((uint32_t)a.n_funcs)];
    buf[w++] = f;
    for (int c = 0; c < fn_arity(f); ++c) pending[np++] = dep + 1;
  }
  *nodes = n;
  return w;
}

__global__ void __launch_bounds__(128) vary_kernel(VaryArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  Draws d;
  d.key = a.key;
  d.i = (uint32_t)i;
  d.g = (uint32_t)(*a.generation + 1);
  d.j = 0;
  d.n = 0;
  const uint32_t pa = tournament(d, a);
  const uint32_t* A = a.cur + (size_t)pa * a.slot;
  const uint32_t lenA = (uint32_t)a.cur_len[pa];
  uint32_t* dst = a.next + (size_t)i * a.slot;
  uint32_t len = 0;
  bool copied = false;
  if (d.next() < a.thr_cross) {
    const uint32_t pb = tournament(d, a);
    const uint32_t* B = a.cur + (size_t)pb * a.slot;
    const uint32_t lenB = (uint32_t)a.cur_len[pb];
    const uint32_t nA = count_nodes(A, lenA), nB = count_nodes(B, lenB);
    const uint32_t sa = node_start(A, d.uniform(nA)), sb = node_start(B, d.uniform(nB));
    uint32_t na_sub, nb_sub;
    const uint32_t ea = subtree_end(A, sa, &na_sub), eb = subtree_end(B, sb, &nb_sub);
    if (nA - na_sub + nb_sub <= (uint32_t)a.max_nodes) {
      for (uint32_t k = 0; k < sa; ++k) dst[len++] = A[k];
      for (uint32_t k = sb; k < eb; ++k) dst[len++] = B[k];
      for (uint32_t k = ea; k < lenA; ++k) dst[len++] = A[k];
      copied = true;
    }
  }
  if (!copied) {
    for (uint32_t k = 0; k < lenA; ++k) dst[k] = A[k];
    len = lenA;
  }
  if (d.next() < a.thr_mut) {
    const uint32_t nc = count_nodes(dst, len);
    const uint32_t sm = node_start(dst, d.uniform(nc));
    uint32_t nm_sub, ng;
    const uint32_t em = subtree_end(dst, sm, &nm_sub);
    uint32_t g[kGrowWords];
    const uint32_t gw = grow(d, a, g, &ng);
    if (nc - nm_sub + ng <= (uint32_t)a.max_nodes) {
      const uint32_t new_len = len - (em - sm) + gw;
      if (sm + gw > em) {  // the suffix moves right: copy from its end
        for (uint32_t k = len; k > em; --k) dst[k - 1 + (sm + gw - em)] = dst[k - 1];
      } else if (sm + gw < em) {
        for (uint32_t k = em; k < len; ++k) dst[k - (em - sm - gw)] = dst[k];
      }
      for (uint32_t k = 0; k < gw; ++k) dst[sm + k] = g[k];
      len = new_len;
    }
  }
  a.next_len[i] = (int32_t)len;
}

__global__ void bump_generation(int32_t* g) { *g += 1; }

// ---------------------------------------------------------------------------
// device encoder: one thread per tree, scratch in shared memory
// ---------------------------------------------------------------------------
struct EncScratch {  // per thread
  uint32_t tok[2 * GP_DEVICE_ENCODE_MAX_NODES];  // the tree's words
  uint16_t pos[GP_DEVICE_ENCODE_MAX_NODES];   // word position of each node
  uint16_t cnt[GP_DEVICE_ENCODE_MAX_NODES];   // nodes in its subtree
  uint8_t op[GP_DEVICE_ENCODE_MAX_NODES];     // opcode
  uint8_t need[GP_DEVICE_ENCODE_MAX_NODES];   // stack levels its subtree needs
  uint8_t ord[GP_DEVICE_ENCODE_MAX_NODES];    // function children in evaluation order:
                                              // child ranks in bits 0-1, 2-3, 4-5, count in 6-7
  uint16_t fnode[GP_DEVICE_ENCODE_MAX_NODES]; // stack: node (parse: open node; emit: frame)
  uint8_t fk[GP_DEVICE_ENCODE_MAX_NODES];     // stack: remaining children / next child
  uint8_t flevel[GP_DEVICE_ENCODE_MAX_NODES]; // stack: level of the frame's result
};
// One tree per warp (a block of one warp): the trees of a warp would take
// different paths through the parser and run one after another (16 trees per
// warp executed 2 threads per instruction, measured); as separate warps the
// scheduler interleaves up to 32 of them per SM.  The warp copies the tree's
// words into shared memory together; lane 0 then parses, orders and emits.
constexpr int kEncThreads = 32;

struct EncArgs {
  const uint32_t* words;
  const int64_t* offsets;
  const int32_t* lengths;
  int32_t n_progs;
  int32_t order;
  uint32_t* out;
  const int64_t* out_offsets;
  int32_t* out_lengths;
  unsigned long long* node_total;  // may be null: adds the nodes of every tree encoded
};

__device__ __forceinline__ int child_at(const EncScratch& s, int v, int rank) {
  int c = v + 1;
  for (int k = 0; k < rank; ++k) c += s.cnt[c];
  return c;
}

__device__ int xbin(uint32_t op) {
  return op == GP_OP_GT ? XB_GT : op == GP_OP_LT ? XB_LT : op == GP_OP_EQ ? XB_EQ
                                : op == GP_OP_AND ? XB_AND : XB_OR;
}

// One tree per thread: (1) copy its words to shared memory and parse them into
// nodes (positions, opcodes, subtree sizes); (2) from the leaves up, the levels
// each subtree needs and the evaluation order of each node's function
// children (by decreasing need, stable, for GP_ORDER_MIN_DEPTH; left to right
// for GP_ORDER_PAPER); (3) emit the S-form post-order: a node's function
// children at levels l, l + 1, ... in that order, then the node at level l.
// The words are the host encoder's (encode.cpp) for the same tree.
__global__ void __launch_bounds__(kEncThreads) encode_kernel(EncArgs a) {
  extern __shared__ EncScratch enc_s[];
  const int p = blockIdx.x;  // one tree per block (a single warp)
  if (p >= a.n_progs) return;
  EncScratch& s = enc_s[0];
  const int len = a.lengths[p];
  bool ok = len > 0 && len <= 2 * GP_DEVICE_ENCODE_MAX_NODES;
  if (ok) {
    const uint32_t* g = a.words + a.offsets[p];
    for (int w = threadIdx.x; w < len; w += kEncThreads) s.tok[w] = g[w];
  }
  __syncwarp();
  if (threadIdx.x != 0) return;
  uint32_t* o = a.out + a.out_offsets[p];
  bool extended = false;
  int max_input = -1, n = 0, top = 0, w = 0;
  // 1. parse
  while (ok && w < len) {
    if (n > 0 && top == 0) { ok = false; break; }          // trailing tokens
    if (n >= GP_DEVICE_ENCODE_MAX_NODES) { ok = false; break; }
    const uint32_t tk = s.tok[w];
    const uint32_t op = tk & 0xffu;
    int ar = 0;
    s.pos[n] = (uint16_t)w;
    s.op[n] = (uint8_t)op;
    if (op == GP_OP_VAR) {
      if ((int)(tk >> 8) > max_input) max_input = (int)(tk >> 8);
      w += 1;
    } else if (op == GP_OP_CONST) {
      if (w + 1 >= len) { ok = false; break; }
      w += 2;
    } else {
      ar = fn_arity(op);
      if (ar < 0) { ok = false; break; }
      if (!(op >= GP_OP_ADD && op <= GP_OP_DIV)) extended = true;
      w += 1;
    }
    if (top) s.fk[top - 1] -= 1;
    if (ar > 0) {
      s.fnode[top] = (uint16_t)n;
      s.fk[top] = (uint8_t)ar;
      ++top;
    } else {
      s.cnt[n] = 1;
    }
    ++n;
    while (top && s.fk[top - 1] == 0) {
      --top;
      s.cnt[s.fnode[top]] = (uint16_t)(n - s.fnode[top]);
    }
  }
  if (ok && (top != 0 || n == 0)) ok = false;                // missing operands
  // 2. needs and child orders (children follow their parent in prefix order)
  int depth = 1;
  if (ok) {
    for (int v = n - 1; v >= 0; --v) {
      const int ar = fn_arity(s.op[v]);
      if (ar <= 0) { s.need[v] = 0; s.ord[v] = 0; continue; }
      int rk[3], nd[3], m = 0;
      int c = v + 1;
      for (int k = 0; k < ar; ++k) {
        if (fn_arity(s.op[c]) > 0) { rk[m] = k; nd[m] = s.need[c]; ++m; }
        c += s.cnt[c];
      }
      if (a.order == GP_ORDER_MIN_DEPTH)  // insertion sort by decreasing need: stable
        for (int x = 1; x < m; ++x)
          for (int y = x; y > 0 && nd[y] > nd[y - 1]; --y) {
            int t0 = rk[y]; rk[y] = rk[y - 1]; rk[y - 1] = t0;
            t0 = nd[y]; nd[y] = nd[y - 1]; nd[y - 1] = t0;
          }
      int need = 1;
      uint32_t packed = (uint32_t)m << 6;
      for (int k = 0; k < m; ++k) {
        need = max(need, k + nd[k]);
        packed |= (uint32_t)rk[k] << (2 * k);
      }
      s.need[v] = (uint8_t)min(need, 255);
      s.ord[v] = (uint8_t)packed;
    }
    depth = fn_arity(s.op[0]) > 0 ? s.need[0] : 1;
    if (depth > R) ok = false;
  }
  if (!ok) {  // a header of kind 0: every evaluation reports the program as malformed
    o[0] = 0u; o[1] = 0u; o[2] = 0u; o[3] = 0u;
    a.out_lengths[p] = 4;
    return;
  }
  // 3. emit
  int ni = 0;
  uint32_t* ins = o + 4;
  if (fn_arity(s.op[0]) <= 0) {  // a single terminal: one move to level 0
    const bool cst = s.op[0] == GP_OP_CONST;
    ins[0] = (uint32_t)sform_code(cst ? SF_MOVC : SF_MOVX, 0, 0);
    ins[1] = cst ? s.tok[1] : (s.tok[0] >> 8);
    ins[2] = 0u;
    ins[3] = 0u;
    ni = 1;
  } else {
    top = 0;
    s.fnode[top] = 0; s.flevel[top] = 0; s.fk[top] = 0; ++top;
    while (top) {
      const int v = s.fnode[top - 1], l = s.flevel[top - 1], k = s.fk[top - 1];
      const uint32_t od = s.ord[v];
      const int np = (int)(od >> 6);
      if (k < np) {  // next function child, at level l + k
        s.fk[top - 1] = (uint8_t)(k + 1);
        s.fnode[top] = (uint16_t)child_at(s, v, (int)((od >> (2 * k)) & 3u));
        s.flevel[top] = (uint8_t)(l + k);
        s.fk[top] = 0;
        ++top;
        continue;
      }
      --top;
      const uint32_t op = s.op[v];
      const int ar = fn_arity(op);
      int kind[3] = {0, 0, 0};   // 0 input, 1 constant, 2 + j stack level l + j
      uint32_t pay[3] = {0u, 0u, 0u};
      int c = v + 1;
      for (int q = 0; q < ar; ++q) {
        if (s.op[c] == GP_OP_VAR) { kind[q] = 0; pay[q] = s.tok[s.pos[c]] >> 8; }
        else if (s.op[c] == GP_OP_CONST) { kind[q] = 1; pay[q] = s.tok[s.pos[c] + 1]; }
        c += s.cnt[c];
      }
      for (int r = 0; r < np; ++r) kind[(od >> (2 * r)) & 3u] = 2 + r;
      uint32_t code;
      if (ar == 1) {
        const int uf = kind[0] == 0 ? UF_X : kind[0] == 1 ? UF_C : UF_S;
        code = (uint32_t)sfx_un_code(uf, l, (int)(op - GP_OP_SIN));
      } else if (ar == 3) {
        code = (uint32_t)sfx_if_code(xif_form_index(kind[0], kind[1], kind[2]), l);
      } else {
        // forms by (a, b): X X, X C, C X, C C, S0 X, X S0, S0 C, C S0, S0 S1, S1 S0
        const int ka = kind[0], kb = kind[1];
        int form;
        if (ka < 2 && kb < 2) form = ka == 0 ? (kb == 0 ? SF_XX : SF_XC) : (kb == 0 ? SF_CX : SF_CC);
        else if (ka == 2 && kb < 2) form = kb == 0 ? SF_SX : SF_SC;
        else if (kb == 2 && ka < 2) form = ka == 0 ? SF_XS : SF_CS;
        else form = ka == 2 ? SF_SS : SF_SSR;
        code = (op >= GP_OP_ADD && op <= GP_OP_DIV) ? (uint32_t)sform_code(form, l, (int)(op - GP_OP_ADD))
                                                   : (uint32_t)sfx_bin_code(form, l, xbin(op));
      }
      uint32_t* q = ins + 4 * ni;
      q[0] = code;
      q[1] = pay[0];
      q[2] = pay[1];
      q[3] = pay[2];
      ++ni;
    }
  }
  o[0] = header0(extended ? (uint32_t)K_SFORMX : (uint32_t)K_SFORM, (uint32_t)a.order);
  o[1] = (uint32_t)ni;
  o[2] = (uint32_t)n;
  o[3] = (uint32_t)depth | ((uint32_t)(max_input + 1) << 16);
  a.out_lengths[p] = 4 + 4 * ni;
  if (a.node_total) atomicAdd(a.node_total, (unsigned long long)n);
}

cudaError_t launch_encode(const EncArgs& a, cudaStream_t s) {
  static std::atomic<size_t> set{0};
  const size_t smem = sizeof(EncScratch);  // one tree per block
  ensure_dynamic_smem(encode_kernel, smem, set);
  encode_kernel<<<a.n_progs, kEncThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace gpdev

using namespace gpdev;

extern "C" int gp_encode_population_device(const uint32_t* words, const int64_t* offsets,
                                           const int32_t* lengths, int32_t n_progs, int32_t order,
                                           uint32_t* out, const int64_t* out_offsets,
                                           int32_t* out_lengths, gp_stream_t stream) {
  gp_clear_error();
  if (n_progs < 0) return gp_fail(GP_ERR_INVALID_ARG, "negative n_progs");
  if (n_progs == 0) return GP_OK;
  if (!words || !offsets || !lengths || !out || !out_offsets || !out_lengths)
    return gp_fail(GP_ERR_INVALID_ARG, "null device array");
  if (order != GP_ORDER_PAPER && order != GP_ORDER_MIN_DEPTH)
    return gp_fail(GP_ERR_INVALID_ARG, "unknown order %d", order);
  EncArgs a{words, offsets, lengths, n_progs, order, out, out_offsets, out_lengths, nullptr};
  cudaError_t e = launch_encode(a, (cudaStream_t)stream);
  if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "encoder launch: %s", cudaGetErrorString(e));
  return GP_OK;
}

// ---------------------------------------------------------------------------
// the run
// ---------------------------------------------------------------------------
struct gp_evolver {
  gp_evolve_params prm;
  int32_t n, slot, eslot;
  const float* cases;
  const float* targets;
  int32_t n_inputs;
  int64_t n_cases;
  cudaStream_t stream = nullptr;
  uint32_t* pop[2] = {nullptr, nullptr};  // [n][slot]
  int32_t* len[2] = {nullptr, nullptr};
  int64_t* off = nullptr;                 // p * slot
  uint32_t* enc = nullptr;                // [n][eslot]
  int64_t* eoff = nullptr;                // p * eslot
  int32_t* elen = nullptr;
  double* fit = nullptr;
  int32_t* gen = nullptr;                 // device: index of the current generation
  unsigned long long* nodes = nullptr;    // device: tree nodes of every generation evaluated
  int cur = 0;
  int32_t generation = 0;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};  // [from buffer]
};

namespace {

int evolve_fail(gp_evolver* ev, int rc) {
  gp_evolve_destroy(ev);
  return rc;
}

uint32_t prob_threshold(float p) {
  const double v = std::floor((double)p * 4294967296.0);
  return (uint32_t)std::fmin(std::fmax(v, 0.0), 4294967295.0);
}

// the steps of one generation, from buffer `from` to the other
int enqueue_generation(gp_evolver* ev, int from) {
  const int to = 1 - from;
  VaryArgs v;
  v.cur = ev->pop[from];
  v.cur_len = ev->len[from];
  v.fitness = ev->fit;
  v.next = ev->pop[to];
  v.next_len = ev->len[to];
  v.generation = ev->gen;
  v.n = ev->n;
  v.slot = ev->slot;
  v.max_nodes = ev->prm.max_nodes;
  v.tournament = ev->prm.tournament;
  v.mutation_depth = ev->prm.mutation_depth;
  v.n_funcs = ev->prm.n_funcs;
  v.n_inputs = ev->n_inputs;
  for (int k = 0; k < 16; ++k) v.funcs[k] = ev->prm.funcs[k];
  v.thr_cross = prob_threshold(ev->prm.p_crossover);
  v.thr_mut = prob_threshold(ev->prm.p_mutation);
  v.thr_const = prob_threshold(ev->prm.p_const);
  v.const_lo = ev->prm.const_lo;
  v.const_hi = ev->prm.const_hi;
  v.key = make_uint2((uint32_t)(ev->prm.seed & 0xffffffffu), (uint32_t)(ev->prm.seed >> 32));
  vary_kernel<<<(ev->n + 127) / 128, 128, 0, ev->stream>>>(v);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "variation launch: %s", cudaGetErrorString(e));
  EncArgs ea{ev->pop[to], ev->off, ev->len[to], ev->n, GP_ORDER_MIN_DEPTH, ev->enc, ev->eoff,
             ev->elen, ev->nodes};
  e = launch_encode(ea, ev->stream);
  if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "encoder launch: %s", cudaGetErrorString(e));
  int rc;
  rc = gp_eval_population_ex(ev->enc, ev->eoff, ev->elen, ev->n, ev->cases, ev->n_inputs,
                             ev->n_cases, ev->targets, ev->fit, nullptr, &ev->prm.eval,
                             (gp_stream_t)ev->stream);
  if (rc) return rc;
  bump_generation<<<1, 1, 0, ev->stream>>>(ev->gen);
  e = cudaGetLastError();
  if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "counter launch: %s", cudaGetErrorString(e));
  return GP_OK;
}

}  // namespace

extern "C" int gp_evolve_create(const gp_evolve_params* params, const uint32_t* words,
                                const int64_t* offsets, const int32_t* lengths, const float* cases,
                                int32_t n_inputs, int64_t n_cases, const float* targets,
                                gp_evolver** out) {
  gp_clear_error();
  if (!params || !words || !offsets || !lengths || !out)
    return gp_fail(GP_ERR_INVALID_ARG, "null argument");
  const gp_evolve_params& P = *params;
  if (P.pop_size < 1) return gp_fail(GP_ERR_INVALID_ARG, "pop_size must be positive");
  if (P.max_nodes < 1 || P.max_nodes > 255) return gp_fail(GP_ERR_INVALID_ARG, "max_nodes must be 1..255");
  if (P.tournament < 1) return gp_fail(GP_ERR_INVALID_ARG, "tournament must be at least 1");
  if (P.mutation_depth < 1 || P.mutation_depth > 4)
    return gp_fail(GP_ERR_INVALID_ARG, "mutation_depth must be 1..4");
  if (P.n_funcs < 1 || P.n_funcs > 16) return gp_fail(GP_ERR_INVALID_ARG, "n_funcs must be 1..16");
  for (int k = 0; k < P.n_funcs; ++k)
    if (fn_arity((uint32_t)P.funcs[k]) < 0 || P.funcs[k] == GP_OP_NAND || P.funcs[k] == GP_OP_NOR)
      return gp_fail(GP_ERR_INVALID_ARG, "funcs[%d] = %d is not a float function", k, P.funcs[k]);
  if (n_inputs < 1 || n_cases < 0 || (n_cases > 0 && (!cases || !targets)))
    return gp_fail(GP_ERR_INVALID_ARG, "bad cases");
  if (!(P.p_crossover >= 0.0f && P.p_crossover <= 1.0f && P.p_mutation >= 0.0f &&
        P.p_mutation <= 1.0f && P.p_const >= 0.0f && P.p_const <= 1.0f))
    return gp_fail(GP_ERR_INVALID_ARG, "probabilities must be in [0, 1]");

  gp_evolver* ev = new gp_evolver();
  ev->prm = P;
  // the extended functions need the extended interpreter
  bool ext_funcs = false;
  for (int k = 0; k < P.n_funcs; ++k)
    if (!(P.funcs[k] >= GP_OP_ADD && P.funcs[k] <= GP_OP_DIV)) ext_funcs = true;
  if (ext_funcs && ev->prm.eval.variant == GP_VARIANT_AUTO) ev->prm.eval.variant = GP_VARIANT_EXTENDED;
  ev->n = P.pop_size;
  ev->slot = 2 * P.max_nodes;
  ev->eslot = 4 + 4 * ev->slot;
  ev->cases = cases;
  ev->targets = targets;
  ev->n_inputs = n_inputs;
  ev->n_cases = n_cases;
  // the initial population in the slot layout
  std::vector<uint32_t> h_words((size_t)ev->n * ev->slot, 0u);
  std::vector<int32_t> h_len(ev->n);
  for (int p = 0; p < ev->n; ++p) {
    const int32_t L = lengths[p];
    if (L < 1 || L > ev->slot || offsets[p] < 0)
      return evolve_fail(ev, gp_fail(GP_ERR_PROGRAM, "tree %d has %d words (1..%d allowed)", p, L, ev->slot));
    const uint32_t* t = words + offsets[p];
    // one well-formed tree of float functions (the variation kernel walks
    // parents as prefix trees without further checks)
    int nodes = 0, owed = 1, w = 0;
    while (w < L && owed > 0) {
      const uint32_t op = t[w] & 0xffu;
      --owed;
      ++nodes;
      if (op == GP_OP_CONST) { w += 2; continue; }
      if (op != GP_OP_VAR) {
        const int ar = fn_arity(op);
        if (ar < 0)
          return evolve_fail(ev, gp_fail(GP_ERR_PROGRAM, "tree %d: opcode %u is not a float function", p, op));
        owed += ar;
      }
      ++w;
    }
    if (owed != 0 || w != L)
      return evolve_fail(ev, gp_fail(GP_ERR_PROGRAM, "tree %d is not one well-formed prefix tree", p));
    if (nodes > P.max_nodes)
      return evolve_fail(ev, gp_fail(GP_ERR_PROGRAM, "tree %d has %d nodes, more than max_nodes", p, nodes));
    memcpy(&h_words[(size_t)p * ev->slot], t, sizeof(uint32_t) * (size_t)L);
    h_len[p] = L;
  }
  std::vector<int64_t> h_off(ev->n), h_eoff(ev->n);
  for (int p = 0; p < ev->n; ++p) {
    h_off[p] = (int64_t)p * ev->slot;
    h_eoff[p] = (int64_t)p * ev->eslot;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&ev->stream, cudaStreamNonBlocking);
  const size_t pw = sizeof(uint32_t) * (size_t)ev->n * ev->slot;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMalloc((void**)&ev->pop[b], pw);
    if (e == cudaSuccess) e = cudaMalloc((void**)&ev->len[b], sizeof(int32_t) * ev->n);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&ev->off, sizeof(int64_t) * ev->n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ev->enc, sizeof(uint32_t) * (size_t)ev->n * ev->eslot);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ev->eoff, sizeof(int64_t) * ev->n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ev->elen, sizeof(int32_t) * ev->n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ev->fit, sizeof(double) * ev->n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ev->gen, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ev->nodes, sizeof(unsigned long long));
  if (e != cudaSuccess)
    return evolve_fail(ev, gp_fail(e == cudaErrorMemoryAllocation ? GP_ERR_OOM : GP_ERR_CUDA,
                                   "run allocation: %s", cudaGetErrorString(e)));
  cudaStream_t s = ev->stream;
  e = cudaMemcpyAsync(ev->pop[0], h_words.data(), pw, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ev->len[0], h_len.data(), sizeof(int32_t) * ev->n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ev->off, h_off.data(), sizeof(int64_t) * ev->n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ev->eoff, h_eoff.data(), sizeof(int64_t) * ev->n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ev->gen, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ev->nodes, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors go out of scope
  if (e != cudaSuccess)
    return evolve_fail(ev, gp_fail(GP_ERR_CUDA, "run upload: %s", cudaGetErrorString(e)));
  // generation 0: encode and evaluate (eagerly: this also sizes the evaluation's workspace)
  EncArgs ea{ev->pop[0], ev->off, ev->len[0], ev->n, GP_ORDER_MIN_DEPTH, ev->enc, ev->eoff,
             ev->elen, ev->nodes};
  e = launch_encode(ea, s);
  int rc = e == cudaSuccess ? GP_OK : gp_fail(GP_ERR_CUDA, "encoder launch: %s", cudaGetErrorString(e));
  if (!rc)
    rc = gp_eval_population_ex(ev->enc, ev->eoff, ev->elen, ev->n, cases, n_inputs, n_cases,
                               targets, ev->fit, nullptr, &ev->prm.eval, (gp_stream_t)s);
  if (rc) return evolve_fail(ev, rc);
  // one graph per direction of the double buffer
  for (int from = 0; from < 2; ++from) {
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return evolve_fail(ev, gp_fail(GP_ERR_CUDA, "capture: %s", cudaGetErrorString(e)));
    rc = enqueue_generation(ev, from);
    e = cudaStreamEndCapture(s, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return evolve_fail(ev, rc);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ev->exec[from], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return evolve_fail(ev, gp_fail(GP_ERR_CUDA, "graph: %s", cudaGetErrorString(e)));
  }
  *out = ev;
  return GP_OK;
}

extern "C" int gp_evolve_run(gp_evolver* ev, int32_t generations) {
  gp_clear_error();
  if (!ev || generations < 0) return gp_fail(GP_ERR_INVALID_ARG, "bad run arguments");
  for (int32_t k = 0; k < generations; ++k) {
    cudaError_t e = cudaGraphLaunch(ev->exec[ev->cur], ev->stream);
    if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    ev->cur = 1 - ev->cur;
    ++ev->generation;
  }
  return GP_OK;
}

extern "C" int gp_evolve_read(gp_evolver* ev, uint32_t* words, int32_t* lengths, double* fitness,
                              int32_t* generation, int64_t* nodes_evaluated) {
  gp_clear_error();
  if (!ev) return gp_fail(GP_ERR_INVALID_ARG, "null run");
  cudaError_t e = cudaStreamSynchronize(ev->stream);
  if (e == cudaSuccess && words)
    e = cudaMemcpy(words, ev->pop[ev->cur], sizeof(uint32_t) * (size_t)ev->n * ev->slot, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && lengths)
    e = cudaMemcpy(lengths, ev->len[ev->cur], sizeof(int32_t) * ev->n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && fitness)
    e = cudaMemcpy(fitness, ev->fit, sizeof(double) * ev->n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && nodes_evaluated) {
    unsigned long long v = 0;
    e = cudaMemcpy(&v, ev->nodes, sizeof(v), cudaMemcpyDeviceToHost);
    *nodes_evaluated = (int64_t)v;
  }
  if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "reading the run: %s", cudaGetErrorString(e));
  if (generation) *generation = ev->generation;
  return GP_OK;
}

extern "C" int gp_evolve_destroy(gp_evolver* ev) {
  gp_clear_error();
  if (!ev) return GP_OK;
  if (ev->stream) cudaStreamSynchronize(ev->stream);
  for (int b = 0; b < 2; ++b) {
    if (ev->exec[b]) cudaGraphExecDestroy(ev->exec[b]);
    if (ev->pop[b]) cudaFree(ev->pop[b]);
    if (ev->len[b]) cudaFree(ev->len[b]);
  }
  if (ev->off) cudaFree(ev->off);
  if (ev->enc) cudaFree(ev->enc);
  if (ev->eoff) cudaFree(ev->eoff);
  if (ev->elen) cudaFree(ev->elen);
  if (ev->fit) cudaFree(ev->fit);
  if (ev->gen) cudaFree(ev->gen);
  if (ev->nodes) cudaFree(ev->nodes);
  if (ev->stream) cudaStreamDestroy(ev->stream);
  delete ev;
  return GP_OK;
}
