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
// device encoder: one tree per warp, scratch in shared memory
// ---------------------------------------------------------------------------
struct EncScratch {  // per tree; node indices fit a byte (at most 256 nodes)
  uint32_t tok[2 * GP_DEVICE_ENCODE_MAX_NODES];  // the tree's words
  union {
    int16_t open[GP_DEVICE_ENCODE_MAX_NODES];  // operand slots open before each node, minus 1
    int32_t path[GP_DEVICE_ENCODE_MAX_NODES];  // placement: first instruction | level << 16
  } u;
  uint16_t pos[GP_DEVICE_ENCODE_MAX_NODES];      // word position of each node
  uint8_t opa[GP_DEVICE_ENCODE_MAX_NODES];       // opcode | arity << 6
  uint8_t par[GP_DEVICE_ENCODE_MAX_NODES];       // parent; then the pointer-jumping link
  uint8_t ch[3][GP_DEVICE_ENCODE_MAX_NODES];     // children, in operand order
  uint8_t need[GP_DEVICE_ENCODE_MAX_NODES];      // stack levels its subtree needs (0: a terminal,
                                                 // or a function node not yet finished)
  uint8_t ord[GP_DEVICE_ENCODE_MAX_NODES];       // function children in evaluation order:
                                                 // child ranks in bits 0-1, 2-3, 4-5, count in 6-7
  uint8_t fc[GP_DEVICE_ENCODE_MAX_NODES];        // function nodes in its subtree
};
// One tree per warp (a block of one warp), every step spread over the lanes:
// as separate warps the scheduler interleaves up to 32 trees per SM.  (One
// lane encoding a tree serially took about 770 cycles per node, measured.)
constexpr int kEncThreads = 32;
constexpr int kEncWordsPerLane = 2 * GP_DEVICE_ENCODE_MAX_NODES / kEncThreads;  // 16
constexpr int kEncNodesPerLane = GP_DEVICE_ENCODE_MAX_NODES / kEncThreads;      // 8
static_assert(kEncWordsPerLane <= 32, "word flags are kept in one 32-bit mask");

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

// gpisa::xif_form_index by the valid-descriptor masks (no scan)
__device__ __forceinline__ int xif_index(int dc, int da, int db) {
  constexpr uint64_t lo = xif_valid_mask(0), hi = xif_valid_mask(64);
  const int t = dc * 25 + da * 5 + db;
  return t < 64 ? __popcll(lo & ((1ull << t) - 1)) : __popcll(lo) + __popcll(hi & ((1ull << (t - 64)) - 1));
}

__device__ int xbin(uint32_t op) {
  return op == GP_OP_GT ? XB_GT : op == GP_OP_LT ? XB_LT : op == GP_OP_EQ ? XB_EQ
                                : op == GP_OP_AND ? XB_AND : XB_OR;
}

__device__ __forceinline__ int enc_arity(const EncScratch& s, int v) { return s.opa[v] >> 6; }

// A function node u whose children are all finished: the levels its subtree
// needs, the evaluation order of its function children (by decreasing need,
// stable, for GP_ORDER_MIN_DEPTH; operand order for GP_ORDER_PAPER) and the
// function nodes of its subtree.  A function child placed k-th is evaluated
// at level l + k, so the subtree needs max over k of (k + the child's need).
__device__ __forceinline__ void enc_finish(EncScratch& s, int u, int ar, int order) {
  int rk0 = 0, rk1 = 0, rk2 = 0, nd0 = -1, nd1 = -1, nd2 = -1, m = 0, f = 1;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (q < ar) {
      const int c = s.ch[q][u];
      const int nd = s.need[c];
      if (nd > 0) {
        if (m == 0) { rk0 = q; nd0 = nd; }
        else if (m == 1) { rk1 = q; nd1 = nd; }
        else { rk2 = q; nd2 = nd; }
        ++m;
        f += s.fc[c];
      }
    }
  }
  if (order == GP_ORDER_MIN_DEPTH) {  // a stable exchange network; empty slots (-1) stay last
    int t;
    if (nd1 > nd0) { t = nd0; nd0 = nd1; nd1 = t; t = rk0; rk0 = rk1; rk1 = t; }
    if (nd2 > nd1) { t = nd1; nd1 = nd2; nd2 = t; t = rk1; rk1 = rk2; rk2 = t; }
    if (nd1 > nd0) { t = nd0; nd0 = nd1; nd1 = t; t = rk0; rk0 = rk1; rk1 = t; }
  }
  int need = 1;
  if (m > 0) need = max(need, nd0);
  if (m > 1) need = max(need, 1 + nd1);
  if (m > 2) need = max(need, 2 + nd2);
  s.need[u] = (uint8_t)min(need, 255);
  s.ord[u] = (uint8_t)(((uint32_t)m << 6) | (uint32_t)rk0 | ((uint32_t)rk1 << 2) | ((uint32_t)rk2 << 4));
  s.fc[u] = (uint8_t)f;
}

// The S-form instruction of function node v with its result at level l: its
// code from the opcode and the operand kinds (input, constant, or stack level
// l + r for the function child evaluated r-th); payloads in operand order.
__device__ __forceinline__ uint4 enc_instruction(const EncScratch& s, int v, int l) {
  const uint32_t op = s.opa[v] & 63u;
  const int ar = enc_arity(s, v);
  const uint32_t od = s.ord[v];
  const int np = (int)(od >> 6);
  int k0 = 0, k1 = 0, k2 = 0;  // 0 input, 1 constant, 2 + r stack level l + r
  uint32_t p0 = 0u, p1 = 0u, p2 = 0u;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (q < ar) {
      const int c = s.ch[q][v];
      if (enc_arity(s, c) == 0) {
        const bool var = (s.opa[c] & 63u) == GP_OP_VAR;
        const uint32_t pay = var ? (s.tok[s.pos[c]] >> 8) : s.tok[s.pos[c] + 1];
        const int kind = var ? 0 : 1;
        if (q == 0) { k0 = kind; p0 = pay; }
        else if (q == 1) { k1 = kind; p1 = pay; }
        else { k2 = kind; p2 = pay; }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    if (r < np) {
      const uint32_t q = (od >> (2 * r)) & 3u;
      if (q == 0) k0 = 2 + r;
      else if (q == 1) k1 = 2 + r;
      else k2 = 2 + r;
    }
  }
  uint32_t code;
  if (ar == 1) {
    const int uf = k0 == 0 ? UF_X : k0 == 1 ? UF_C : UF_S;
    code = (uint32_t)sfx_un_code(uf, l, (int)(op - GP_OP_SIN));
  } else if (ar == 3) {
    code = (uint32_t)sfx_if_code(xif_index(k0, k1, k2), l);
  } else {
    // forms by (a, b): X X, X C, C X, C C, S0 X, X S0, S0 C, C S0, S0 S1, S1 S0
    int form;
    if (k0 < 2 && k1 < 2) form = k0 == 0 ? (k1 == 0 ? SF_XX : SF_XC) : (k1 == 0 ? SF_CX : SF_CC);
    else if (k0 == 2 && k1 < 2) form = k1 == 0 ? SF_SX : SF_SC;
    else if (k1 == 2 && k0 < 2) form = k0 == 0 ? SF_XS : SF_CS;
    else form = k0 == 2 ? SF_SS : SF_SSR;
    if (op == GP_OP_DIV && k1 == 1 && div_fast_operand(p1) && (k0 != 1 || div_fast_operand(p0))) {
      // a constant divisor inside the fast range: its reciprocal rounded to
      // nearest even in payload c, as the host encoder writes it
      form = k0 == 0 ? SF_XI : k0 == 1 ? SF_CI : SF_SI;
      p2 = __float_as_uint(__frcp_rn(__uint_as_float(p1)));
    }
    code = (op >= GP_OP_ADD && op <= GP_OP_DIV) ? (uint32_t)sform_code(form, l, (int)(op - GP_OP_ADD))
                                               : (uint32_t)sfx_bin_code(form, l, xbin(op));
  }
  return make_uint4(code, p0, p1, p2);
}

__device__ __forceinline__ int enc_warp_scan(int x, int lane) {  // inclusive prefix sum
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  return x;
}

// One tree per warp (Sec. 5's conversion, every step over the lanes):
// (1) the words' node starts (a scan over a two-state automaton: a word is a
//     node unless it is a constant's payload) and each node's opcode and arity;
// (2) open[v], the sum of (arity - 1) over the nodes before v (a scan);
// (3) each node's parent, the nearest earlier node u with open[u] <= open[v],
//     and its operand position open[u] - open[v] + arity(u) - 1;
// (4) from the leaves up, in rounds, each function node's need, child order
//     and function count;
// (5) the S-form post-order placement: a node's function children in
//     evaluation order take levels l, l + 1, ... and consecutive runs of
//     instructions from the start of the node's own run, which the node's
//     instruction ends -- path sums from the root, by pointer jumping;
// (6) the instructions, one node per lane.
// The words are the host encoder's (encode.cpp) for the same tree.  The
// warp's control flow is uniform: `ok` and n come from warp votes and
// shuffles.
__global__ void __launch_bounds__(kEncThreads) encode_kernel(EncArgs a) {
  extern __shared__ EncScratch enc_s[];
  const int p = blockIdx.x;  // one tree per block (a single warp)
  if (p >= a.n_progs) return;
  EncScratch& s = enc_s[0];
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x;
  const int len = a.lengths[p];
  uint32_t* o = a.out + a.out_offsets[p];
  uint32_t* ins = o + 4;
  bool ok = len > 0 && len <= 2 * GP_DEVICE_ENCODE_MAX_NODES;
  if (ok) {
    const uint32_t* g = a.words + a.offsets[p];
    for (int w = lane; w < len; w += kEncThreads) s.tok[w] = g[w];
  }
  __syncwarp();
  int n = 0, max_input = -1, depth = 1;
  bool extended = false;
  if (ok) {
    // 1. node starts.  A lane's words map the state on entry (0: at a node,
    //    1: at a payload) to the state on exit; a scan of the maps gives each
    //    lane its entry state.
    const int w0 = lane * kEncWordsPerLane;
    uint32_t cmask = 0u, m0 = 0u, m1 = 1u;
    for (int i = 0; i < kEncWordsPerLane; ++i) {
      if (w0 + i < len) {
        const bool c = (s.tok[w0 + i] & 0xffu) == GP_OP_CONST;
        cmask |= (uint32_t)c << i;
        m0 = (m0 == 0u && c) ? 1u : 0u;
        m1 = (m1 == 0u && c) ? 1u : 0u;
      }
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {  // the maps of lanes <= lane, composed
      const uint32_t p0 = __shfl_up_sync(kAll, m0, d), p1 = __shfl_up_sync(kAll, m1, d);
      if (lane >= d) {
        const uint32_t n0 = p0 == 0u ? m0 : m1, n1 = p1 == 0u ? m0 : m1;
        m0 = n0;
        m1 = n1;
      }
    }
    uint32_t st = __shfl_up_sync(kAll, m0, 1);
    if (lane == 0) st = 0u;
    const bool ends_in_payload = __shfl_sync(kAll, m0, 31) != 0u;  // a constant without its word
    uint32_t smask = 0u;
    for (int i = 0; i < kEncWordsPerLane; ++i) {
      if (w0 + i < len) {
        if (st == 0u) smask |= 1u << i;
        st = (st == 0u && ((cmask >> i) & 1u)) ? 1u : 0u;
      }
    }
    const int cnt = __popc(smask);
    const int incl = enc_warp_scan(cnt, lane);
    n = __shfl_sync(kAll, incl, 31);
    ok = !ends_in_payload && n <= GP_DEVICE_ENCODE_MAX_NODES;
    if (ok) {
      bool bad = false, ext = false;
      int mi = -1, idx = incl - cnt;
      for (uint32_t b = smask; b; b &= b - 1) {
        const int w = w0 + __ffs(b) - 1;
        const uint32_t tk = s.tok[w], op = tk & 0xffu;
        int ar = 0;
        if (op == GP_OP_VAR) {
          mi = max(mi, (int)(tk >> 8));
        } else if (op != GP_OP_CONST) {
          ar = fn_arity(op);
          if (ar < 0) { bad = true; ar = 0; }
          if (!(op >= GP_OP_ADD && op <= GP_OP_DIV)) ext = true;
        }
        s.pos[idx] = (uint16_t)w;
        s.opa[idx] = (uint8_t)((op & 63u) | ((uint32_t)ar << 6));
        ++idx;
      }
      ok = !__any_sync(kAll, bad);
      extended = __any_sync(kAll, ext);
      max_input = __reduce_max_sync(kAll, mi);
    }
  }
  if (ok) {
    __syncwarp();
    // 2. open[v]; a tree has open[v] >= 0 for v >= 1 and a total of -1
    const int v0 = lane * kEncNodesPerLane;
    int loc = 0;
    for (int i = 0; i < kEncNodesPerLane; ++i)
      if (v0 + i < n) loc += enc_arity(s, v0 + i) - 1;
    const int incl = enc_warp_scan(loc, lane);
    int run = incl - loc;
    bool neg = false;
    for (int i = 0; i < kEncNodesPerLane; ++i) {
      const int v = v0 + i;
      if (v < n) {
        s.u.open[v] = (int16_t)run;
        if (v > 0 && run < 0) neg = true;  // tokens after a complete tree
        run += enc_arity(s, v) - 1;
      }
    }
    ok = !__any_sync(kAll, neg) && __shfl_sync(kAll, incl, 31) == -1;  // else operands missing
  }
  if (ok) {
    __syncwarp();
    // 3. parents and children (the slots opened after u stay filled until v)
    bool bad = false;
    for (int v = lane; v < n; v += kEncThreads) {
      s.need[v] = 0;
      s.ord[v] = 0;
      s.fc[v] = 0;
      if (v == 0) {
        s.par[0] = 0;
        continue;
      }
      const int ov = s.u.open[v];
      int u = v - 1;
      while (u > 0 && s.u.open[u] > ov) --u;
      const int au = enc_arity(s, u);
      const int k = s.u.open[u] - ov + au - 1;
      if (k < 0 || k >= au) {  // cannot happen for a tree that passed (2)
        bad = true;
        continue;
      }
      s.ch[k][u] = (uint8_t)v;
      s.par[v] = (uint8_t)u;
    }
    ok = !__any_sync(kAll, bad);
  }
  if (ok) {
    __syncwarp();
    // 4. each round finishes the unfinished function nodes of greatest
    //    height (all their function children finished): at most n rounds
    uint32_t pend = 0u;  // bit j: node lane + 32 j, an unfinished function node
    for (int j = 0; j < kEncNodesPerLane; ++j) {
      const int v = lane + kEncThreads * j;
      if (v < n && enc_arity(s, v) > 0) pend |= 1u << j;
    }
    for (int round = 0; round < n && __any_sync(kAll, pend != 0u); ++round) {
      uint32_t ready = 0u;
      for (uint32_t b = pend; b; b &= b - 1) {
        const int j = __ffs(b) - 1, v = lane + kEncThreads * j, ar = enc_arity(s, v);
        bool r = true;
        for (int q = 0; q < ar; ++q) {
          const int c = s.ch[q][v];
          if (enc_arity(s, c) > 0 && s.need[c] == 0) r = false;
        }
        if (r) ready |= 1u << j;
      }
      __syncwarp();
      for (uint32_t b = ready; b; b &= b - 1) {
        const int v = lane + kEncThreads * (__ffs(b) - 1);
        enc_finish(s, v, enc_arity(s, v), a.order);
      }
      pend &= ~ready;
      __syncwarp();
    }
    ok = !__any_sync(kAll, pend != 0u);
    depth = enc_arity(s, 0) > 0 ? s.need[0] : 1;
    if (depth > R) ok = false;
  }
  const bool fn_root = ok && enc_arity(s, 0) > 0;
  if (fn_root) {
    // 5. a function node's step from its parent: the function nodes of the
    //    children evaluated before it | its rank << 16; then path sums
    //    (a path has at most 255 edges: 8 doublings)
    for (int v = lane; v < n; v += kEncThreads) {
      if (enc_arity(s, v) == 0) continue;
      int d = 0;
      if (v > 0) {
        const int u = s.par[v];
        const uint32_t od = s.ord[u];
        const int np = (int)(od >> 6);
        int off = 0, r = 0;
        bool found = false;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          if (t < np && !found) {
            const int c = s.ch[(od >> (2 * t)) & 3u][u];
            if (c == v) { found = true; r = t; } else { off += s.fc[c]; }
          }
        }
        d = off | (r << 16);
      }
      s.u.path[v] = d;
    }
    __syncwarp();
    for (int round = 0; round < 8; ++round) {
      int nv[kEncNodesPerLane], nj[kEncNodesPerLane];
      bool more = false;
#pragma unroll
      for (int j = 0; j < kEncNodesPerLane; ++j) {
        const int v = lane + kEncThreads * j;
        nv[j] = 0;
        nj[j] = 0;
        if (v < n && enc_arity(s, v) > 0) {
          const int jv = s.par[v];
          nv[j] = s.u.path[v] + s.u.path[jv];
          nj[j] = s.par[jv];
          more |= jv != 0;
        }
      }
      if (!__any_sync(kAll, more)) break;  // every link at the root: the sums are complete
      __syncwarp();
#pragma unroll
      for (int j = 0; j < kEncNodesPerLane; ++j) {
        const int v = lane + kEncThreads * j;
        if (v < n && enc_arity(s, v) > 0) {
          s.u.path[v] = nv[j];
          s.par[v] = (uint8_t)nj[j];
        }
      }
      __syncwarp();
    }
  }
  if (lane == 0) {
    if (!ok) {  // a header of kind 0: every evaluation reports the program as malformed
      o[0] = 0u; o[1] = 0u; o[2] = 0u; o[3] = 0u;
      a.out_lengths[p] = 4;
    } else {
      int ni = 1;
      if (!fn_root) {  // a single terminal: one move to level 0
        const bool cst = (s.opa[0] & 63u) == GP_OP_CONST;
        ins[0] = (uint32_t)sform_code(cst ? SF_MOVC : SF_MOVX, 0, 0);
        ins[1] = cst ? s.tok[1] : (s.tok[0] >> 8);
        ins[2] = 0u;
        ins[3] = 0u;
      } else {
        ni = s.fc[0];
      }
      o[0] = header0(extended ? (uint32_t)K_SFORMX : (uint32_t)K_SFORM, (uint32_t)a.order);
      o[1] = (uint32_t)ni;
      o[2] = (uint32_t)n;
      o[3] = (uint32_t)depth | ((uint32_t)(max_input + 1) << 16);
      a.out_lengths[p] = 4 + 4 * ni;
      if (a.node_total) atomicAdd(a.node_total, (unsigned long long)n);
    }
  }
  if (fn_root) {
    // 6. the instructions (16-byte stores where the slot is aligned, as
    //    offsets in multiples of 4 words make it)
    const bool vec = (reinterpret_cast<uintptr_t>(ins) & 15u) == 0;
    const int ni = s.fc[0];
    for (int v = lane; v < n; v += kEncThreads) {
      if (enc_arity(s, v) == 0) continue;
      const int pth = s.u.path[v];
      const int at = (pth & 0xffff) + s.fc[v] - 1;
      if (at < 0 || at >= ni) continue;  // never for a tree; keeps every store inside the slot
      const uint4 in = enc_instruction(s, v, pth >> 16);
      uint32_t* q = ins + 4 * at;
      if (vec) {
        *reinterpret_cast<uint4*>(q) = in;
      } else {
        q[0] = in.x; q[1] = in.y; q[2] = in.z; q[3] = in.w;
      }
    }
  }
}

// The back-to-back layout of the encoder's output slots: out_offsets[p] =
// the sum over q < p of 4 + 4 max(lengths[q], 0) words.  One block; each
// thread a run of consecutive programs, then a scan over the block.
__global__ void __launch_bounds__(1024) encode_slots_kernel(const int32_t* __restrict__ lengths, int32_t n,
                                                            int64_t* __restrict__ out_offsets) {
  __shared__ long long warp_before[32];
  constexpr unsigned kAll = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t per = ((int64_t)n + 1023) / 1024;
  const int64_t b = (int64_t)tid * per;
  const int64_t e = b + per < (int64_t)n ? b + per : (int64_t)n;
  long long loc = 0;
  for (int64_t p = b; p < e; ++p) loc += 4 + 4 * (long long)max(lengths[p], 0);
  long long incl = loc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long y = __shfl_up_sync(kAll, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) warp_before[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const long long w = warp_before[lane];
    long long wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long y = __shfl_up_sync(kAll, wi, d);
      if (lane >= d) wi += y;
    }
    warp_before[lane] = wi - w;
  }
  __syncthreads();
  long long run = warp_before[wid] + incl - loc;
  for (int64_t p = b; p < e; ++p) {
    out_offsets[p] = run;
    run += 4 + 4 * (long long)max(lengths[p], 0);
  }
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

extern "C" int gp_encode_slots_device(const int32_t* lengths, int32_t n_progs, int64_t* out_offsets,
                                      gp_stream_t stream) {
  gp_clear_error();
  if (n_progs < 0) return gp_fail(GP_ERR_INVALID_ARG, "negative n_progs");
  if (n_progs == 0) return GP_OK;
  if (!lengths || !out_offsets) return gp_fail(GP_ERR_INVALID_ARG, "null device array");
  encode_slots_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(lengths, n_progs, out_offsets);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "slot offsets launch: %s", cudaGetErrorString(e));
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
