// encode.cpp -- host encoder: prefix trees and register programs -> the
// instruction streams the CUDA interpreters run.
//
// Sec. 5 of the paper converts a tree (held in reverse-Polish order) into a
// prefix linear "S-form" with a symbolic stack: terminals are pushed as
// symbols, a function is written out followed by the symbols it pops, and S
// (the stack top) is pushed for its result.  This encoder does the same from
// the prefix tree, and in addition records, for every instruction, the stack
// level it reads and writes.  Levels are static in a straight-line program, so
// the interpreters keep the stack in registers addressed by constants
// (Sec. 6.2 keeps the lowest levels in registers through a switch on the
// dynamic stack pointer; the static level removes that switch).
//
// Child order.  GP_ORDER_PAPER evaluates children left to right, which is
// the converter of Sec. 5 exactly (the worked example there is a test
// fixture).  GP_ORDER_MIN_DEPTH evaluates the child that needs more levels
// first (Sethi and Ullman, "The generation of optimal code for arithmetic
// expressions", JACM 1970); the operands of every function are unchanged, so
// every per-case value is bit-identical, and any binary tree of up to 511
// functions fits the 8 register levels.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <thread>
#include <vector>

#include "../../include/gpeval.h"
#include "isa.h"
#include "status.h"

using namespace gpisa;

namespace {

struct Node {
  uint32_t op;       // user opcode
  uint32_t payload;  // input index (VAR) or binary32 bits (CONST)
  int child[3];
  int nchild;
  int need;          // stack levels needed to evaluate this subtree
};

bool is_float_fn(uint32_t op) { return op >= GP_OP_ADD && op <= GP_OP_DIV; }
bool is_bool_fn(uint32_t op) { return op >= GP_OP_AND && op <= GP_OP_IF; }
// the extended float functions (Sec. 4.2 function sets); AND, OR and IF are
// float functions in a float tree
bool is_float_unary(uint32_t op) { return op >= GP_OP_SIN && op <= GP_OP_LOG; }
bool is_float_ext(uint32_t op) {
  return is_float_unary(op) || (op >= GP_OP_GT && op <= GP_OP_EQ) || op == GP_OP_AND ||
         op == GP_OP_OR || op == GP_OP_IF;
}
int arity(uint32_t op) { return op == GP_OP_IF ? 3 : is_float_unary(op) ? 1 : 2; }
int xbin_index(uint32_t op) {
  switch (op) {
    case GP_OP_GT: return XB_GT;
    case GP_OP_LT: return XB_LT;
    case GP_OP_EQ: return XB_EQ;
    case GP_OP_AND: return XB_AND;
    default: return XB_OR;
  }
}

constexpr int64_t kMaxTokens = 16 * MAX_INSTR;

// Parses prefix tokens into nodes (index 0 = root; children after parents).
int parse_prefix(const uint32_t* w, int64_t n, bool boolean, std::vector<Node>& nodes,
                 int* max_input, bool* extended) {
  nodes.clear();
  *max_input = -1;
  *extended = false;
  if (!w || n <= 0) return gp_fail(GP_ERR_PROGRAM, "empty program");
  if (n > kMaxTokens) return gp_fail(GP_ERR_PROGRAM, "program longer than %lld words", (long long)kMaxTokens);
  struct Open { int node; int filled; };
  std::vector<Open> open;
  int64_t i = 0;
  while (i < n) {
    if (!nodes.empty() && open.empty())
      return gp_fail(GP_ERR_PROGRAM, "trailing tokens after the root's subtree at word %lld", (long long)i);
    uint32_t t = w[i];
    Node nd{};
    nd.op = t & 0xffu;
    nd.child[0] = nd.child[1] = nd.child[2] = -1;
    if (nd.op == GP_OP_VAR) {
      nd.payload = t >> 8;
      if ((int)nd.payload > *max_input) *max_input = (int)nd.payload;
      i += 1;
    } else if (nd.op == GP_OP_CONST && !boolean) {
      if (i + 1 >= n) return gp_fail(GP_ERR_PROGRAM, "constant without its value word");
      nd.payload = w[i + 1];
      i += 2;
    } else if ((boolean && is_bool_fn(nd.op)) || (!boolean && is_float_fn(nd.op))) {
      nd.nchild = arity(nd.op);
      i += 1;
    } else if (!boolean && is_float_ext(nd.op)) {
      nd.nchild = arity(nd.op);
      *extended = true;
      i += 1;
    } else {
      return gp_fail(GP_ERR_PROGRAM, "opcode %u not allowed at word %lld", nd.op, (long long)i);
    }
    int idx = (int)nodes.size();
    nodes.push_back(nd);
    if (!open.empty()) {
      Open& o = open.back();
      nodes[o.node].child[o.filled++] = idx;
      if (o.filled == nodes[o.node].nchild) open.pop_back();
    }
    if (nd.nchild > 0) open.push_back({idx, 0});
    // pop every finished ancestor
    while (!open.empty() && open.back().filled == nodes[open.back().node].nchild) open.pop_back();
  }
  if (!open.empty()) return gp_fail(GP_ERR_PROGRAM, "program ends with %d operands missing", (int)open.size());
  return GP_OK;
}

bool is_fn(const Node& n) { return n.nchild > 0; }

// evaluation order of the children of node n (indices into n.child)
void child_order(const std::vector<Node>& nodes, const Node& n, int order, bool rpn, int* perm, int* np) {
  int k = 0;
  for (int c = 0; c < n.nchild; ++c)
    if (rpn || is_fn(nodes[n.child[c]])) perm[k++] = c;
  *np = k;
  if (order == GP_ORDER_MIN_DEPTH)  // stable: ties keep left-to-right order
    std::stable_sort(perm, perm + k, [&](int a, int b) {
      return nodes[n.child[a]].need > nodes[n.child[b]].need;
    });
}

void compute_needs(std::vector<Node>& nodes, int order, bool rpn) {
  for (int i = (int)nodes.size() - 1; i >= 0; --i) {
    Node& n = nodes[i];
    if (!is_fn(n)) { n.need = rpn ? 1 : 0; continue; }
    int perm[3], np;
    child_order(nodes, n, order, rpn, perm, &np);
    int need = 1;
    for (int k = 0; k < np; ++k) need = std::max(need, k + nodes[n.child[perm[k]]].need);
    n.need = need;
  }
}

struct Emitter {
  const std::vector<Node>& nodes;
  int order;
  uint32_t kind;
  std::vector<uint32_t> ins;  // 4 words per instruction
  int stack_reads = 0;

  void put(uint32_t code, uint32_t a, uint32_t b, uint32_t c) {
    ins.push_back(code); ins.push_back(a); ins.push_back(b); ins.push_back(c);
  }

  // S-form (float or Boolean): returns nothing; result of function n at level l
  void sform(int ni, int l) {
    const Node& n = nodes[ni];
    int perm[3], np;
    child_order(nodes, n, order, false, perm, &np);
    int lvl[3] = {-1, -1, -1};  // relative stack slot of each argument (0,1,2) or -1
    for (int k = 0; k < np; ++k) {
      sform(n.child[perm[k]], l + k);
      lvl[perm[k]] = k;
    }
    uint32_t pay[3] = {0, 0, 0};
    for (int c = 0; c < n.nchild; ++c) {
      const Node& ch = nodes[n.child[c]];
      if (lvl[c] < 0) pay[c] = ch.payload; else ++stack_reads;
    }
    auto kindof = [&](int c) -> int {  // 0 X, 1 C, 2 + j stack level l + j
      const Node& ch = nodes[n.child[c]];
      if (lvl[c] >= 0) return 2 + lvl[c];
      return ch.op == GP_OP_CONST ? 1 : 0;
    };
    if (kind == K_BOOL) {
      if (n.op == GP_OP_IF) {
        int d[3];
        for (int c = 0; c < 3; ++c) d[c] = lvl[c] < 0 ? 0 : 1 + lvl[c];
        put(bool_if_code(if_form_index(d[0], d[1], d[2]), l), pay[0], pay[1], pay[2]);
        return;
      }
      int a = kindof(0), b = kindof(1), form;
      if (a == 0 && b == 0) form = BF_XX;
      else if (a == 0 && b == 2) form = BF_XS;
      else if (a == 2 && b == 0) form = BF_SX;
      else if (a == 2 && b == 3) form = BF_SS;
      else form = BF_SSR;  // a == 3 && b == 2
      put(bool_bin_code(form, l, (int)(n.op - GP_OP_AND)), pay[0], pay[1], 0);
      return;
    }
    if (n.nchild == 1) {  // SIN, COS, EXP, LOG
      const int k = kindof(0);
      const int uform = k == 0 ? UF_X : k == 1 ? UF_C : UF_S;
      put(sfx_un_code(uform, l, (int)(n.op - GP_OP_SIN)), pay[0], 0, 0);
      return;
    }
    if (n.nchild == 3) {  // float IF: descriptors X 0, C 1, stack level l+j 2+j
      const int d0 = kindof(0), d1 = kindof(1), d2 = kindof(2);
      put(sfx_if_code(xif_form_index(d0, d1, d2), l), pay[0], pay[1], pay[2]);
      return;
    }
    static const int table[4][4] = {
        // b:   X       C       S0      S1
        {SF_XX, SF_XC, SF_XS, -1},      // a = X
        {SF_CX, SF_CC, SF_CS, -1},      // a = C
        {SF_SX, SF_SC, -1, SF_SS},      // a = S0
        {-1, -1, SF_SSR, -1},           // a = S1
    };
    int form = table[kindof(0)][kindof(1)];
    if (n.op == GP_OP_DIV && kindof(1) == 1 && div_fast_operand(pay[1]) &&
        (kindof(0) != 1 || div_fast_operand(pay[0]))) {
      // a constant divisor inside the fast range: its reciprocal, rounded to
      // nearest even in binary32 (IEEE division on the host), goes to
      // payload c, and the interpreter divides with a multiplication and one
      // remainder correction
      float b;
      memcpy(&b, &pay[1], 4);
      const float y = 1.0f / b;
      uint32_t ybits;
      memcpy(&ybits, &y, 4);
      const int k0 = kindof(0);
      const int iform = k0 == 0 ? SF_XI : k0 == 1 ? SF_CI : SF_SI;
      put(sform_code(iform, l, F_DIV), pay[0], pay[1], ybits);
      return;
    }
    if (is_float_fn(n.op)) put(sform_code(form, l, (int)(n.op - GP_OP_ADD)), pay[0], pay[1], 0);
    else put(sfx_bin_code(form, l, xbin_index(n.op)), pay[0], pay[1], 0);
  }

  // postfix (RPN): the value of node n ends on level l
  void rpn(int ni, int l) {
    const Node& n = nodes[ni];
    if (!is_fn(n)) {
      if (n.op == GP_OP_CONST) put(rpn_code(RF_PUSHC, l, 0), n.payload, 0, 0);
      else put(rpn_code(RF_PUSHX, l, 0), n.payload, 0, 0);
      return;
    }
    int perm[3], np;
    child_order(nodes, n, order, true, perm, &np);
    for (int k = 0; k < np; ++k) rpn(n.child[perm[k]], l + k);
    stack_reads += n.nchild;
    if (n.nchild == 1) {  // SIN, COS, EXP, LOG on level l
      put(rpx_un_code(l, (int)(n.op - GP_OP_SIN)), 0, 0, 0);
      return;
    }
    if (n.nchild == 3) {  // float IF: its operands on levels l .. l+2 in evaluation order
      int lvl[3];
      for (int k = 0; k < 3; ++k) lvl[perm[k]] = k;
      put(rpx_if_code(rpx_perm_index(lvl[0], lvl[1], lvl[2]), l), 0, 0, 0);
      return;
    }
    int form = (perm[0] == 0) ? RF_OP : RF_OPR;  // first argument on level l or l+1
    if (is_float_fn(n.op)) put(rpn_code(form, l, (int)(n.op - GP_OP_ADD)), 0, 0, 0);
    else put(rpx_bin_code(form == RF_OP ? 0 : 1, l, xbin_index(n.op)), 0, 0, 0);
  }
};

int encode_one(const uint32_t* prefix, int64_t n_words, int32_t kind, int32_t order,
               std::vector<uint32_t>& out, gp_prog_info* info) {
  if (kind != K_SFORM && kind != K_RPN && kind != K_BOOL)
    return gp_fail(GP_ERR_INVALID_ARG, "kind %d is not a tree kind", kind);
  if (order != GP_ORDER_PAPER && order != GP_ORDER_MIN_DEPTH)
    return gp_fail(GP_ERR_INVALID_ARG, "unknown order %d", order);
  std::vector<Node> nodes;
  int max_input = -1;
  bool extended = false;
  int rc = parse_prefix(prefix, n_words, kind == K_BOOL, nodes, &max_input, &extended);
  if (rc) return rc;
  const bool rpn = (kind == K_RPN);
  compute_needs(nodes, order, rpn);
  Emitter em{nodes, order, (uint32_t)kind, {}, 0};
  em.ins.reserve(16 * nodes.size());
  int depth;
  if (rpn) {
    em.rpn(0, 0);
    depth = nodes[0].need;
  } else if (is_fn(nodes[0])) {
    em.sform(0, 0);
    depth = nodes[0].need;
  } else {  // a single terminal: one move to level 0
    const Node& t = nodes[0];
    if (kind == K_BOOL) em.put(BOOL_MOVX, t.payload, 0, 0);
    else em.put(sform_code(t.op == GP_OP_CONST ? SF_MOVC : SF_MOVX, 0, 0), t.payload, 0, 0);
    depth = 1;
  }
  int n_instr = (int)(em.ins.size() / 4);
  gp_prog_info inf{};
  inf.n_nodes = (int)nodes.size();
  inf.n_instr = n_instr;
  inf.max_depth = depth;
  inf.stack_reads = em.stack_reads;
  inf.max_input = max_input;
  inf.words = 4 + 4 * n_instr;
  inf.extended = extended ? 1 : 0;
  {
    std::vector<uint32_t> vars;
    for (const Node& nd : nodes)
      if (nd.op == GP_OP_VAR) vars.push_back(nd.payload);
    std::sort(vars.begin(), vars.end());
    inf.inputs_used = (int32_t)(std::unique(vars.begin(), vars.end()) - vars.begin());
  }
  if (info) *info = inf;
  if (depth > R)
    return gp_fail(GP_ERR_PROGRAM, "program needs %d stack levels, more than %d (encode with GP_ORDER_MIN_DEPTH)", depth, R);
  if (n_instr > MAX_INSTR)
    return gp_fail(GP_ERR_PROGRAM, "program has %d instructions, more than %d", n_instr, MAX_INSTR);
  out.clear();
  out.push_back(header0(extended ? (uint32_t)(rpn ? K_RPNX : K_SFORMX) : (uint32_t)kind, (uint32_t)order));
  out.push_back((uint32_t)n_instr);
  out.push_back((uint32_t)inf.n_nodes);
  out.push_back((uint32_t)depth | ((uint32_t)(max_input + 1) << 16));
  out.insert(out.end(), em.ins.begin(), em.ins.end());
  return GP_OK;
}

}  // namespace

extern "C" int gp_encode_tree(const uint32_t* prefix, int64_t n_words, int32_t kind, int32_t order,
                              uint32_t* out, int64_t cap_words, gp_prog_info* info) {
  gp_clear_error();
  std::vector<uint32_t> buf;
  gp_prog_info inf{};
  int rc = encode_one(prefix, n_words, kind, order, buf, &inf);
  if (info) *info = inf;
  if (rc) return rc;
  if (!out || cap_words < (int64_t)buf.size())
    return gp_fail(GP_ERR_INVALID_ARG, "output capacity %lld < %zu words", (long long)cap_words, buf.size());
  memcpy(out, buf.data(), buf.size() * sizeof(uint32_t));
  return GP_OK;
}

// Population encoding runs on several host threads: programs are split into
// contiguous ranges, each thread encodes its range into its own buffer, and
// the buffers are laid out in program order.  The result is identical to a
// sequential encoding.
namespace {
struct Piece {
  std::vector<uint32_t> words;
  std::vector<int32_t> lengths;
  int64_t nodes = 0;
  int rc = GP_OK;
  int32_t bad = -1;
  std::string msg;
};

int encode_threads(int32_t n_progs) {
  unsigned hc = std::thread::hardware_concurrency();
  int t = (int)std::min<unsigned>(hc ? hc : 1, 32);
  return std::max(1, std::min<int>(t, n_progs / 128));
}
}  // namespace

extern "C" int gp_encode_population(const uint32_t* words, const int64_t* offsets,
                                    const int32_t* lengths, int32_t n_progs, int32_t kind,
                                    int32_t order, uint32_t* out, int64_t cap_words,
                                    int64_t* out_offsets, int32_t* out_lengths,
                                    int64_t* total_words, int64_t* total_nodes,
                                    gp_prog_info* info, int32_t* bad_prog) {
  gp_clear_error();
  if (bad_prog) *bad_prog = -1;
  if (n_progs < 0 || (n_progs > 0 && (!words || !offsets || !lengths)))
    return gp_fail(GP_ERR_INVALID_ARG, "bad population arguments");
  if (out && (!out_offsets || !out_lengths))
    return gp_fail(GP_ERR_INVALID_ARG, "out_offsets and out_lengths are required with out");
  const int nt = encode_threads(n_progs);
  std::vector<Piece> pieces(nt);
  auto work = [&](int t) {
    const int32_t b = (int32_t)((int64_t)n_progs * t / nt), e = (int32_t)((int64_t)n_progs * (t + 1) / nt);
    Piece& pc = pieces[t];
    std::vector<uint32_t> buf;
    for (int32_t p = b; p < e; ++p) {
      gp_prog_info inf{};
      int rc;
      if (lengths[p] <= 0 || offsets[p] < 0)
        rc = gp_fail(GP_ERR_PROGRAM, "program %d has no words", p);
      else
        rc = encode_one(words + offsets[p], lengths[p], kind, order, buf, &inf);
      if (info) info[p] = inf;
      if (rc) {
        pc.rc = rc;
        pc.bad = p;
        pc.msg = gp_error_string();
        return;
      }
      pc.words.insert(pc.words.end(), buf.begin(), buf.end());
      pc.lengths.push_back((int32_t)buf.size());
      pc.nodes += inf.n_nodes;
    }
  };
  if (nt == 1) {
    work(0);
  } else {
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) th.emplace_back(work, t);
    for (auto& x : th) x.join();
  }
  int64_t pos = 0, nodes = 0;
  for (int t = 0; t < nt; ++t) {
    if (pieces[t].rc) {  // the first bad program in program order
      if (bad_prog) *bad_prog = pieces[t].bad;
      return gp_fail(pieces[t].rc, "%s", pieces[t].msg.c_str());
    }
    pos += (int64_t)pieces[t].words.size();
    nodes += pieces[t].nodes;
  }
  if (total_words) *total_words = pos;
  if (total_nodes) *total_nodes = nodes;
  if (!out) return GP_OK;
  if (pos > cap_words)
    return gp_fail(GP_ERR_INVALID_ARG, "output capacity %lld < %lld words", (long long)cap_words, (long long)pos);
  int64_t w = 0;
  int32_t p = 0;
  for (int t = 0; t < nt; ++t) {
    memcpy(out + w, pieces[t].words.data(), pieces[t].words.size() * sizeof(uint32_t));
    for (int32_t len : pieces[t].lengths) {
      out_offsets[p] = w;
      out_lengths[p] = len;
      w += len;
      ++p;
    }
  }
  return GP_OK;
}

extern "C" int gp_encode_linear_population(const uint8_t* instr, const int64_t* offsets,
                                           const int32_t* lengths, int32_t n_progs,
                                           uint32_t* out, int64_t cap_words,
                                           int64_t* out_offsets, int32_t* out_lengths,
                                           int64_t* total_words, int64_t* total_nodes,
                                           int32_t* bad_prog) {
  gp_clear_error();
  if (bad_prog) *bad_prog = -1;
  if (n_progs < 0 || (n_progs > 0 && (!instr || !offsets || !lengths)))
    return gp_fail(GP_ERR_INVALID_ARG, "bad population arguments");
  if (out && (!out_offsets || !out_lengths))
    return gp_fail(GP_ERR_INVALID_ARG, "out_offsets and out_lengths are required with out");
  int64_t pos = 0, nodes = 0;
  for (int32_t p = 0; p < n_progs; ++p) {
    int32_t n = lengths[p];
    if (n < 0 || n > MAX_INSTR || offsets[p] < 0) {
      if (bad_prog) *bad_prog = p;
      return gp_fail(GP_ERR_PROGRAM, "register program %d has %d instructions (0..%d allowed)", p, n, MAX_INSTR);
    }
    const uint8_t* ins = instr + offsets[p] * 4;
    for (int32_t i = 0; i < n; ++i) {
      uint8_t d = ins[4 * i], op = ins[4 * i + 1], a = ins[4 * i + 2], b = ins[4 * i + 3];
      if (d >= NREG || a >= NREG || b >= NREG || !is_float_fn(op)) {
        if (bad_prog) *bad_prog = p;
        return gp_fail(GP_ERR_PROGRAM, "register program %d instruction %d is malformed", p, i);
      }
    }
    int64_t words = 4 + 4 * (int64_t)n;
    if (out) {
      if (pos + words > cap_words)
        return gp_fail(GP_ERR_INVALID_ARG, "output capacity %lld too small", (long long)cap_words);
      uint32_t* o = out + pos;
      o[0] = header0(K_LINEAR, 0);
      o[1] = (uint32_t)n;
      o[2] = (uint32_t)n;
      o[3] = 0;
      // Payload b carries flags for the interpreter with the registers in
      // shared memory (the register variant ignores them).  That
      // interpreter keeps two values in machine registers: A, the previous
      // instruction's result, and B, a value it loaded from the register
      // file earlier.  Bits 0-1: where operand a comes from (0 the file, 1
      // A, 2 B); bits 2-3: operand b likewise (at most one operand from A
      // or B); bit 4: the result is
      // overwritten before anything reads it from the file (a read from A
      // or B does not count) and it is not register 0 at the end.
      // Forward pass: A holds register d of the previous instruction; B
      // holds the register whose value the body's fixed rules last loaded
      // into B (operand a from the file is loaded into A, or into B when b
      // is A; operand b from the file into B, or into A when a is B), valid
      // until that register is written.
      int a_reg = -1, b_reg = -1;
      for (int32_t i = 0; i < n; ++i) {
        const uint8_t d = ins[4 * i], op = ins[4 * i + 1], a = ins[4 * i + 2], b = ins[4 * i + 3];
        auto src = [&](int r) -> uint32_t { return r == a_reg ? 1u : (r == b_reg ? 2u : 0u); };
        // (both operands from A or B -- 6% of the instructions of random
        // programs -- take b from the file: the interpreter has no bodies for
        // them, which keeps its code small)
        const uint32_t sa = src(a), sb = sa ? 0u : src(b);
        int nb = b_reg;
        if (sa == 0 && sb == 0) nb = b;
        else if (sa == 0 && sb == 1) nb = a;
        else if (sa == 1 && sb == 0) nb = b;
        a_reg = d;
        b_reg = nb == d ? -1 : nb;
        o[4 + 4 * i] = (uint32_t)lin_code(op - GP_OP_ADD, a, b);
        o[5 + 4 * i] = d;
        o[6 + 4 * i] = sa | (sb << 2);
        o[7 + 4 * i] = 0;
      }
      // Backward pass from {register 0}: registers whose value in the file
      // a later read from the file (or the output) needs.
      uint32_t live = 1u;
      for (int32_t i = n - 1; i >= 0; --i) {
        const uint8_t d = ins[4 * i], a = ins[4 * i + 2], b = ins[4 * i + 3];
        const uint32_t f = o[6 + 4 * i];
        const uint32_t dead = (live >> d) & 1u ? 0u : 1u;
        live &= ~(1u << d);
        if ((f & 3u) == 0) live |= 1u << a;
        if (((f >> 2) & 3u) == 0) live |= 1u << b;
        o[6 + 4 * i] = f | (dead << 4);
      }
      out_offsets[p] = pos;
      out_lengths[p] = (int32_t)words;
    }
    pos += words;
    nodes += n;
  }
  if (total_words) *total_words = pos;
  if (total_nodes) *total_nodes = nodes;
  return GP_OK;
}
