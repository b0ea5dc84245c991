// isa.h -- instruction codes of the encoded programs, shared by the host
// encoder and the CUDA interpreters (both are product code).
//
// Every interpreter instruction is four uint32 words {code, pa, pb, pc}.  The
// code is dense so that the interpreters dispatch with one jump table; it
// folds together the function, the kind of each operand and the stack level
// the instruction works on.  Stack levels are known statically for a
// straight-line program (Sec. 5: the symbolic-stack conversion already knows,
// at each function, which operands come from the stack), so the level is part
// of the code and the register interpreters index their stack registers with
// compile-time constants.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define GPISA_HD __host__ __device__
#else
#define GPISA_HD
#endif

namespace gpisa {

constexpr int R = 8;            // stack levels held per case (GP_STACK_LEVELS)
constexpr int MAX_INSTR = 1024; // GP_MAX_INSTR
constexpr uint32_t VERSION = 2;  // 2: the reciprocal-divisor S-forms

enum Kind : uint32_t { K_SFORM = 1, K_RPN = 2, K_LINEAR = 3, K_BOOL = 4, K_SFORMX = 5, K_RPNX = 6 };

// float function index = user opcode - 1 (ADD, SUB, MUL, DIV)
enum FOp : int { F_ADD = 0, F_SUB = 1, F_MUL = 2, F_DIV = 3 };

// ---- float S-form (Sec. 5): operands X = input, C = constant, S0/S1 = the
// stack level l / l+1; the result is written to level l.
enum SForm : int {
  SF_XX = 0, SF_XC, SF_CX, SF_CC,  // no stack operand
  SF_SX, SF_XS, SF_SC, SF_CS,      // one stack operand at level l
  SF_SS,                            // a = level l, b = level l+1
  SF_SSR,                           // a = level l+1, b = level l
  SF_MOVX, SF_MOVC,                 // a program that is a single terminal
  // division (op F_DIV only) by a constant b (payload b) whose binary32
  // reciprocal RN(1/b) the encoder supplies in payload c; the numerator is an
  // input, stack level l or a constant.  Used when div_fast_operand(b) holds
  // (and, for SF_CI, div_fast_operand(a)); other constant divisors keep the
  // SF_XC, SF_SC, SF_CC forms.
  SF_XI, SF_SI, SF_CI,
  SF_NFORMS
};
GPISA_HD constexpr int sform_code(int form, int level, int op) { return (form * R + level) * 4 + op; }
constexpr int SF_NCODES = SF_NFORMS * R * 4;
// A binary32 operand (bit pattern) inside the fast range of the division
// sequences, 2^-50 <= |v| <= 2^50 (finite, normal): within it every
// intermediate value of the reciprocal-and-remainder sequences is normal.
GPISA_HD constexpr bool div_fast_operand(uint32_t bits) {
  return (bits & 0x7fffffffu) >= 0x26800000u && (bits & 0x7fffffffu) <= 0x58800000u;
}

// ---- extended float S-form (the function sets of Sec. 4.2's float
// problems).  Its code space starts with the basic S-form's codes, unchanged,
// so the extended interpreter also runs basic programs; the extended codes
// follow.  Comparisons and logic GT, LT, EQ, AND, OR take the ten binary
// operand forms SF_XX..SF_SSR; the unary functions SIN, COS, EXP, LOG take an
// input, a constant or the stack level l as operand; IF(c, a, b) takes each
// operand as an input (0), a constant (1) or stack level l + j (2 + j), the
// stack operands using exactly the levels l .. l + m - 1.  Every result goes
// to level l.
enum XBin : int { XB_GT = 0, XB_LT, XB_EQ, XB_AND, XB_OR, XB_NOPS };
enum XUn : int { XU_SIN = 0, XU_COS, XU_EXP, XU_LOG, XU_NOPS };
enum UForm : int { UF_X = 0, UF_C, UF_S, UF_NFORMS };
constexpr int SFX_BIN_BASE = SF_NFORMS * R * 4;  // 480
GPISA_HD constexpr int sfx_bin_code(int form, int level, int op) {
  return SFX_BIN_BASE + (form * R + level) * XB_NOPS + op;  // form SF_XX..SF_SSR
}
constexpr int SFX_UN_BASE = SFX_BIN_BASE + (SF_SSR + 1) * R * XB_NOPS;  // 880
GPISA_HD constexpr int sfx_un_code(int uform, int level, int fn) {
  return SFX_UN_BASE + (uform * R + level) * XU_NOPS + fn;
}
constexpr int SFX_IF_BASE = SFX_UN_BASE + UF_NFORMS * R * XU_NOPS;  // 976
// operand descriptor d in 0..4 (X, C, S0, S1, S2); valid when the stack
// operands use exactly levels l .. l+m-1, each once
GPISA_HD constexpr bool xif_desc_valid(int dc, int da, int db) {
  int m = (dc >= 2) + (da >= 2) + (db >= 2);
  bool used[3] = {false, false, false};
  const int d[3] = {dc, da, db};
  for (int i = 0; i < 3; ++i) {
    if (d[i] < 2) continue;
    const int j = d[i] - 2;
    if (j >= m || used[j]) return false;
    used[j] = true;
  }
  return true;
}
// descriptors numbered in increasing order of dc*25 + da*5 + db
GPISA_HD constexpr int xif_form_index(int dc, int da, int db) {
  int idx = 0;
  for (int t = 0; t < dc * 25 + da * 5 + db; ++t)
    if (xif_desc_valid(t / 25, (t / 5) % 5, t % 5)) ++idx;
  return idx;
}
GPISA_HD constexpr int xif_form_desc(int idx) {  // inverse: dc*25 + da*5 + db
  int seen = 0;
  for (int t = 0; t < 125; ++t)
    if (xif_desc_valid(t / 25, (t / 5) % 5, t % 5)) { if (seen == idx) return t; ++seen; }
  return -1;
}
constexpr int SFX_IF_FORMS = 38;
// xif_form_desc without the scan, for the kernels' per-instruction decoding:
// the 38 descriptors (7 bits each) packed nine to a 64-bit constant
GPISA_HD constexpr uint64_t xif_desc_pack(int first) {
  uint64_t w = 0;
  for (int j = 0; j < 9 && first + j < SFX_IF_FORMS; ++j) w |= (uint64_t)xif_form_desc(first + j) << (7 * j);
  return w;
}
GPISA_HD constexpr int xif_form_desc_fast(int idx) {  // idx in [0, SFX_IF_FORMS)
  constexpr uint64_t w0 = xif_desc_pack(0), w1 = xif_desc_pack(9), w2 = xif_desc_pack(18);
  constexpr uint64_t w3 = xif_desc_pack(27), w4 = xif_desc_pack(36);
  const int q = idx / 9;
  const uint64_t w = q == 0 ? w0 : q == 1 ? w1 : q == 2 ? w2 : q == 3 ? w3 : w4;
  return (int)((w >> (7 * (idx - 9 * q))) & 127u);
}
GPISA_HD constexpr bool xif_fast_matches() {
  for (int i = 0; i < SFX_IF_FORMS; ++i)
    if (xif_form_desc_fast(i) != xif_form_desc(i)) return false;
  return true;
}
static_assert(xif_fast_matches(), "packed IF descriptors differ from the scan");
// xif_form_index without the scan: bit t of the 128-bit mask (lo, hi) is set
// for each valid descriptor t; the index is the number of set bits below t
GPISA_HD constexpr uint64_t xif_valid_mask(int first) {
  uint64_t m = 0;
  for (int j = 0; j < 64 && first + j < 125; ++j) {
    const int t = first + j;
    if (xif_desc_valid(t / 25, (t / 5) % 5, t % 5)) m |= (uint64_t)1 << j;
  }
  return m;
}
GPISA_HD constexpr int popcount64_c(uint64_t x) {  // (constant evaluation only)
  int c = 0;
  for (; x; x &= x - 1) ++c;
  return c;
}
GPISA_HD constexpr bool xif_masks_match() {
  for (int t = 0; t < 125; ++t) {
    const uint64_t lo = xif_valid_mask(0), hi = xif_valid_mask(64);
    const int idx = t < 64 ? popcount64_c(lo & (((uint64_t)1 << t) - 1))
                           : popcount64_c(lo) + popcount64_c(hi & (((uint64_t)1 << (t - 64)) - 1));
    if (xif_desc_valid(t / 25, (t / 5) % 5, t % 5) && idx != xif_form_index(t / 25, (t / 5) % 5, t % 5))
      return false;
  }
  return true;
}
static_assert(xif_masks_match(), "the valid-descriptor masks do not give the scan's index");
GPISA_HD constexpr int sfx_if_code(int iform, int level) { return SFX_IF_BASE + iform * R + level; }
constexpr int SFX_NCODES = SFX_IF_BASE + SFX_IF_FORMS * R;  // 1280

// ---- float RPN (Sec. 4): push a terminal to level l, or combine levels
// l and l+1 into level l.
enum RForm : int { RF_PUSHX = 0, RF_PUSHC, RF_OP, RF_OPR, RF_NFORMS };
GPISA_HD constexpr int rpn_code(int form, int level, int op) { return (form * R + level) * 4 + op; }
constexpr int RF_NCODES = RF_NFORMS * R * 4;

// ---- extended float RPN (the function sets of Sec. 4.2 in postfix form):
// the basic RPN codes first, then comparisons and logic (RF_OP: a = level l,
// b = level l+1; RF_OPR: a = l+1, b = l), the unary functions on level l,
// and IF(c, a, b) whose operands sit on levels l .. l+2 in one of the six
// orders (permutation index: the levels of c, a, b as a permutation of
// 0, 1, 2 in lexicographic order).  Every result goes to level l.
constexpr int RPX_BIN_BASE = RF_NCODES;  // 128
GPISA_HD constexpr int rpx_bin_code(int opr, int level, int op) {  // opr: 0 RF_OP, 1 RF_OPR
  return RPX_BIN_BASE + (opr * R + level) * XB_NOPS + op;
}
constexpr int RPX_UN_BASE = RPX_BIN_BASE + 2 * R * XB_NOPS;  // 208
GPISA_HD constexpr int rpx_un_code(int level, int fn) { return RPX_UN_BASE + level * XU_NOPS + fn; }
constexpr int RPX_IF_BASE = RPX_UN_BASE + R * XU_NOPS;  // 240
GPISA_HD constexpr int rpx_if_code(int perm, int level) { return RPX_IF_BASE + perm * R + level; }
// permutation index of (level of c, level of a, level of b), each 0..2, distinct
GPISA_HD constexpr int rpx_perm_index(int lc, int la, int lb) {
  return lc * 2 + ((la > lb) ? 1 : 0);  // lc picks the first element; the rest in order or swapped
}
constexpr int RPX_NCODES = RPX_IF_BASE + 6 * R;  // 288

// ---- register linear GP: code = (op, a, b); pa = destination register.
constexpr int NREG = 8;
GPISA_HD constexpr int lin_code(int op, int a, int b) { return (op * NREG + a) * NREG + b; }
constexpr int LIN_NCODES = 4 * NREG * NREG;

// ---- Boolean S-form.  Binary functions AND, OR, NAND, NOR (index 0..3).
enum BOp : int { B_AND = 0, B_OR = 1, B_NAND = 2, B_NOR = 3 };
enum BForm : int { BF_XX = 0, BF_XS, BF_SX, BF_SS, BF_SSR, BF_NFORMS };
GPISA_HD constexpr int bool_bin_code(int form, int level, int op) { return (form * R + level) * 4 + op; }
constexpr int BOOL_IF_BASE = BF_NFORMS * R * 4;  // 160
// IF(c, a, b): each operand is X (0) or stack level l+0, l+1, l+2 (1, 2, 3);
// the stack operands use exactly levels l .. l+m-1.  The 16 valid operand
// descriptors are numbered in increasing order of (dc*16 + da*4 + db).
GPISA_HD constexpr bool if_desc_valid(int dc, int da, int db) {
  int m = (dc > 0) + (da > 0) + (db > 0);
  bool used[3] = {false, false, false};
  if (dc > 0) { if (dc - 1 >= m || used[dc - 1]) return false; used[dc - 1] = true; }
  if (da > 0) { if (da - 1 >= m || used[da - 1]) return false; used[da - 1] = true; }
  if (db > 0) { if (db - 1 >= m || used[db - 1]) return false; used[db - 1] = true; }
  return true;
}
GPISA_HD constexpr int if_form_index(int dc, int da, int db) {
  int idx = 0;
  for (int t = 0; t < dc * 16 + da * 4 + db; ++t)
    if (if_desc_valid(t / 16, (t / 4) % 4, t % 4)) ++idx;
  return idx;
}
GPISA_HD constexpr int if_form_desc(int idx) {  // inverse: returns dc*16+da*4+db
  int seen = 0;
  for (int t = 0; t < 64; ++t)
    if (if_desc_valid(t / 16, (t / 4) % 4, t % 4)) { if (seen == idx) return t; ++seen; }
  return -1;
}
constexpr int BOOL_IF_FORMS = 16;
// if_form_desc without the scan: the 16 descriptors (6 bits each) packed
// eight to a 64-bit constant
GPISA_HD constexpr uint64_t if_desc_pack(int first) {
  uint64_t w = 0;
  for (int j = 0; j < 8; ++j) w |= (uint64_t)if_form_desc(first + j) << (6 * j);
  return w;
}
GPISA_HD constexpr int if_form_desc_fast(int idx) {  // idx in [0, BOOL_IF_FORMS)
  constexpr uint64_t lo = if_desc_pack(0), hi = if_desc_pack(8);
  return (int)(((idx < 8 ? lo : hi) >> (6 * (idx & 7))) & 63u);
}
GPISA_HD constexpr bool if_fast_matches() {
  for (int i = 0; i < BOOL_IF_FORMS; ++i)
    if (if_form_desc_fast(i) != if_form_desc(i)) return false;
  return true;
}
static_assert(if_fast_matches(), "packed IF descriptors differ from the scan");
GPISA_HD constexpr int bool_if_code(int iform, int level) { return BOOL_IF_BASE + iform * R + level; }
constexpr int BOOL_MOVX = BOOL_IF_BASE + BOOL_IF_FORMS * R;  // 288
constexpr int BOOL_NCODES = BOOL_MOVX + 1;

// header word 0
GPISA_HD constexpr uint32_t header0(uint32_t kind, uint32_t order) {
  return kind | (order << 8) | (VERSION << 16);
}

}  // namespace gpisa
