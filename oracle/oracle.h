/*
 * oracle.h -- plain, slow, obviously correct CPU evaluator for GP populations.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the parity reference for the CUDA
 * path.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no source, header, table or helper with the
 * CUDA library (paper_1601_00221_gb300/csrc) and must never be called from it.
 *
 * What it computes (Chitty, "Faster GPU Based Genetic Programming Using A Two
 * Dimensional Stack"):
 *   - Sec. 3: a GP program is a tree; its value on one fitness case is the tree
 *     evaluated on that case's inputs.  GPop/s counts tree nodes x cases.
 *   - Sec. 4: the two-dimensional stack only changes the evaluation schedule
 *     (K cases per interpreter pass), never the value of any case, so the
 *     plain per-case definition below is the exact reference for every
 *     kernel variant.
 *   - Sec. 4.2: problem classes are symbolic regression over {+,-,*,/} and
 *     bit-packed Boolean problems over {AND,OR,NAND,NOR} (+IF), 32 cases per
 *     32-bit word (sub-machine-code GP).
 *
 * Readings where the paper is silent (each pinned by a test):
 *   - "/" is protected: a zero denominator (+0 or -0) returns 1.0f, otherwise
 *     IEEE-754 binary32 division rounded to nearest even.
 *   - every node is one binary32 operation rounded to nearest even; no fused
 *     multiply-add, no flush-to-zero (build with -ffp-contract=off, no
 *     fast-math).
 *   - SUB(a,b) = a - b and DIV(a,b) = a / b where a is the first child in
 *     prefix order.
 *   - regression fitness F = sum over cases of |o - y|, where the per-case
 *     error is computed in binary32 and the sum is taken in binary64; if any
 *     per-case error is not finite, F = +inf.
 *   - Boolean: IF(c,a,b) = (c AND a) OR (NOT c AND b); case index c maps to
 *     word c>>5, bit c&31; hits count cases where output == target.
 *   - register linear GP (not in the paper; instructions r[d] = r[a] op r[b]
 *     over 8 binary32 registers): r[i] starts as input i for i < n_inputs
 *     (else 0.0f); the program's output is r[0] after the last instruction.
 *
 * User token format of a prefix tree (uint32 words):
 *   bits 0..7 opcode, bits 8..31 operand (input index for VAR).
 *   A CONST token is followed by one word holding the binary32 bit pattern.
 *
 * All functions return 0 on success and a negative code on a malformed
 * program: -1 unknown opcode, -2 truncated (missing operands), -3 trailing
 * tokens after the root's subtree, -4 input index >= n_inputs, -5 bad argument.
 */
#ifndef GP_ORACLE_H
#define GP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_ADD = 1, ORC_SUB = 2, ORC_MUL = 3, ORC_DIV = 4,
  ORC_VAR = 5, ORC_CONST = 6,
  ORC_AND = 7, ORC_OR = 8, ORC_NAND = 9, ORC_NOR = 10, ORC_IF = 11,
  /* the rest of the float function sets of Sec. 4.2 (oracle_fset.c) */
  ORC_SIN = 12, ORC_COS = 13, ORC_EXP = 14, ORC_LOG = 15,
  ORC_GT = 16, ORC_LT = 17, ORC_EQ = 18
};

/* fitness measures */
enum { ORC_FIT_ABS = 0, ORC_FIT_MSE = 1, ORC_FIT_CLASS = 2 };

/* Single binary32 operation as the oracle defines it (pinned against numpy). */
float oracle_apply_op(int op, float a, float b);

/* Per-case outputs of one prefix tree by recursive descent (the definition). */
int oracle_tree_outputs(const uint32_t* prog, int64_t len, const float* cases,
                        int32_t n_inputs, int64_t n_cases, float* out);

/* Per-case outputs by an independent algorithm: scan the prefix tokens from
 * right to left with an explicit value stack. */
int oracle_tree_outputs_stack(const uint32_t* prog, int64_t len, const float* cases,
                              int32_t n_inputs, int64_t n_cases, float* out);

/* Number of nodes (functions + terminals) of a prefix tree, over every
 * function of oracle.h (Boolean and the full float sets); <0 on error. */
int64_t oracle_tree_nodes(const uint32_t* prog, int64_t len);

/* Sum |o-y| in binary64 over the per-case binary32 errors (+inf if any is
 * not finite). */
int oracle_tree_fitness(const uint32_t* prog, int64_t len, const float* cases,
                        int32_t n_inputs, int64_t n_cases, const float* targets,
                        double* fitness);

/* Population of trees: program p occupies programs[offsets[p] .. +lengths[p]).
 * Evaluates programs [p_begin, p_end). Returns the first error code met. */
int oracle_population_fitness(const uint32_t* programs, const int64_t* offsets,
                              const int32_t* lengths, int32_t p_begin, int32_t p_end,
                              const float* cases, int32_t n_inputs, int64_t n_cases,
                              const float* targets, double* fitness_out);

/* Boolean tree on bit-packed cases: case_bits[v*n_words + w]. */
int oracle_bool_outputs(const uint32_t* prog, int64_t len, const uint32_t* case_bits,
                        int32_t n_inputs, int64_t n_words, uint32_t* out_words);

/* Hits = number of cases c < n_cases with output bit == target bit. */
int oracle_bool_hits(const uint32_t* prog, int64_t len, const uint32_t* case_bits,
                     int32_t n_inputs, int64_t n_cases, const uint32_t* target_bits,
                     uint64_t* hits);

int oracle_bool_population_hits(const uint32_t* programs, const int64_t* offsets,
                                const int32_t* lengths, int32_t p_begin, int32_t p_end,
                                const uint32_t* case_bits, int32_t n_inputs,
                                int64_t n_cases, const uint32_t* target_bits,
                                uint64_t* hits_out);

/* Register linear GP: instruction i is (dst[i], op[i], a[i], b[i]);
 * registers 0..7; op in {ADD,SUB,MUL,DIV}. */
int oracle_linear_outputs(const uint8_t* dst, const uint8_t* op, const uint8_t* a,
                          const uint8_t* b, int32_t n_instr, const float* cases,
                          int32_t n_inputs, int64_t n_cases, float* out);

/* Population of register programs: instr[(offsets[p] + i)*4 + {0,1,2,3}] =
 * {dst, op, a, b} for i < lengths[p]. */
int oracle_linear_population_fitness(const uint8_t* instr, const int64_t* offsets,
                                     const int32_t* lengths, int32_t p_begin,
                                     int32_t p_end, const float* cases,
                                     int32_t n_inputs, int64_t n_cases,
                                     const float* targets, double* fitness_out);

/* ------------------------------------------------------------------------
 * Full float function sets (oracle_fset.c).  Sec. 4.2 names the sets of the
 * float problems -- sextic regression {+,-,*,/,Sin,Cos,Log,Exp}; Shuttle
 * {+,-,*,/,>,<,==,AND,OR,IF}; KDDcup both together -- and defines none of
 * them beyond the name.  Readings (each pinned by a test):
 *   SIN, COS, EXP  binary32 sine, cosine (radians) and e^a.
 *   LOG(a)         0 if a == 0 (either sign), else the natural log of |a|.
 *   GT, LT, EQ     1.0f if a > b (a < b, a == b) else 0.0f; IEEE comparisons,
 *                  so a NaN operand gives 0.0f and -0 == +0.
 *   AND, OR        1.0f if a != 0 and (or) b != 0, else 0.0f; a NaN counts as
 *                  non-zero (it is != 0).
 *   IF(c, a, b)    a if c != 0 else b (a NaN condition selects a).
 * Fitness measures (the paper's parameter table: mean squared error for
 * regression, the number of incorrect classifications for classification):
 *   ORC_FIT_ABS    sum of |o - y| (binary32 error, binary64 sum).
 *   ORC_FIT_MSE    (sum of d*d, d = o - y, both binary32; binary64 sum) / n.
 *   ORC_FIT_CLASS  number of cases whose output, rounded to the nearest
 *                  integer (ties to even), differs from the target label.
 * A non-finite binary32 error (ABS, MSE) makes the fitness +inf; n = 0
 * gives 0.
 *
 * There is no single correct binary32 sine: implementations differ by an
 * ulp or two.  The point evaluator takes the binary32 value nearest the
 * binary64 libm result.  The enclosure evaluator instead bounds EVERY
 * implementation that rounds +,-,*,/ correctly, takes the comparisons, logic
 * and IF exactly, and returns sin, cos and exp within 2 ulp and log within
 * 1 ulp of the correctly rounded value (the documented maximum errors of
 * CUDA's sinf, cosf, expf and logf): the output of any such implementation
 * lies in [lo, hi], or is NaN where may_nan is set.  Without a transcendental
 * node, lo == hi is the exact output (up to the sign of zero).
 * ------------------------------------------------------------------------ */

/* Arity of a float function of the full sets (0 for a terminal, -1 unknown). */
int oracle_fset_arity(int op);

/* Per-case outputs of a tree over the full function sets (point evaluation). */
int oracle_fset_outputs(const uint32_t* prog, int64_t len, const float* cases,
                        int32_t n_inputs, int64_t n_cases, float* out);

/* Per-case enclosures: lo[c] <= output <= hi[c], or NaN if may_nan[c]. */
int oracle_fset_enclosure(const uint32_t* prog, int64_t len, const float* cases,
                          int32_t n_inputs, int64_t n_cases, float* lo, float* hi,
                          uint8_t* may_nan);

/* Fitness of per-case outputs under a measure. */
int oracle_fitness_of_outputs(const float* out, const float* targets, int64_t n_cases,
                              int32_t kind, double* fitness);

/* Fitness bounds from per-case enclosures: every output inside its enclosure
 * gives a fitness in [f_lo, f_hi] (before the binary64 sum's rounding), or
 * +inf where *may_inf; *must_inf when every choice gives +inf. */
int oracle_fitness_enclosure(const float* lo, const float* hi, const uint8_t* may_nan,
                             const float* targets, int64_t n_cases, int32_t kind,
                             double* f_lo, double* f_hi, int32_t* may_inf,
                             int32_t* must_inf);

/* Population over the full function sets, point evaluation, any measure. */
int oracle_fset_population_fitness(const uint32_t* programs, const int64_t* offsets,
                                   const int32_t* lengths, int32_t p_begin, int32_t p_end,
                                   const float* cases, int32_t n_inputs, int64_t n_cases,
                                   const float* targets, int32_t kind, double* fitness_out);

#ifdef __cplusplus
}
#endif
#endif
