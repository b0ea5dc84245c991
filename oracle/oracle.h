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
  ORC_AND = 7, ORC_OR = 8, ORC_NAND = 9, ORC_NOR = 10, ORC_IF = 11
};

/* Single binary32 operation as the oracle defines it (pinned against numpy). */
float oracle_apply_op(int op, float a, float b);

/* Per-case outputs of one prefix tree by recursive descent (the definition). */
int oracle_tree_outputs(const uint32_t* prog, int64_t len, const float* cases,
                        int32_t n_inputs, int64_t n_cases, float* out);

/* Per-case outputs by an independent algorithm: scan the prefix tokens from
 * right to left with an explicit value stack. */
int oracle_tree_outputs_stack(const uint32_t* prog, int64_t len, const float* cases,
                              int32_t n_inputs, int64_t n_cases, float* out);

/* Number of nodes (functions + terminals) of a prefix tree; <0 on error. */
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

#ifdef __cplusplus
}
#endif
#endif
