/*
 * oracle.c -- plain CPU reference for GP fitness evaluation.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h): loaded by the tests, the smoke check
 * and the benchmark's CPU-baseline leg; never by the CUDA library.
 *
 * Every function evaluates one fitness case at a time, one node at a time, in
 * the order the tree defines (Sec. 3 and Sec. 4 of the paper: the value of a
 * program on a case does not depend on how many cases an interpreter pass
 * covers).  Build flags: -O2 -ffp-contract=off, no fast-math, so that each
 * node is exactly one binary32 operation rounded to nearest even.
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the oracle needs binary32 arithmetic evaluated in binary32 (FLT_EVAL_METHOD 0)"
#endif

/* ------------------------------------------------------------------------ */
/* One node's arithmetic (Sec. 4.2 function set {+,-,*,/}; "/" protected).   */
/* ------------------------------------------------------------------------ */
float oracle_apply_op(int op, float a, float b) {
  volatile float r; /* volatile: force a binary32 store of every result */
  switch (op) {
    case ORC_ADD: r = a + b; break;
    case ORC_SUB: r = a - b; break;
    case ORC_MUL: r = a * b; break;
    case ORC_DIV: r = (b == 0.0f) ? 1.0f : a / b; break;
    default: r = NAN; break;
  }
  return r;
}

static uint32_t bool_apply(int op, uint32_t a, uint32_t b, uint32_t c) {
  switch (op) {
    case ORC_AND: return a & b;
    case ORC_OR: return a | b;
    case ORC_NAND: return ~(a & b);
    case ORC_NOR: return ~(a | b);
    case ORC_IF: return (a & b) | (~a & c); /* IF(cond=a, then=b, else=c) */
    default: return 0u;
  }
}

static int is_float_fn(int op) { return op >= ORC_ADD && op <= ORC_DIV; }
static int is_bool_fn(int op) { return op >= ORC_AND && op <= ORC_IF; }
static int bool_arity(int op) { return op == ORC_IF ? 3 : 2; }

/* ------------------------------------------------------------------------ */
/* Recursive prefix evaluation of one case (the definition of a tree value).  */
/* ------------------------------------------------------------------------ */
typedef struct {
  const uint32_t* prog;
  int64_t len;
  const float* cases;
  int32_t n_inputs;
  int64_t n_cases;
  int64_t c; /* case index */
  int err;
} fctx;

static float frec(fctx* k, int64_t* pos) {
  if (*pos >= k->len) { k->err = -2; return 0.0f; }
  uint32_t t = k->prog[*pos];
  int op = (int)(t & 0xffu);
  uint32_t arg = t >> 8;
  *pos += 1;
  if (op == ORC_VAR) {
    if ((int64_t)arg >= k->n_inputs) { k->err = -4; return 0.0f; }
    if (!k->cases) return 0.0f; /* no cases: validation only */
    return k->cases[(int64_t)arg * k->n_cases + k->c];
  }
  if (op == ORC_CONST) {
    if (*pos >= k->len) { k->err = -2; return 0.0f; }
    float v;
    uint32_t bits = k->prog[*pos];
    memcpy(&v, &bits, sizeof v);
    *pos += 1;
    return v;
  }
  if (!is_float_fn(op)) { k->err = -1; return 0.0f; }
  float a = frec(k, pos); /* first child */
  if (k->err) return 0.0f;
  float b = frec(k, pos); /* second child */
  if (k->err) return 0.0f;
  return oracle_apply_op(op, a, b);
}

int oracle_tree_outputs(const uint32_t* prog, int64_t len, const float* cases,
                        int32_t n_inputs, int64_t n_cases, float* out) {
  if (!prog || len <= 0 || n_cases < 0 || (n_cases > 0 && !out)) return -5;
  for (int64_t c = 0; c < n_cases; ++c) {
    fctx k = {prog, len, cases, n_inputs, n_cases, c, 0};
    int64_t pos = 0;
    float v = frec(&k, &pos);
    if (k.err) return k.err;
    if (pos != len) return -3;
    out[c] = v;
  }
  if (n_cases == 0) { /* still validate the program */
    fctx k = {prog, len, NULL, n_inputs, 0, 0, 0};
    int64_t pos = 0;
    (void)frec(&k, &pos);
    if (k.err) return k.err;
    if (pos != len) return -3;
  }
  return 0;
}

int64_t oracle_tree_nodes(const uint32_t* prog, int64_t len) {
  /* Count nodes and check that the tokens form exactly one tree: track how
   * many subtrees are still owed while reading left to right. */
  int64_t owed = 1, nodes = 0, i = 0;
  while (i < len) {
    if (owed == 0) return -3;
    int op = (int)(prog[i] & 0xffu);
    owed -= 1;
    nodes += 1;
    if (op == ORC_CONST) { if (i + 1 >= len) return -2; i += 2; continue; }
    if (op == ORC_VAR) { i += 1; continue; }
    if (is_float_fn(op)) owed += 2;
    else if (is_bool_fn(op)) owed += bool_arity(op);
    else if (oracle_fset_arity(op) > 0) owed += oracle_fset_arity(op); /* SIN .. EQ */
    else return -1;
    i += 1;
  }
  if (owed != 0) return -2;
  return nodes;
}

/* ------------------------------------------------------------------------ */
/* Independent evaluator: right-to-left scan of the prefix string with an     */
/* explicit stack.  Reading prefix backwards, both operands of a function are */
/* already on the stack, the first child on top.                              */
/* ------------------------------------------------------------------------ */
int oracle_tree_outputs_stack(const uint32_t* prog, int64_t len, const float* cases,
                              int32_t n_inputs, int64_t n_cases, float* out) {
  if (!prog || len <= 0 || n_cases < 0) return -5;
  /* token start positions: a CONST's payload word is not a token */
  int64_t* starts = (int64_t*)malloc(sizeof(int64_t) * (size_t)len);
  float* stack = (float*)malloc(sizeof(float) * (size_t)len);
  if (!starts || !stack) { free(starts); free(stack); return -5; }
  int64_t nt = 0;
  for (int64_t i = 0; i < len;) {
    int op = (int)(prog[i] & 0xffu);
    starts[nt++] = i;
    if (op == ORC_CONST) { if (i + 1 >= len) { free(starts); free(stack); return -2; } i += 2; }
    else i += 1;
  }
  int rc = 0;
  for (int64_t c = 0; c < n_cases && rc == 0; ++c) {
    int64_t sp = 0;
    for (int64_t j = nt - 1; j >= 0; --j) {
      uint32_t t = prog[starts[j]];
      int op = (int)(t & 0xffu);
      uint32_t arg = t >> 8;
      if (op == ORC_VAR) {
        if ((int64_t)arg >= n_inputs) { rc = -4; break; }
        stack[sp++] = cases[(int64_t)arg * n_cases + c];
      } else if (op == ORC_CONST) {
        float v;
        uint32_t bits = prog[starts[j] + 1];
        memcpy(&v, &bits, sizeof v);
        stack[sp++] = v;
      } else if (is_float_fn(op)) {
        if (sp < 2) { rc = -2; break; }
        float a = stack[sp - 1]; /* first child: pushed last */
        float b = stack[sp - 2];
        sp -= 2;
        stack[sp++] = oracle_apply_op(op, a, b);
      } else {
        rc = -1;
        break;
      }
    }
    if (rc == 0 && sp != 1) rc = (sp == 0) ? -2 : -3;
    if (rc == 0) out[c] = stack[0];
  }
  free(starts);
  free(stack);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Regression fitness: sum |o - y| (binary32 error, binary64 sum).            */
/* ------------------------------------------------------------------------ */
static double abs_error_sum(const float* out, const float* targets, int64_t n_cases) {
  double s = 0.0;
  int nonfinite = 0;
  for (int64_t c = 0; c < n_cases; ++c) {
    volatile float d = out[c] - targets[c];
    float e = fabsf(d);
    if (!isfinite(e)) nonfinite = 1;
    else s += (double)e;
  }
  return nonfinite ? INFINITY : s;
}

int oracle_tree_fitness(const uint32_t* prog, int64_t len, const float* cases,
                        int32_t n_inputs, int64_t n_cases, const float* targets,
                        double* fitness) {
  if (!fitness) return -5;
  float* out = (float*)malloc(sizeof(float) * (size_t)(n_cases > 0 ? n_cases : 1));
  if (!out) return -5;
  int rc = oracle_tree_outputs(prog, len, cases, n_inputs, n_cases, out);
  if (rc == 0) *fitness = abs_error_sum(out, targets, n_cases);
  free(out);
  return rc;
}

int oracle_population_fitness(const uint32_t* programs, const int64_t* offsets,
                              const int32_t* lengths, int32_t p_begin, int32_t p_end,
                              const float* cases, int32_t n_inputs, int64_t n_cases,
                              const float* targets, double* fitness_out) {
  int first = 0;
  for (int32_t p = p_begin; p < p_end; ++p) {
    int rc = oracle_tree_fitness(programs + offsets[p], lengths[p], cases, n_inputs,
                                 n_cases, targets, &fitness_out[p]);
    if (rc != 0) {
      fitness_out[p] = NAN;
      if (!first) first = rc;
    }
  }
  return first;
}

/* ------------------------------------------------------------------------ */
/* Boolean programs on bit-packed cases (Sec. 4.2, 32 cases per word).        */
/* ------------------------------------------------------------------------ */
typedef struct {
  const uint32_t* prog;
  int64_t len;
  const uint32_t* bits;
  int32_t n_inputs;
  int64_t n_words;
  int64_t w;
  int err;
} bctx;

static uint32_t brec(bctx* k, int64_t* pos) {
  if (*pos >= k->len) { k->err = -2; return 0u; }
  uint32_t t = k->prog[*pos];
  int op = (int)(t & 0xffu);
  uint32_t arg = t >> 8;
  *pos += 1;
  if (op == ORC_VAR) {
    if ((int64_t)arg >= k->n_inputs) { k->err = -4; return 0u; }
    return k->bits[(int64_t)arg * k->n_words + k->w];
  }
  if (!is_bool_fn(op)) { k->err = -1; return 0u; }
  uint32_t a = brec(k, pos);
  if (k->err) return 0u;
  uint32_t b = brec(k, pos);
  if (k->err) return 0u;
  uint32_t c = 0u;
  if (op == ORC_IF) {
    c = brec(k, pos);
    if (k->err) return 0u;
  }
  return bool_apply(op, a, b, c);
}

int oracle_bool_outputs(const uint32_t* prog, int64_t len, const uint32_t* case_bits,
                        int32_t n_inputs, int64_t n_words, uint32_t* out_words) {
  if (!prog || len <= 0 || n_words < 0) return -5;
  for (int64_t w = 0; w < n_words; ++w) {
    bctx k = {prog, len, case_bits, n_inputs, n_words, w, 0};
    int64_t pos = 0;
    uint32_t v = brec(&k, &pos);
    if (k.err) return k.err;
    if (pos != len) return -3;
    out_words[w] = v;
  }
  return 0;
}

int oracle_bool_hits(const uint32_t* prog, int64_t len, const uint32_t* case_bits,
                     int32_t n_inputs, int64_t n_cases, const uint32_t* target_bits,
                     uint64_t* hits) {
  if (!hits || n_cases < 0) return -5;
  int64_t n_words = (n_cases + 31) / 32;
  uint32_t* out = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n_words > 0 ? n_words : 1));
  if (!out) return -5;
  int rc = oracle_bool_outputs(prog, len, case_bits, n_inputs, n_words, out);
  if (rc == 0) {
    uint64_t h = 0;
    /* case by case, straight from the definition of a hit */
    for (int64_t c = 0; c < n_cases; ++c) {
      uint32_t o = (out[c >> 5] >> (c & 31)) & 1u;
      uint32_t t = (target_bits[c >> 5] >> (c & 31)) & 1u;
      h += (o == t) ? 1u : 0u;
    }
    *hits = h;
  }
  free(out);
  return rc;
}

int oracle_bool_population_hits(const uint32_t* programs, const int64_t* offsets,
                                const int32_t* lengths, int32_t p_begin, int32_t p_end,
                                const uint32_t* case_bits, int32_t n_inputs,
                                int64_t n_cases, const uint32_t* target_bits,
                                uint64_t* hits_out) {
  int first = 0;
  for (int32_t p = p_begin; p < p_end; ++p) {
    int rc = oracle_bool_hits(programs + offsets[p], lengths[p], case_bits, n_inputs,
                              n_cases, target_bits, &hits_out[p]);
    if (rc != 0) {
      hits_out[p] = UINT64_MAX;
      if (!first) first = rc;
    }
  }
  return first;
}

/* ------------------------------------------------------------------------ */
/* Register linear GP: r[d] = r[a] op r[b] over 8 binary32 registers.         */
/* ------------------------------------------------------------------------ */
#define ORC_NREG 8

int oracle_linear_outputs(const uint8_t* dst, const uint8_t* op, const uint8_t* a,
                          const uint8_t* b, int32_t n_instr, const float* cases,
                          int32_t n_inputs, int64_t n_cases, float* out) {
  if (n_instr < 0 || n_cases < 0) return -5;
  for (int32_t i = 0; i < n_instr; ++i) {
    if (dst[i] >= ORC_NREG || a[i] >= ORC_NREG || b[i] >= ORC_NREG) return -4;
    if (!is_float_fn(op[i])) return -1;
  }
  for (int64_t c = 0; c < n_cases; ++c) {
    float r[ORC_NREG];
    for (int i = 0; i < ORC_NREG; ++i)
      r[i] = (i < n_inputs) ? cases[(int64_t)i * n_cases + c] : 0.0f;
    for (int32_t i = 0; i < n_instr; ++i)
      r[dst[i]] = oracle_apply_op(op[i], r[a[i]], r[b[i]]);
    out[c] = r[0];
  }
  return 0;
}

int oracle_linear_population_fitness(const uint8_t* instr, const int64_t* offsets,
                                     const int32_t* lengths, int32_t p_begin,
                                     int32_t p_end, const float* cases,
                                     int32_t n_inputs, int64_t n_cases,
                                     const float* targets, double* fitness_out) {
  int first = 0;
  float* out = (float*)malloc(sizeof(float) * (size_t)(n_cases > 0 ? n_cases : 1));
  int32_t maxlen = 0;
  for (int32_t p = p_begin; p < p_end; ++p) if (lengths[p] > maxlen) maxlen = lengths[p];
  uint8_t* cols = (uint8_t*)malloc((size_t)4 * (size_t)(maxlen > 0 ? maxlen : 1));
  if (!out || !cols) { free(out); free(cols); return -5; }
  for (int32_t p = p_begin; p < p_end; ++p) {
    const uint8_t* ins = instr + offsets[p] * 4;
    int32_t n = lengths[p];
    uint8_t *d = cols, *o = cols + maxlen, *aa = cols + 2 * maxlen, *bb = cols + 3 * maxlen;
    for (int32_t i = 0; i < n; ++i) {
      d[i] = ins[4 * i + 0];
      o[i] = ins[4 * i + 1];
      aa[i] = ins[4 * i + 2];
      bb[i] = ins[4 * i + 3];
    }
    int rc = oracle_linear_outputs(d, o, aa, bb, n, cases, n_inputs, n_cases, out);
    if (rc != 0) {
      fitness_out[p] = NAN;
      if (!first) first = rc;
    } else {
      fitness_out[p] = abs_error_sum(out, targets, n_cases);
    }
  }
  free(out);
  free(cols);
  return first;
}
