/*
 * oracle_fset.c -- the full float function sets of the paper's problems, the
 * fitness measures, and per-case output enclosures.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h): loaded by the tests, the smoke
 * check and the benchmark's CPU-baseline leg; never by the CUDA library.
 *
 * Sec. 4.2 gives the function sets of the float problems (sextic regression:
 * +, -, *, /, Sin, Cos, Log, Exp; Shuttle: +, -, *, /, >, <, ==, AND, OR, IF;
 * KDDcup: all of them) and the parameter table gives the fitness measures
 * (mean squared error for regression, the number of incorrect
 * classifications for classification).  The meaning of each function is
 * this library's reading, stated in oracle.h.  Everything here evaluates one
 * case at a time, one node at a time, by recursive descent over the prefix
 * tokens, exactly as oracle.c does for {+, -, *, /}.
 *
 * Enclosures.  A binary32 sine is not unique: implementations differ in the
 * last bit or two.  So for trees that use SIN, COS, EXP or LOG the parity
 * check cannot be bit-exact; instead every node is evaluated as an interval
 * that holds the value of every admissible implementation (see oracle.h) --
 * interval arithmetic in which each correctly rounded operation is applied
 * to the interval's end points (it is monotone in each operand), each
 * transcendental function's exact range over the operand interval is taken
 * in binary64 and widened by its ulp bound plus one ulp for the binary64
 * evaluation, and NaN is tracked as a separate possibility.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the oracle needs binary32 arithmetic evaluated in binary32 (FLT_EVAL_METHOD 0)"
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* documented maximum errors (ulp) of the binary32 functions being bounded */
#define ULP_SIN 2
#define ULP_COS 2
#define ULP_EXP 2
#define ULP_LOG 1

int oracle_fset_arity(int op) {
  switch (op) {
    case ORC_VAR: case ORC_CONST: return 0;
    case ORC_SIN: case ORC_COS: case ORC_EXP: case ORC_LOG: return 1;
    case ORC_ADD: case ORC_SUB: case ORC_MUL: case ORC_DIV:
    case ORC_GT: case ORC_LT: case ORC_EQ: case ORC_AND: case ORC_OR: return 2;
    case ORC_IF: return 3;
    default: return -1;
  }
}

/* ------------------------------------------------------------------------ */
/* Point evaluation                                                          */
/* ------------------------------------------------------------------------ */
static float unary_point(int op, float a) {
  volatile float r;
  switch (op) {
    case ORC_SIN: r = (float)sin((double)a); break;
    case ORC_COS: r = (float)cos((double)a); break;
    case ORC_EXP: r = (float)exp((double)a); break;
    case ORC_LOG: r = (a == 0.0f) ? 0.0f : (float)log(fabs((double)a)); break;
    default: r = NAN; break;
  }
  return r;
}

static float binary_point(int op, float a, float b) {
  switch (op) {
    case ORC_GT: return a > b ? 1.0f : 0.0f;
    case ORC_LT: return a < b ? 1.0f : 0.0f;
    case ORC_EQ: return a == b ? 1.0f : 0.0f;
    case ORC_AND: return (a != 0.0f && b != 0.0f) ? 1.0f : 0.0f;
    case ORC_OR: return (a != 0.0f || b != 0.0f) ? 1.0f : 0.0f;
    default: return oracle_apply_op(op, a, b); /* +, -, *, protected / */
  }
}

typedef struct {
  const uint32_t* prog;
  int64_t len;
  const float* cases;
  int32_t n_inputs;
  int64_t n_cases;
  int64_t c;
  int err;
} pctx;

/* reads one terminal's value, or sets err */
static int terminal(pctx* k, int op, uint32_t arg, int64_t* pos, float* v) {
  if (op == ORC_VAR) {
    if ((int64_t)arg >= k->n_inputs) { k->err = -4; return 0; }
    *v = k->cases ? k->cases[(int64_t)arg * k->n_cases + k->c] : 0.0f; /* no cases: validation only */
    return 1;
  }
  if (*pos >= k->len) { k->err = -2; return 0; }
  uint32_t bits = k->prog[*pos];
  memcpy(v, &bits, sizeof *v);
  *pos += 1;
  return 1;
}

static float prec(pctx* k, int64_t* pos) {
  if (*pos >= k->len) { k->err = -2; return 0.0f; }
  uint32_t t = k->prog[*pos];
  int op = (int)(t & 0xffu);
  *pos += 1;
  int ar = oracle_fset_arity(op);
  if (ar < 0 || op == ORC_NAND || op == ORC_NOR) { k->err = -1; return 0.0f; }
  if (ar == 0) {
    float v = 0.0f;
    terminal(k, op, t >> 8, pos, &v);
    return v;
  }
  float a[3] = {0.0f, 0.0f, 0.0f};
  for (int i = 0; i < ar; ++i) { /* children in prefix order */
    a[i] = prec(k, pos);
    if (k->err) return 0.0f;
  }
  if (ar == 1) return unary_point(op, a[0]);
  if (ar == 3) return (a[0] != 0.0f) ? a[1] : a[2]; /* IF(c, a, b) */
  return binary_point(op, a[0], a[1]);
}

int oracle_fset_outputs(const uint32_t* prog, int64_t len, const float* cases,
                        int32_t n_inputs, int64_t n_cases, float* out) {
  if (!prog || len <= 0 || n_cases < 0 || (n_cases > 0 && !out)) return -5;
  for (int64_t c = 0; c < (n_cases > 0 ? n_cases : 1); ++c) {
    /* with no cases the program is still parsed and validated */
    pctx k = {prog, len, n_cases > 0 ? cases : NULL, n_inputs, n_cases, c, 0};
    int64_t pos = 0;
    float v = prec(&k, &pos);
    if (k.err) return k.err;
    if (pos != len) return -3;
    if (n_cases > 0) out[c] = v;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Enclosures                                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
  float lo, hi; /* real values [lo, hi]; empty when lo > hi */
  int nan;      /* NaN possible */
} ival;

static ival iv_empty(void) { ival r = {INFINITY, -INFINITY, 0}; return r; }
static int iv_is_empty(ival a) { return a.lo > a.hi; }

static void iv_add_value(ival* r, float v) {
  if (isnan(v)) { r->nan = 1; return; }
  if (v < r->lo) r->lo = v;
  if (v > r->hi) r->hi = v;
}

static ival iv_point(float v) {
  ival r = iv_empty();
  iv_add_value(&r, v);
  return r;
}

static ival iv_hull(ival a, ival b) {
  ival r = a;
  if (!iv_is_empty(b)) { iv_add_value(&r, b.lo); iv_add_value(&r, b.hi); }
  r.nan = a.nan || b.nan;
  return r;
}

static int iv_has_zero(ival a) { return !iv_is_empty(a) && a.lo <= 0.0f && a.hi >= 0.0f; }
static int iv_has_inf(ival a) { return !iv_is_empty(a) && (isinf(a.lo) || isinf(a.hi)); }

/* f(a, b) for every corner of the operand box: the exact range of an
 * operation that is monotone in each operand on the box (correct rounding
 * keeps monotonicity). */
static ival iv_corners(int op, ival a, ival b) {
  ival r = iv_empty();
  r.nan = a.nan || b.nan;
  if (iv_is_empty(a) || iv_is_empty(b)) return r;
  const float as[2] = {a.lo, a.hi}, bs[2] = {b.lo, b.hi};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) iv_add_value(&r, oracle_apply_op(op, as[i], bs[j]));
  return r;
}

/* a * b: bilinear, so the corners bound it; 0 * inf (NaN) can come from an
 * interior zero, so it is checked separately. */
static ival iv_mul(ival a, ival b) {
  ival r = iv_corners(ORC_MUL, a, b);
  if ((iv_has_zero(a) && iv_has_inf(b)) || (iv_has_zero(b) && iv_has_inf(a))) r.nan = 1;
  return r;
}

/* protected a / b: 1 where b is zero, whatever a is (even NaN); elsewhere
 * a / b is monotone in each operand while b keeps one sign, so each sign of
 * b is bounded by corners. */
static ival iv_div(ival a, ival b) {
  ival r = iv_empty();
  const int b_nonzero = !iv_is_empty(b) && !(b.lo == 0.0f && b.hi == 0.0f);
  r.nan = b.nan || (a.nan && b_nonzero);
  if (iv_has_zero(b)) iv_add_value(&r, 1.0f);
  if (iv_is_empty(a) || !b_nonzero) return r;
  if (b.lo < 0.0f) {
    ival bn = {b.lo, fminf(b.hi, -FLT_TRUE_MIN), 0};
    r = iv_hull(r, iv_corners(ORC_DIV, a, bn));
  }
  if (b.hi > 0.0f) {
    ival bp = {fmaxf(b.lo, FLT_TRUE_MIN), b.hi, 0};
    r = iv_hull(r, iv_corners(ORC_DIV, a, bp));
  }
  return r;
}

/* {0, 1} outcome sets of the comparisons and logic */
static ival iv_bool(int can_false, int can_true) {
  ival r = iv_empty();
  if (can_false) iv_add_value(&r, 0.0f);
  if (can_true) iv_add_value(&r, 1.0f);
  return r;
}

static int can_be_nonzero(ival a) { return a.nan || (!iv_is_empty(a) && !(a.lo == 0.0f && a.hi == 0.0f)); }

static ival iv_compare(int op, ival a, ival b) {
  int can_true = 0, can_false = a.nan || b.nan; /* NaN compares false */
  if (!iv_is_empty(a) && !iv_is_empty(b)) {
    switch (op) {
      case ORC_GT: can_true = a.hi > b.lo; can_false |= a.lo <= b.hi; break;
      case ORC_LT: can_true = a.lo < b.hi; can_false |= a.hi >= b.lo; break;
      default: /* EQ */
        can_true = a.lo <= b.hi && b.lo <= a.hi;
        can_false |= !(a.lo == a.hi && b.lo == b.hi && a.lo == b.lo);
        break;
    }
  }
  return iv_bool(can_false, can_true);
}

static ival iv_logic(int op, ival a, ival b) {
  const int ta = can_be_nonzero(a), tb = can_be_nonzero(b);
  const int fa = iv_has_zero(a), fb = iv_has_zero(b);
  if (op == ORC_AND) return iv_bool(fa || fb, ta && tb);
  return iv_bool(fa && fb, ta || tb); /* OR */
}

/* [dlo, dhi] (binary64, exact range) rounded to binary32 and widened by
 * `steps` binary32 spacings on each side */
static ival iv_widen(double dlo, double dhi, int steps) {
  ival r = iv_empty();
  float lo = (float)dlo, hi = (float)dhi;
  for (int i = 0; i < steps; ++i) {
    lo = nextafterf(lo, -INFINITY);
    hi = nextafterf(hi, INFINITY);
  }
  iv_add_value(&r, lo);
  iv_add_value(&r, hi);
  return r;
}

/* is some phase + 2*pi*k inside [lo, hi]?  (with a slack, so that binary64
 * rounding can only answer yes wrongly, which widens the enclosure) */
static int has_phase(double lo, double hi, double phase) {
  const double two_pi = 2.0 * M_PI, slack = 1e-9 * (1.0 + fabs(lo) + fabs(hi));
  double k = ceil((lo - slack - phase) / two_pi);
  return phase + two_pi * k <= hi + slack;
}

static ival iv_trig(ival a, int cosine) {
  ival r = iv_empty();
  r.nan = a.nan;
  if (iv_is_empty(a)) return r;
  if (iv_has_inf(a)) r.nan = 1; /* sin(+-inf), cos(+-inf) */
  double lo = a.lo, hi = a.hi;
  if (isinf(lo) && isinf(hi) && lo == hi) return r; /* only an infinity */
  if (isinf(lo)) lo = -FLT_MAX;
  if (isinf(hi)) hi = FLT_MAX;
  double mn, mx;
  if (hi - lo >= 2.0 * M_PI || fmax(fabs(lo), fabs(hi)) > 1.0e6) {
    mn = -1.0;
    mx = 1.0;
  } else {
    const double flo = cosine ? cos(lo) : sin(lo), fhi = cosine ? cos(hi) : sin(hi);
    mn = fmin(flo, fhi);
    mx = fmax(flo, fhi);
    if (has_phase(lo, hi, cosine ? 0.0 : M_PI / 2)) mx = 1.0;   /* a maximum inside */
    if (has_phase(lo, hi, cosine ? M_PI : -M_PI / 2)) mn = -1.0; /* a minimum inside */
  }
  return iv_hull(r, iv_widen(mn, mx, (cosine ? ULP_COS : ULP_SIN) + 1));
}

static ival iv_exp(ival a) {
  ival r = iv_empty();
  r.nan = a.nan;
  if (iv_is_empty(a)) return r;
  return iv_hull(r, iv_widen(exp((double)a.lo), exp((double)a.hi), ULP_EXP + 1));
}

static ival iv_log(ival a) {
  ival r = iv_empty();
  r.nan = a.nan;
  if (iv_is_empty(a)) return r;
  if (iv_has_zero(a)) iv_add_value(&r, 0.0f); /* the protected zero */
  double mlo, mhi; /* magnitudes of the non-zero part */
  if (a.lo > 0.0f) { mlo = a.lo; mhi = a.hi; }
  else if (a.hi < 0.0f) { mlo = -(double)a.hi; mhi = -(double)a.lo; }
  else {
    if (a.lo == 0.0f && a.hi == 0.0f) return r;
    mlo = FLT_TRUE_MIN;
    mhi = fmax(-(double)a.lo, (double)a.hi);
  }
  return iv_hull(r, iv_widen(log(mlo), log(mhi), ULP_LOG + 1));
}

static ival irec(pctx* k, int64_t* pos) {
  if (*pos >= k->len) { k->err = -2; return iv_empty(); }
  uint32_t t = k->prog[*pos];
  int op = (int)(t & 0xffu);
  *pos += 1;
  int ar = oracle_fset_arity(op);
  if (ar < 0 || op == ORC_NAND || op == ORC_NOR) { k->err = -1; return iv_empty(); }
  if (ar == 0) {
    float v = 0.0f;
    terminal(k, op, t >> 8, pos, &v);
    return iv_point(v);
  }
  ival a[3];
  for (int i = 0; i < ar; ++i) {
    a[i] = irec(k, pos);
    if (k->err) return iv_empty();
  }
  switch (op) {
    case ORC_ADD: case ORC_SUB: return iv_corners(op, a[0], a[1]);
    case ORC_MUL: return iv_mul(a[0], a[1]);
    case ORC_DIV: return iv_div(a[0], a[1]);
    case ORC_GT: case ORC_LT: case ORC_EQ: return iv_compare(op, a[0], a[1]);
    case ORC_AND: case ORC_OR: return iv_logic(op, a[0], a[1]);
    case ORC_SIN: return iv_trig(a[0], 0);
    case ORC_COS: return iv_trig(a[0], 1);
    case ORC_EXP: return iv_exp(a[0]);
    case ORC_LOG: return iv_log(a[0]);
    default: { /* IF(c, a, b) */
      ival r = iv_empty();
      if (can_be_nonzero(a[0])) r = iv_hull(r, a[1]);
      if (iv_has_zero(a[0])) r = iv_hull(r, a[2]);
      return r;
    }
  }
}

int oracle_fset_enclosure(const uint32_t* prog, int64_t len, const float* cases,
                          int32_t n_inputs, int64_t n_cases, float* lo, float* hi,
                          uint8_t* may_nan) {
  if (!prog || len <= 0 || n_cases < 0 || (n_cases > 0 && (!lo || !hi || !may_nan))) return -5;
  for (int64_t c = 0; c < (n_cases > 0 ? n_cases : 1); ++c) {
    pctx k = {prog, len, n_cases > 0 ? cases : NULL, n_inputs, n_cases, c, 0};
    int64_t pos = 0;
    ival v = irec(&k, &pos);
    if (k.err) return k.err;
    if (pos != len) return -3;
    if (n_cases > 0) {
      lo[c] = v.lo;
      hi[c] = v.hi;
      may_nan[c] = (uint8_t)(v.nan ? 1 : 0);
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Fitness measures                                                          */
/* ------------------------------------------------------------------------ */
static float case_error(float o, float y, int32_t kind) {
  volatile float d = o - y;
  if (kind == ORC_FIT_CLASS) return (rintf(o) == y) ? 0.0f : 1.0f;
  if (kind == ORC_FIT_MSE) { volatile float e = d * d; return e; }
  return fabsf(d);
}

int oracle_fitness_of_outputs(const float* out, const float* targets, int64_t n_cases,
                              int32_t kind, double* fitness) {
  if (!fitness || n_cases < 0 || kind < ORC_FIT_ABS || kind > ORC_FIT_CLASS) return -5;
  double s = 0.0;
  int nonfinite = 0;
  for (int64_t c = 0; c < n_cases; ++c) {
    float e = case_error(out[c], targets[c], kind);
    if (!isfinite(e)) nonfinite = 1;
    else s += (double)e;
  }
  if (nonfinite) s = INFINITY;
  else if (kind == ORC_FIT_MSE && n_cases > 0) s = s / (double)n_cases;
  *fitness = s;
  return 0;
}

/* the binary32 error of every output in [lo, hi] lies in [elo, ehi] */
static void error_range(float lo, float hi, float y, int32_t kind, float* elo, float* ehi) {
  if (kind == ORC_FIT_CLASS) {
    const float rlo = rintf(lo), rhi = rintf(hi); /* rint is monotone */
    if (rlo == y && rhi == y) { *elo = 0.0f; *ehi = 0.0f; }
    else if (y < rlo || y > rhi) { *elo = 1.0f; *ehi = 1.0f; }
    else { *elo = 0.0f; *ehi = 1.0f; }
    return;
  }
  volatile float dlo = lo - y, dhi = hi - y; /* o - y is monotone in o */
  float mlo, mhi;                            /* |d| range */
  if (dlo <= 0.0f && dhi >= 0.0f) { mlo = 0.0f; mhi = fmaxf(-dlo, dhi); }
  else if (dlo > 0.0f) { mlo = dlo; mhi = dhi; }
  else { mlo = -dhi; mhi = -dlo; }
  if (kind == ORC_FIT_MSE) {
    volatile float a = mlo * mlo, b = mhi * mhi;
    *elo = a;
    *ehi = b;
  } else {
    *elo = mlo;
    *ehi = mhi;
  }
}

int oracle_fitness_enclosure(const float* lo, const float* hi, const uint8_t* may_nan,
                             const float* targets, int64_t n_cases, int32_t kind,
                             double* f_lo, double* f_hi, int32_t* may_inf,
                             int32_t* must_inf) {
  if (!f_lo || !f_hi || !may_inf || !must_inf || n_cases < 0 ||
      kind < ORC_FIT_ABS || kind > ORC_FIT_CLASS)
    return -5;
  double slo = 0.0, shi = 0.0;
  int any_inf = 0, sure_inf = 0;
  for (int64_t c = 0; c < n_cases; ++c) {
    const int empty = lo[c] > hi[c];
    if (kind == ORC_FIT_CLASS) {
      /* NaN (and an empty real part) is a wrong class, never +inf */
      if (empty) { slo += 1.0; shi += 1.0; continue; }
      float elo, ehi;
      error_range(lo[c], hi[c], targets[c], kind, &elo, &ehi);
      if (may_nan[c]) ehi = 1.0f;
      slo += elo;
      shi += ehi;
      continue;
    }
    if (empty) { sure_inf = 1; any_inf = 1; continue; } /* only NaN: +inf */
    if (may_nan[c]) any_inf = 1;
    float elo, ehi;
    error_range(lo[c], hi[c], targets[c], kind, &elo, &ehi);
    if (!isfinite(elo)) { sure_inf = 1; continue; }
    slo += (double)elo;
    /* a finite fitness has every error finite: at most FLT_MAX here */
    if (!isfinite(ehi)) { any_inf = 1; shi += (double)FLT_MAX; }
    else shi += (double)ehi;
  }
  if (kind == ORC_FIT_MSE && n_cases > 0) { slo /= (double)n_cases; shi /= (double)n_cases; }
  *f_lo = slo;
  *f_hi = shi;
  *may_inf = any_inf || sure_inf;
  *must_inf = sure_inf;
  return 0;
}

int oracle_fset_population_fitness(const uint32_t* programs, const int64_t* offsets,
                                   const int32_t* lengths, int32_t p_begin, int32_t p_end,
                                   const float* cases, int32_t n_inputs, int64_t n_cases,
                                   const float* targets, int32_t kind, double* fitness_out) {
  int first = 0;
  float* out = (float*)malloc(sizeof(float) * (size_t)(n_cases > 0 ? n_cases : 1));
  if (!out) return -5;
  for (int32_t p = p_begin; p < p_end; ++p) {
    int rc = oracle_fset_outputs(programs + offsets[p], lengths[p], cases, n_inputs, n_cases, out);
    if (rc == 0) rc = oracle_fitness_of_outputs(out, targets, n_cases, kind, &fitness_out[p]);
    if (rc != 0) {
      fitness_out[p] = NAN;
      if (!first) first = rc;
    }
  }
  free(out);
  return first;
}
