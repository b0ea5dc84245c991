"""Pins of the oracle's full float function sets, fitness measures and
enclosures (CPU only).

Sec. 4.2 names the float function sets (sextic: *, /, +, -, Sin, Cos, Log,
Exp; Shuttle: *, /, +, -, >, <, ==, AND, OR, IF; KDDcup: all) and the
parameter table the fitness measures (mean squared error; number of incorrect
classifications).  The oracle's readings of these are pinned here to things
other than itself: numpy's IEEE comparisons, selections and binary32
arithmetic, closed forms (sin^2 + cos^2 = 1, log(exp(x)) = x, the sextic
polynomial's roots), and brute force over admissible implementations: a
Python evaluator that moves every transcendental result by a random number of
ulps within the documented bound must land inside the oracle's enclosure on
every case.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from synth import (ADD, SUB, MUL, DIV, VAR, CONST, AND, OR, NAND, IF, SIN, COS, EXP, LOG, GT, LT,
                   EQ, tok, const_tokens)

X0, X1 = tok(VAR, 0), tok(VAR, 1)
ULP = {SIN: 2, COS: 2, EXP: 2, LOG: 1}


def prog(*parts):
    out = []
    for p in parts:
        out.extend(p if isinstance(p, list) else [p])
    return np.asarray(out, np.uint32)


def C(v):
    return const_tokens(v)


SPECIALS = np.array([0.0, -0.0, 1.0, -1.0, 0.5, 2.0, -3.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45,
                     1e-38, 3.4e38, -3.4e38, 100.0, 1e6, -7.25], np.float32)


# ---------------------------------------------------------------------------
# an independent Python evaluator (numpy binary32 scalars), with optional
# perturbation of the transcendental results inside their ulp bounds
# ---------------------------------------------------------------------------
def _step(v, k):
    v = np.float32(v)
    d = np.float32(np.inf) if k > 0 else np.float32(-np.inf)
    for _ in range(abs(k)):
        v = np.nextafter(v, d)
    return v


def _unary(op, a, rng):
    a64 = np.float64(a)
    with np.errstate(all="ignore"):
        if op == LOG:
            if a == 0:
                return np.float32(0.0)
            exact = np.log(np.abs(a64))
        elif op == SIN:
            exact = np.sin(a64)
        elif op == COS:
            exact = np.cos(a64)
        else:
            exact = np.exp(a64)
        v = np.float32(exact)
    if rng is not None and not np.isnan(v):
        v = _step(v, int(rng.integers(-ULP[op], ULP[op] + 1)))
    return v


def py_eval(p, xs, rng=None):
    """Value of prefix tree p on one case (xs: the inputs, binary32)."""
    def ev(pos):
        t = int(p[pos])
        op, arg = t & 0xFF, t >> 8
        pos += 1
        if op == VAR:
            return np.float32(xs[arg]), pos
        if op == CONST:
            return np.uint32(p[pos]).view(np.float32), pos + 1
        args = []
        for _ in range(synth.ARITY[op]):
            v, pos = ev(pos)
            args.append(v)
        with np.errstate(all="ignore"):
            if op in ULP:
                return _unary(op, args[0], rng), pos
            a = args[0]
            b = args[1] if len(args) > 1 else None
            if op == ADD:
                return np.float32(a + b), pos
            if op == SUB:
                return np.float32(a - b), pos
            if op == MUL:
                return np.float32(a * b), pos
            if op == DIV:
                return (np.float32(1.0) if b == 0 else np.float32(a / b)), pos
            if op == GT:
                return np.float32(1.0 if a > b else 0.0), pos
            if op == LT:
                return np.float32(1.0 if a < b else 0.0), pos
            if op == EQ:
                return np.float32(1.0 if a == b else 0.0), pos
            if op == AND:
                return np.float32(1.0 if (a != 0 and b != 0) else 0.0), pos
            if op == OR:
                return np.float32(1.0 if (a != 0 or b != 0) else 0.0), pos
            if op == IF:
                return (args[1] if a != 0 else args[2]), pos
        raise AssertionError(op)

    v, end = ev(0)
    assert end == len(p)
    return v


def special_cases(seed, n_inputs, n):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-3, 3, (n_inputs, n)).astype(np.float32)
    m = rng.random((n_inputs, n)) < 0.3
    x[m] = SPECIALS[rng.integers(0, SPECIALS.size, int(m.sum()))]
    return x


def inside(v, lo, hi, may_nan):
    if np.isnan(v):
        return bool(may_nan)
    return bool(lo <= v <= hi)


# ---------------------------------------------------------------------------
def test_arity_and_errors():
    assert [oracle.fset_arity(op) for op in (VAR, CONST, SIN, COS, EXP, LOG, ADD, GT, AND, IF)] == \
        [0, 0, 1, 1, 1, 1, 2, 2, 2, 3]
    x = np.zeros((2, 3), np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.fset_outputs(prog(NAND, X0, X0), x)          # Boolean-only function
    with pytest.raises(oracle.OracleError):
        oracle.fset_outputs(prog(SIN), x)                   # missing operand
    with pytest.raises(oracle.OracleError):
        oracle.fset_outputs(prog(ADD, X0, tok(VAR, 2)), x)  # input out of range
    with pytest.raises(oracle.OracleError):
        oracle.fset_enclosure(prog(X0, X0), x)              # trailing tokens
    assert oracle.fset_outputs(prog(SIN, tok(VAR, 1)), np.zeros((2, 0), np.float32)).size == 0


def test_basic_set_agrees_with_the_pinned_evaluator():
    progs = synth.ramped_half_and_half(21, 120, 2, 6, 64, n_inputs=2)
    x = special_cases(22, 2, 40)
    for p in progs:
        a = oracle.fset_outputs(p, x)
        b = oracle.tree_outputs(p, x)
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32)) or \
            np.all((a.view(np.uint32) == b.view(np.uint32)) | (np.isnan(a) & np.isnan(b)))


@pytest.mark.parametrize("op", [GT, LT, EQ, AND, OR])
def test_comparisons_and_logic_match_numpy(op):
    a, b = np.meshgrid(SPECIALS, SPECIALS)
    a, b = a.ravel(), b.ravel()
    x = np.stack([a, b])
    got = oracle.fset_outputs(prog(op, X0, X1), x)
    ref = {GT: np.greater(a, b), LT: np.less(a, b), EQ: np.equal(a, b),
           AND: np.logical_and(a != 0, b != 0), OR: np.logical_or(a != 0, b != 0)}[op]
    assert np.array_equal(got, ref.astype(np.float32))
    lo, hi, nan = oracle.fset_enclosure(prog(op, X0, X1), x)
    assert np.array_equal(lo, got) and np.array_equal(hi, got) and not nan.any()


def test_if_selects_and_max_identity():
    rng = np.random.default_rng(3)
    c = np.concatenate([SPECIALS, rng.standard_normal(50).astype(np.float32)])
    a = rng.standard_normal(c.size).astype(np.float32)
    b = rng.standard_normal(c.size).astype(np.float32)
    got = oracle.fset_outputs(prog(IF, X0, X1, tok(VAR, 2)), np.stack([c, a, b]))
    assert np.array_equal(got, np.where(c != 0, a, b))  # NaN != 0 selects a
    x = rng.uniform(-2, 2, 200).astype(np.float32)
    m = oracle.fset_outputs(prog(IF, GT, X0, C(0.25), X0, C(0.25)), x)
    assert np.array_equal(m, np.maximum(x, np.float32(0.25)))


def test_transcendental_closed_forms():
    x = np.array([0.0], np.float32)
    lo, hi, nan = oracle.fset_enclosure(prog(LOG, C(0.0)), x)
    assert lo[0] == 0 and hi[0] == 0 and not nan[0]          # protected log(0) is exactly 0
    lo, hi, _ = oracle.fset_enclosure(prog(LOG, C(-0.0)), x)
    assert lo[0] == 0 and hi[0] == 0
    for p, truth in ((prog(SIN, C(0.0)), 0.0), (prog(COS, C(0.0)), 1.0), (prog(EXP, C(0.0)), 1.0),
                     (prog(LOG, C(1.0)), 0.0), (prog(LOG, C(-math.e)), 1.0),
                     (prog(SIN, C(math.pi / 6)), math.sin(float(np.float32(math.pi / 6))))):
        lo, hi, nan = oracle.fset_enclosure(p, x)
        assert lo[0] <= truth <= hi[0] and not nan[0]
    xs = np.linspace(-3, 3, 301).astype(np.float32)
    pos = np.abs(xs) + np.float32(0.01)
    # sin^2 + cos^2 = 1
    lo, hi, nan = oracle.fset_enclosure(prog(ADD, MUL, SIN, X0, SIN, X0, MUL, COS, X0, COS, X0), xs)
    assert np.all((lo <= 1) & (hi >= 1)) and not nan.any()
    assert np.all((hi - lo) <= 16 * np.spacing(np.float32(1)))
    # exp(log(x)) = x for x > 0, log(exp(x)) = x
    lo, hi, _ = oracle.fset_enclosure(prog(EXP, LOG, X0), pos)
    assert np.all((lo <= pos) & (pos <= hi))
    lo, hi, _ = oracle.fset_enclosure(prog(LOG, EXP, X0), xs)
    assert np.all((lo <= xs.astype(np.float64)) & (xs.astype(np.float64) <= hi))
    # sine is odd, cosine even: enclosures mirror
    lo1, hi1, _ = oracle.fset_enclosure(prog(SIN, X0), xs)
    lo2, hi2, _ = oracle.fset_enclosure(prog(SIN, X0), -xs)
    assert np.array_equal(lo1, -hi2) and np.array_equal(hi1, -lo2)
    lo1, hi1, _ = oracle.fset_enclosure(prog(COS, X0), xs)
    lo2, hi2, _ = oracle.fset_enclosure(prog(COS, X0), -xs)
    assert np.array_equal(lo1, lo2) and np.array_equal(hi1, hi2)
    # sin(0) may be exactly 0 and exp(1000) is +inf: 0 * inf is NaN although
    # neither operand's enclosure ends at a zero times an infinity
    lo, hi, nan = oracle.fset_enclosure(prog(MUL, SIN, C(0.0), EXP, X0), np.array([1000.0], np.float32))
    assert nan[0] and lo[0] == -np.inf and hi[0] == np.inf
    assert np.isnan(py_eval(prog(MUL, SIN, C(0.0), EXP, X0), [np.float32(1000.0)]))
    # non-finite operands
    lo, hi, nan = oracle.fset_enclosure(prog(SIN, X0), np.array([np.inf, -np.inf, np.nan], np.float32))
    assert nan.all() and np.all(lo > hi)                       # NaN only
    lo, hi, nan = oracle.fset_enclosure(prog(EXP, X0), np.array([np.inf, -np.inf, 100.0], np.float32))
    assert hi[0] == np.inf and lo[1] <= 0 <= hi[1] and hi[2] == np.inf and not nan.any()


@pytest.mark.parametrize("op", [SIN, COS, EXP, LOG])
def test_single_function_enclosure_is_tight(op):
    rng = np.random.default_rng(40 + op)
    x = rng.uniform(-20, 20, 2000).astype(np.float32)
    lo, hi, nan = oracle.fset_enclosure(prog(op, X0), x)
    pt = oracle.fset_outputs(prog(op, X0), x)
    assert not nan.any()
    assert np.all((lo <= pt) & (pt <= hi))
    # width: at most 2 * (bound + 1) binary32 steps around the point value
    steps_lo = np.array([_count_steps(a, b) for a, b in zip(lo, pt)])
    steps_hi = np.array([_count_steps(a, b) for a, b in zip(pt, hi)])
    assert steps_lo.max() <= ULP[op] + 2 and steps_hi.max() <= ULP[op] + 2


def _count_steps(a, b):
    """binary32 steps from a up to b (a <= b)."""
    n = 0
    a = np.float32(a)
    while a < b and n < 100:
        a = np.nextafter(a, np.float32(np.inf))
        n += 1
    return n


def test_admissible_implementations_fall_inside():
    """Brute force: random trees over the full sets on inputs with specials;
    every case of every perturbed (admissible) evaluation is inside."""
    funcs = (ADD, SUB, MUL, DIV, SIN, COS, EXP, LOG, GT, LT, EQ, AND, OR, IF)
    progs = synth.ramped_half_and_half(31, 160, 2, 5, 48, funcs=funcs, n_inputs=3,
                                       const_lo=-2.0, const_hi=2.0)
    x = special_cases(32, 3, 24)
    rng = np.random.default_rng(33)
    checked = 0
    for p in progs:
        lo, hi, nan = oracle.fset_enclosure(p, x)
        for trial in range(3):
            for c in range(x.shape[1]):
                v = py_eval(p, x[:, c], rng)
                assert inside(v, lo[c], hi[c], nan[c]), (p.tolist(), c, v, lo[c], hi[c], nan[c])
                checked += 1
    assert checked == 160 * 3 * 24


def test_exact_function_sets_give_point_enclosures():
    funcs = (ADD, SUB, MUL, DIV, GT, LT, EQ, AND, OR, IF)   # no transcendental
    progs = synth.ramped_half_and_half(34, 150, 2, 6, 64, funcs=funcs, n_inputs=3,
                                       const_lo=-200.0, const_hi=200.0)
    x = special_cases(35, 3, 30)
    for p in progs:
        out = oracle.fset_outputs(p, x)
        lo, hi, nan = oracle.fset_enclosure(p, x)
        ref = np.array([py_eval(p, x[:, c]) for c in range(x.shape[1])], np.float32)
        fin = ~np.isnan(ref)
        assert np.array_equal(np.isnan(out), ~fin)
        assert np.array_equal(out[fin], ref[fin])            # ignores the sign of zero
        assert np.array_equal(lo[fin], ref[fin]) and np.array_equal(hi[fin], ref[fin])
        assert np.all(nan[~fin]) and np.all(lo[~fin] > hi[~fin])


# ---------------------------------------------------------------------------
# fitness measures
# ---------------------------------------------------------------------------
def test_fitness_measures_match_numpy():
    rng = np.random.default_rng(50)
    o = rng.standard_normal(1000).astype(np.float32)
    y = rng.standard_normal(1000).astype(np.float32)
    d = o - y
    assert oracle.fitness_of_outputs(o, y, oracle.FIT_ABS) == math.fsum(np.abs(d).astype(np.float64)) or \
        abs(oracle.fitness_of_outputs(o, y, oracle.FIT_ABS) - math.fsum(np.abs(d).astype(np.float64))) < 1e-9
    mse = oracle.fitness_of_outputs(o, y, oracle.FIT_MSE)
    assert abs(mse - math.fsum((d * d).astype(np.float64)) / 1000) < 1e-12
    labels = rng.integers(0, 5, 1000).astype(np.float32)
    outs = (labels + rng.choice(np.array([-0.7, -0.4, 0.0, 0.49, 0.5, 1.5, np.nan], np.float32),
                                1000)).astype(np.float32)
    wrong = np.count_nonzero(np.rint(outs) != labels)        # NaN never matches; ties to even
    assert oracle.fitness_of_outputs(outs, labels, oracle.FIT_CLASS) == wrong
    # a non-finite error makes ABS and MSE +inf, never CLASS
    o2 = o.copy()
    o2[3] = np.float32(3e19)                                  # square overflows
    assert oracle.fitness_of_outputs(o2, y, oracle.FIT_MSE) == np.inf
    assert np.isfinite(oracle.fitness_of_outputs(o2, y, oracle.FIT_ABS))
    o2[4] = np.nan
    assert oracle.fitness_of_outputs(o2, y, oracle.FIT_ABS) == np.inf
    assert oracle.fitness_of_outputs(o2, labels, oracle.FIT_CLASS) <= 1000
    assert oracle.fitness_of_outputs(o[:0], y[:0], oracle.FIT_MSE) == 0.0


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_fitness_enclosure_contains_admissible_fitness(kind):
    funcs = (ADD, SUB, MUL, DIV, SIN, COS, EXP, LOG, GT, LT, IF)
    progs = synth.ramped_half_and_half(60 + kind, 60, 2, 5, 40, funcs=funcs, n_inputs=2)
    x = special_cases(63, 2, 32)
    x[:, :4] = np.float32(0.25)  # some finite cases on every program
    y = np.rint(np.random.default_rng(64).uniform(-2, 2, 32)).astype(np.float32)
    rng = np.random.default_rng(65)
    for p in progs:
        lo, hi, nan = oracle.fset_enclosure(p, x)
        f_lo, f_hi, may_inf, must_inf = oracle.fitness_enclosure(lo, hi, nan, y, kind)
        assert f_lo <= f_hi
        for trial in range(4):
            out = np.array([py_eval(p, x[:, c], rng) for c in range(32)], np.float32)
            f = oracle.fitness_of_outputs(out, y, kind)
            if f == np.inf:
                assert may_inf
            else:
                assert not must_inf and f_lo <= f <= f_hi, (f_lo, f, f_hi)


def test_point_fitness_enclosure_is_the_fitness():
    progs = synth.ramped_half_and_half(70, 40, 2, 6, 64)
    x = synth.uniform_cases(71, 1, 256)
    y = synth.quartic_target(x[0])
    for kind in (0, 1, 2):
        for p in progs:
            out = oracle.fset_outputs(p, x)
            lo, hi, nan = oracle.fset_enclosure(p, x)
            f = oracle.fitness_of_outputs(out, y, kind)
            f_lo, f_hi, may_inf, must_inf = oracle.fitness_enclosure(lo, hi, nan, y, kind)
            if f == np.inf:
                assert may_inf
            else:
                assert f_lo == f == f_hi


def test_sextic_target_roots_and_values():
    """x^6 - 2x^4 + x^2 = x^2 (x^2 - 1)^2 (Sec. 4.2): zero at 0 and +-1."""
    xx = [MUL, X0, X0]
    p = prog(MUL, xx, MUL, SUB, xx, C(1.0), SUB, xx, C(1.0))
    x = np.array([0.0, 1.0, -1.0, 0.5, -0.25], np.float32)
    out = oracle.fset_outputs(p, x)
    assert np.all(out[:3] == 0)
    x64 = x.astype(np.float64)
    assert np.allclose(out, x64 ** 6 - 2 * x64 ** 4 + x64 ** 2, rtol=1e-6, atol=0)
    y = synth.sextic_target(x)
    assert np.all(y[:3] == 0) and np.allclose(y, x64 ** 6 - 2 * x64 ** 4 + x64 ** 2, rtol=1e-7)
