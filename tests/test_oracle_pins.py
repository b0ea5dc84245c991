"""Pins of the CPU oracle to things other than itself (CPU only).

Each test ties the oracle to a fact the paper or mathematics fixes: numpy's
IEEE binary32 arithmetic (library special case), closed-form programs, exact
sums (math.fsum), brute-force truth tables, and a second, independent
evaluation algorithm.  A dropped term, a swapped operand or a wrong sign in the
oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from synth import ADD, SUB, MUL, DIV, VAR, AND, OR, NAND, NOR, IF, tok, const_tokens

X0 = tok(VAR, 0)


def f32(v):
    return np.float32(v)


def same_bits(a, b):
    """Bit equality, except that any NaN equals any NaN."""
    a = np.asarray(a, np.float32)
    b = np.asarray(b, np.float32)
    both_nan = np.isnan(a) & np.isnan(b)
    return np.all((a.view(np.uint32) == b.view(np.uint32)) | both_nan)


def special_operands(rng, n):
    specials = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45,
                         1.17549435e-38, 3.4028235e38, -3.4028235e38, 5e-39, 0.5, 2.0, 3.0],
                        np.float32)
    a = rng.standard_normal(n).astype(np.float32) * np.float32(10) ** rng.integers(-40, 39, n).astype(np.float32)
    idx = rng.integers(0, n, n // 4)
    a[idx] = specials[rng.integers(0, specials.size, idx.size)]
    return a.astype(np.float32)


# ---------------------------------------------------------------------------
# per-node arithmetic: numpy binary32 (round to nearest even, no FMA)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("op", [ADD, SUB, MUL, DIV])
def test_apply_op_matches_numpy_binary32(op):
    rng = np.random.default_rng(10 + op)
    a = special_operands(rng, 4000)
    b = special_operands(rng, 4000)
    with np.errstate(all="ignore"):
        if op == ADD:
            ref = a + b
        elif op == SUB:
            ref = a - b
        elif op == MUL:
            ref = a * b
        else:  # protected division: denominator +0 or -0 -> 1.0f
            ref = np.where(b == 0, np.float32(1.0), a / np.where(b == 0, np.float32(1), b))
    got = np.array([oracle.apply_op(op, x, y) for x, y in zip(a, b)], np.float32)
    assert same_bits(got, ref.astype(np.float32))


def test_protected_division_zero_denominators():
    for num in [0.0, -0.0, 1.0, -5.0, np.inf, np.nan]:
        assert oracle.apply_op(DIV, num, 0.0) == f32(1.0)
        assert oracle.apply_op(DIV, num, -0.0) == f32(1.0)
    # a subnormal denominator divides normally
    assert oracle.apply_op(DIV, 1e-45, 1e-45) == f32(1.0)
    assert np.isinf(oracle.apply_op(DIV, 1.0, 1e-45))


# ---------------------------------------------------------------------------
# closed-form programs
# ---------------------------------------------------------------------------
def xcases(n=2049, seed=5, include_zeros=True):
    x = synth.uniform_cases(seed, 1, n)
    if include_zeros:
        x[0, :4] = [0.0, -0.0, 1.0, -1.0]
    return x


def test_quartic_tree_scores_exactly_zero():
    x = xcases()
    y = synth.quartic_target(x[0])
    prog = synth.quartic_program()
    assert oracle.tree_nodes(prog) == 19
    out = oracle.tree_outputs(prog, x)
    assert same_bits(out, y)
    assert oracle.tree_fitness(prog, x, y) == 0.0


def test_x_minus_x_and_x_over_x():
    x = xcases()
    out = oracle.tree_outputs([tok(SUB), X0, X0], x)
    assert np.all(out == 0.0)
    out = oracle.tree_outputs([tok(DIV), X0, X0], x)
    assert np.all(out == 1.0)  # x != 0 divides to 1; x = +-0 is protected to 1


@pytest.mark.parametrize("op,fn", [
    (SUB, lambda x, c: x - c),
    (DIV, lambda x, c: np.where(c == 0, np.float32(1), x / c)),
])
def test_operand_order_first_child_is_left_operand(op, fn):
    x = xcases()
    c = f32(0.37)
    got = oracle.tree_outputs([tok(op), X0] + const_tokens(c), x)
    assert same_bits(got, fn(x[0], c).astype(np.float32))
    got = oracle.tree_outputs([tok(op)] + const_tokens(c) + [X0], x)
    with np.errstate(all="ignore"):
        ref = (c - x[0]) if op == SUB else np.where(x[0] == 0, np.float32(1), c / x[0])
    assert same_bits(got, ref.astype(np.float32))


def test_constant_tree_and_products():
    x = xcases()
    prog = [tok(ADD)] + const_tokens(0.25) + const_tokens(-0.75)
    assert np.all(oracle.tree_outputs(prog, x) == f32(-0.5))
    prog = [tok(MUL), tok(MUL), X0, X0, tok(MUL), X0, X0]
    ref = (x[0] * x[0]) * (x[0] * x[0])
    assert same_bits(oracle.tree_outputs(prog, x), ref)


def test_paper_worked_example_value():
    # Sec. 5 worked example, RPN (((X,(X,X)+)*,X)-,((X,(X,X)+)*,X)-)* ; as a tree
    # it is ((x*(x+x)) - x) * ((x*(x+x)) - x) with 15 nodes.
    sub = [tok(SUB), tok(MUL), X0, tok(ADD), X0, X0, X0]
    prog = [tok(MUL)] + sub + sub
    x = xcases()
    assert oracle.tree_nodes(prog) == 15
    t = x[0] * (x[0] + x[0]) - x[0]
    assert same_bits(oracle.tree_outputs(prog, x), t * t)


def test_multi_input_indexing():
    x = synth.uniform_cases(7, 3, 301)
    prog = [tok(SUB), tok(VAR, 2), tok(MUL), tok(VAR, 0), tok(VAR, 1)]
    assert same_bits(oracle.tree_outputs(prog, x), x[2] - x[0] * x[1])


# ---------------------------------------------------------------------------
# two independent evaluation algorithms agree on random trees
# ---------------------------------------------------------------------------
def test_recursive_and_stack_evaluators_agree():
    progs = synth.ramped_half_and_half(11, 400, 2, 8, 400, n_inputs=3)
    x = synth.uniform_cases(12, 3, 257)
    x[:, 0] = 0.0  # exercise protected division
    for p in progs:
        a = oracle.tree_outputs(p, x, "recursive")
        b = oracle.tree_outputs(p, x, "stack")
        assert same_bits(a, b)


def test_malformed_programs_rejected():
    x = xcases(8)
    with pytest.raises(oracle.OracleError):
        oracle.tree_outputs([tok(ADD), X0], x)            # truncated
    with pytest.raises(oracle.OracleError):
        oracle.tree_outputs([X0, X0], x)                  # trailing tokens
    with pytest.raises(oracle.OracleError):
        oracle.tree_outputs([tok(99)], x)                 # unknown opcode
    with pytest.raises(oracle.OracleError):
        oracle.tree_outputs([tok(VAR, 1)], x)             # input index out of range


# ---------------------------------------------------------------------------
# fitness: exact sums, non-finite flag
# ---------------------------------------------------------------------------
def test_fitness_matches_exact_sum():
    rng = np.random.default_rng(3)
    progs = synth.ramped_half_and_half(13, 50, 2, 6, 64)
    x = synth.uniform_cases(14, 1, 1000)
    y = rng.uniform(-1, 1, 1000).astype(np.float32)
    for p in progs:
        out = oracle.tree_outputs(p, x)
        with np.errstate(all="ignore"):
            e = np.abs(out - y).astype(np.float32)
        ref = math.fsum(float(v) for v in e) if np.all(np.isfinite(e)) else math.inf
        got = oracle.tree_fitness(p, x, y)
        if math.isinf(ref):
            assert got == math.inf
        else:
            assert abs(got - ref) <= 1e-12 * max(ref, 1e-300)


def test_fitness_nonfinite_is_inf():
    x = xcases(64)
    y = np.zeros(64, np.float32)
    prog = [tok(MUL)] + const_tokens(3e38) + const_tokens(3e38)  # +inf on every case
    assert oracle.tree_fitness(prog, x, y) == math.inf
    prog = [tok(SUB), tok(MUL)] + const_tokens(3e38) + const_tokens(3e38) + \
        [tok(MUL)] + const_tokens(3e38) + const_tokens(3e38)  # inf - inf = NaN
    assert oracle.tree_fitness(prog, x, y) == math.inf


def test_population_fitness_matches_single():
    w = synth.regression_small(n_progs=20, n_cases=128)
    f = oracle.population_fitness(w.pop.words, w.pop.offsets, w.pop.lengths, w.cases, w.targets)
    for p in range(w.pop.n):
        assert f[p] == oracle.tree_fitness(w.pop.program(p), w.cases, w.targets)


# ---------------------------------------------------------------------------
# Boolean: truth tables of known-correct programs, brute force per case
# ---------------------------------------------------------------------------
def xor_tree(a, b):
    # XOR(a, b) = AND(OR(a, b), NAND(a, b))
    return [tok(AND), tok(OR)] + a + b + [tok(NAND)] + a + b


def xnor_tree(a, b):
    # XNOR(a, b) = OR(AND(a, b), NOR(a, b))
    return [tok(OR), tok(AND)] + a + b + [tok(NOR)] + a + b


def even_parity_program(k):
    e = xnor_tree([tok(VAR, 0)], [tok(VAR, 1)])
    for i in range(2, k):
        e = xor_tree(e, [tok(VAR, i)])
    return e


def even_parity_program_if(k):
    """Even-k-parity with XOR(a, b) = IF(a, NOR(b, b), b): linear in k."""
    # XNOR(x0, x1) = IF(x0, x1, NOR(x1, x1))
    e = [tok(IF), tok(VAR, 0), tok(VAR, 1), tok(NOR), tok(VAR, 1), tok(VAR, 1)]
    for i in range(2, k):
        xi = tok(VAR, i)
        e = [tok(IF)] + e + [tok(NOR), xi, xi, xi]
    return e


def mux_program_if(k):
    a = synth.mux_address_bits(k)

    def sel(level, base):
        if level < 0:
            return [tok(VAR, a + base)]
        # address bit `level` set -> upper half
        return [tok(IF), tok(VAR, level)] + sel(level - 1, base + (1 << level)) + sel(level - 1, base)
    return sel(a - 1, 0)


@pytest.mark.parametrize("k", [6, 11])
def test_even_parity_program_scores_all_hits(k):
    prog = even_parity_program(k)
    cb = synth.bool_case_bits(k)
    t = synth.even_parity_target(k)
    assert oracle.bool_hits(prog, cb, 1 << k, t) == 1 << k
    if k == 6:
        assert oracle.tree_nodes(prog) == 187  # the paper-sized XOR chain for 6 inputs


@pytest.mark.parametrize("k", [6, 11, 20])
def test_even_parity_if_program_scores_all_hits(k):
    prog = even_parity_program_if(k)
    assert oracle.bool_hits(prog, synth.bool_case_bits(k), 1 << k, synth.even_parity_target(k)) == 1 << k
    assert oracle.tree_nodes(prog) == 6 + 5 * (k - 2)


@pytest.mark.parametrize("k", [6, 11])
def test_mux_program_scores_all_hits(k):
    prog = mux_program_if(k)
    cb = synth.bool_case_bits(k)
    # 2^a - 1 IF nodes, as many address terminals, 2^a data terminals
    assert oracle.tree_nodes(prog) == (10 if k == 6 else 22)
    assert oracle.bool_hits(prog, cb, 1 << k, synth.mux_target(k)) == 1 << k


def test_nand_negation_scores_zero():
    cb = synth.bool_case_bits(6)
    prog = [tok(NAND), tok(VAR, 0), tok(VAR, 0)]
    assert oracle.bool_hits(prog, cb, 64, cb[0]) == 0


def _brute_bool(prog, k, c):
    bits = [(c >> i) & 1 for i in range(k)]
    pos = 0

    def rec():
        nonlocal pos
        t = int(prog[pos]); pos += 1
        op, arg = t & 0xFF, t >> 8
        if op == VAR:
            return bits[arg]
        a = rec(); b = rec()
        if op == AND:
            return a & b
        if op == OR:
            return a | b
        if op == NAND:
            return 1 - (a & b)
        if op == NOR:
            return 1 - (a | b)
        c3 = rec()
        return b if a else c3
    return rec()


def test_bool_outputs_brute_force_per_case():
    k = 5  # 32 cases: one word
    progs = synth.ramped_half_and_half(21, 60, 2, 6, 80, funcs=synth.BOOL_FUNCS + (IF,),
                                       n_inputs=k, p_const=0.0, full_fallback_to_grow=True)
    cb = synth.bool_case_bits(k)
    for p in progs:
        out = oracle.bool_outputs(p, cb)
        for c in range(32):
            assert ((int(out[0]) >> c) & 1) == _brute_bool(p, k, c)


def test_bool_hits_masks_tail_cases():
    # 3 inputs -> 8 cases in one word; bits 8..31 of every word are not cases
    cb = synth.bool_case_bits(3)
    t = np.array([0xFFFFFFFF], np.uint32)  # target 1 everywhere (incl. padding)
    prog = [tok(OR), tok(VAR, 0), tok(NOR), tok(VAR, 0), tok(VAR, 0)]  # a OR NOT a = 1
    assert oracle.bool_hits(prog, cb, 8, t) == 8


# ---------------------------------------------------------------------------
# register linear GP
# ---------------------------------------------------------------------------
def test_linear_closed_forms():
    x = synth.normal_cases(31, 8, 513)
    x[1, :3] = 0.0
    ins = np.array([[0, ADD, 0, 1]], np.uint8)
    assert same_bits(oracle.linear_outputs(ins, x), x[0] + x[1])
    ins = np.array([[3, SUB, 1, 2], [0, DIV, 3, 1]], np.uint8)
    t = x[1] - x[2]
    ref = np.where(x[1] == 0, np.float32(1), t / np.where(x[1] == 0, np.float32(1), x[1]))
    assert same_bits(oracle.linear_outputs(ins, x), ref)
    # registers beyond the inputs start at 0
    ins = np.array([[0, ADD, 6, 7]], np.uint8)
    assert np.all(oracle.linear_outputs(ins, x[:2]) == 0.0)


def test_linear_matches_brute_force():
    pop = synth.linear_programs(32, 30, 4, 40)
    x = synth.normal_cases(33, 8, 17)
    for p in range(pop.n):
        ins = pop.program(p)
        got = oracle.linear_outputs(ins, x)
        ref = np.empty(x.shape[1], np.float32)
        for c in range(x.shape[1]):
            r = [np.float32(x[i, c]) for i in range(8)]
            for d, op, a, b in ins:
                ra, rb = r[a], r[b]
                with np.errstate(all="ignore"):
                    if op == ADD:
                        v = ra + rb
                    elif op == SUB:
                        v = ra - rb
                    elif op == MUL:
                        v = ra * rb
                    else:
                        v = np.float32(1) if rb == 0 else ra / rb
                r[d] = np.float32(v)
            ref[c] = r[0]
        assert same_bits(got, ref)


def test_linear_agrees_with_tree_encoding():
    """A constant-free tree over x0..x3, written as register code by a small
    test-side translation (stack level L -> register 4 + L, the root writes r0),
    evaluates bit-identically in the two oracles."""
    progs = synth.ramped_half_and_half(41, 200, 2, 4, 15, n_inputs=4, p_const=0.0)
    x = synth.uniform_cases(42, 4, 200)
    x[:, :2] = 0.0
    for p in progs:
        rows = []

        def emit(pos, level):
            t = int(p[pos])
            op, arg = t & 0xFF, t >> 8
            if op == VAR:
                return pos + 1, arg
            pos, ra = emit(pos + 1, level)
            pos, rb = emit(pos, level + 1)
            rows.append([4 + level, op, ra, rb])
            return pos, 4 + level

        end, _ = emit(0, 0)
        assert end == len(p)
        rows[-1][0] = 0  # the root's result goes to the output register
        ins = np.array(rows, np.uint8)
        assert same_bits(oracle.linear_outputs(ins, x), oracle.tree_outputs(p, x))
