"""Host encoder tests (CPU): the paper's worked example, stack-depth bounds,
and encoded programs evaluated by the test-side reader against the oracle."""
import os

import numpy as np
import pytest

import oracle
import synth
import paper_1601_00221_gb300 as gp
from synth import ADD, SUB, MUL, DIV, VAR, CONST, tok, const_tokens
import encoded_ref as ref
from div_trees import constant_divisor_trees, edge_cases, bitsf32

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sec5_worked_example.txt")


def load_golden():
    d = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split(":", 1)
            d[k.strip()] = v.strip()
    return d


def parse_rpn_text(s):
    """'(A,B)op' nested RPN text of the paper -> prefix tokens (X = input 0)."""
    ops = {"+": ADD, "-": SUB, "*": MUL, "/": DIV}
    pos = 0

    def elem():
        nonlocal pos
        if s[pos] == "X":
            pos += 1
            return [tok(VAR, 0)]
        assert s[pos] == "("
        pos += 1
        a = elem()
        assert s[pos] == ","
        pos += 1
        b = elem()
        assert s[pos] == ")"
        pos += 1
        op = ops[s[pos]]
        pos += 1
        return [tok(op)] + a + b
    t = elem()
    assert pos == len(s)
    return t


def same_bits(a, b):
    a = np.asarray(a, np.float32)
    b = np.asarray(b, np.float32)
    return np.all((a.view(np.uint32) == b.view(np.uint32)) | (np.isnan(a) & np.isnan(b)))


def test_worked_example_sec5():
    g = load_golden()
    prog = parse_rpn_text(g["rpn"])
    assert oracle.tree_nodes(prog) == int(g["nodes"])
    w, info = gp.encode_tree(prog, gp.KIND_SFORM, gp.ORDER_PAPER)
    assert ref.render_sform(w) == g["sform"]
    assert info["n_instr"] == int(g["sform_instructions"])
    assert info["n_instr"] + 2 * info["n_instr"] == int(g["sform_values"])  # functions + operands
    assert info["stack_reads"] == int(g["sform_stack_fetches"])
    assert info["max_depth"] == int(g["sform_max_stack"])
    w, info = gp.encode_tree(prog, gp.KIND_RPN, gp.ORDER_PAPER)
    assert info["n_instr"] == int(g["rpn_instructions"])
    assert info["stack_reads"] == int(g["rpn_stack_fetches"])
    assert info["max_depth"] == int(g["rpn_max_stack"])


def postfix_depth(prog):
    """Classical stack depth of the postfix order (children left to right)."""
    d, best = 0, 0
    # postfix = reverse of the right-to-left prefix scan's push sequence; scan
    # recursively instead
    pos = 0

    def rec():
        nonlocal pos, d, best
        t = int(prog[pos]); op = t & 0xFF
        pos += 2 if op == CONST else 1
        if op in (VAR, CONST):
            d += 1
            best = max(best, d)
            return
        rec(); rec()
        d -= 1
    rec()
    return best


def sethi_ullman(prog):
    """Registers needed when terminals need none and the bigger child goes first."""
    pos = 0

    def rec():
        nonlocal pos
        t = int(prog[pos]); op = t & 0xFF
        pos += 2 if op == CONST else 1
        if op in (VAR, CONST):
            return 0
        a, b = rec(), rec()
        if a == 0 and b == 0:
            return 1
        return max(a, b) if a != b else a + 1
    return rec()


def test_depths_match_independent_counts():
    progs = synth.ramped_half_and_half(51, 300, 2, 8, 255, n_inputs=2)
    for p in progs:
        _, info = gp.encode_tree(p, gp.KIND_RPN, gp.ORDER_PAPER)
        assert info["max_depth"] == postfix_depth(p)
        _, info = gp.encode_tree(p, gp.KIND_SFORM, gp.ORDER_MIN_DEPTH)
        assert info["max_depth"] == max(1, sethi_ullman(p))
        assert info["n_nodes"] == synth.count_nodes(p)


def chain_tree(n_funcs):
    """Right-leaning chain f(x, f(x, ...)): deep in paper order."""
    t = []
    for i in range(n_funcs):
        t += [tok([ADD, SUB, MUL, DIV][i % 4]), tok(VAR, 0)]
    return t + [tok(VAR, 0)]


def balanced(depth):
    if depth == 1:
        return [tok(VAR, 0)]
    return [tok(SUB)] + balanced(depth - 1) + balanced(depth - 1)


def test_min_depth_fits_register_levels():
    # a full tree of 255 functions (depth 9) needs 8 S-form levels
    p = balanced(9)
    _, info = gp.encode_tree(p, gp.KIND_SFORM, gp.ORDER_MIN_DEPTH)
    assert info["max_depth"] == 8
    # a left-deep-right chain is shallow in either order for S-form
    _, info = gp.encode_tree(chain_tree(100), gp.KIND_SFORM, gp.ORDER_PAPER)
    assert info["max_depth"] == 1
    # in RPN paper order the chain is too deep for the register levels
    with pytest.raises(gp.GPError) as e:
        gp.encode_tree(chain_tree(20), gp.KIND_RPN, gp.ORDER_PAPER)
    assert e.value.code == 2
    _, info = gp.encode_tree(chain_tree(20), gp.KIND_RPN, gp.ORDER_MIN_DEPTH)
    assert info["max_depth"] == 2


@pytest.mark.parametrize("kind", [gp.KIND_SFORM, gp.KIND_RPN])
@pytest.mark.parametrize("order", [gp.ORDER_PAPER, gp.ORDER_MIN_DEPTH])
def test_encoded_programs_match_oracle(kind, order):
    w = synth.regression_small(seed=61, n_progs=120, n_cases=97)
    x = w.cases.copy()
    x[0, :3] = [0.0, -0.0, 1e-40]
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, kind, order)
    assert enc.nodes == int(w.pop.nodes.sum())
    for p in range(w.pop.n):
        words = enc.words[enc.offsets[p]: enc.offsets[p] + enc.lengths[p]]
        assert same_bits(ref.run_float(words, x), oracle.tree_outputs(w.pop.program(p), x))


def test_encoded_multi_input_and_single_terminals():
    progs = synth.ramped_half_and_half(62, 80, 2, 5, 64, n_inputs=3)
    progs += [np.array([tok(VAR, 2)], np.uint32), np.array(const_tokens(0.625), np.uint32)]
    x = synth.uniform_cases(63, 3, 33)
    for kind in (gp.KIND_SFORM, gp.KIND_RPN):
        for p in progs:
            words, info = gp.encode_tree(p, kind, gp.ORDER_MIN_DEPTH)
            assert same_bits(ref.run_float(words, x), oracle.tree_outputs(p, x))


def test_encoded_bool_matches_oracle():
    for kind, k in (("parity", 6), ("mux", 6), ("mux", 11)):
        w = synth.boolean_problem(kind, k, seed=64, n_progs=60)
        enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_BOOL,
                                   gp.ORDER_MIN_DEPTH)
        for p in range(w.pop.n):
            words = enc.words[enc.offsets[p]: enc.offsets[p] + enc.lengths[p]]
            got = ref.run_bool(words, w.case_bits)
            exp = oracle.bool_outputs(w.pop.program(p), w.case_bits)
            assert np.array_equal(got, exp)


def test_encoded_linear_matches_oracle():
    pop = synth.linear_programs(65, 40, 1, 60)
    x = synth.normal_cases(66, 8, 41)
    enc = gp.encode_linear_population(pop.instr, pop.offsets, pop.lengths)
    assert enc.nodes == int(pop.lengths.sum())
    for p in range(pop.n):
        words = enc.words[enc.offsets[p]: enc.offsets[p] + enc.lengths[p]]
        assert same_bits(ref.run_float(words, x), oracle.linear_outputs(pop.program(p), x))


def test_register_file_flags_are_sound():
    """The encoder's operand-source and dead-result flags: a program run with
    operands taken from A (the previous result) or B (the value the load
    rules last put there) and dead results never written gives the oracle's
    outputs, on programs full of repeated registers (2 and 8 registers in
    use), with 3 to 11 inputs; and the flags do fire (operands from A and
    from B, dead results)."""
    x = synth.normal_cases(67, 11, 29)
    fwd = from_b = dead = 0
    for seed, n_regs in ((68, 2), (69, 8), (70, 3)):
        pop = synth.linear_programs(seed, 60, 1, 90, n_regs=n_regs)
        enc = gp.encode_linear_population(pop.instr, pop.offsets, pop.lengths)
        for n_in in (3, 8, 11):
            xi = x[:n_in]
            for p in range(pop.n):
                words = enc.words[enc.offsets[p]: enc.offsets[p] + enc.lengths[p]]
                assert same_bits(ref.run_float(words, xi, register_file=True),
                                 oracle.linear_outputs(pop.program(p), xi)), (seed, n_in, p)
        flags = np.array([f for _, _, f, _ in (ins for p in range(pop.n) for ins in
                          ref.instrs(enc.words[enc.offsets[p]: enc.offsets[p] + enc.lengths[p]]))])
        fwd += int(np.sum(flags & 3 == 1) + np.sum((flags >> 2) & 3 == 1))
        from_b += int(np.sum(flags & 3 == 2) + np.sum((flags >> 2) & 3 == 2))
        dead += int(np.sum(flags & 16 != 0))
        assert not np.any((flags & 3 != 0) & ((flags >> 2) & 3 != 0))  # at most one operand held
    assert fwd > 100 and from_b > 100 and dead > 100


@pytest.mark.parametrize("bad", [
    [tok(ADD), tok(VAR, 0)],                      # missing operand
    [tok(VAR, 0), tok(VAR, 0)],                    # trailing tokens
    [tok(77)],                                     # unknown opcode
    [tok(CONST)],                                  # constant without value
    [tok(synth.NAND), tok(VAR, 0), tok(VAR, 1)],   # Boolean-only function in a float tree
])
def test_malformed_trees_rejected(bad):
    with pytest.raises(gp.GPError) as e:
        gp.encode_tree(bad, gp.KIND_SFORM)
    assert e.value.code == 2


def test_population_reports_bad_index():
    progs = [np.array([tok(VAR, 0)], np.uint32)] * 3 + [np.array([tok(ADD)], np.uint32)]
    pop = synth.pack(progs)
    with pytest.raises(gp.GPError):
        gp.encode_population(pop.words, pop.offsets, pop.lengths)


def test_programs_are_16_byte_aligned():
    w = synth.regression_small(n_progs=33, n_cases=8)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths)
    assert enc.words.ctypes.data % 16 == 0
    assert np.all(enc.offsets % 4 == 0) and np.all(enc.lengths % 4 == 0)


# ---------------------------------------------------------------------------
# the full float function sets (Sec. 4.2): extended S-form encoding
# ---------------------------------------------------------------------------
EXACT_SETS = (synth.SHUTTLE_FUNCS,)
ALL_SET = synth.KDD_FUNCS


def test_extended_trees_encode_with_the_extended_kind():
    progs = synth.ramped_half_and_half(81, 60, 2, 6, 64, funcs=ALL_SET, n_inputs=3)
    pop = synth.pack(progs)
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths, with_info=True)
    kinds = enc.words[enc.offsets] & 0xFF
    uses = np.array([any((int(t) & 0xFF) in (synth.SIN, synth.COS, synth.EXP, synth.LOG, synth.GT,
                                             synth.LT, synth.EQ, synth.AND, synth.OR, synth.IF)
                         for t in _tokens(p)) for p in progs])
    assert np.array_equal(kinds == gp.KIND_SFORM_EXT, uses)
    assert np.array_equal(enc.info["extended"] == 1, uses)
    assert enc.extended == bool(uses.any())
    basic = synth.pack(synth.ramped_half_and_half(82, 20, 2, 5, 40))
    assert not gp.encode_population(basic.words, basic.offsets, basic.lengths).extended


def _tokens(p):
    """Opcode tokens of a prefix tree (constant payload words skipped)."""
    out, i = [], 0
    while i < len(p):
        out.append(p[i])
        i += 2 if (int(p[i]) & 0xFF) == synth.CONST else 1
    return out


@pytest.mark.parametrize("order", [gp.ORDER_PAPER, gp.ORDER_MIN_DEPTH])
def test_encoded_exact_extended_programs_match_oracle(order):
    """No transcendental function: the encoded program reproduces the oracle
    bit for bit (NaN == NaN)."""
    progs = synth.ramped_half_and_half(83, 150, 2, 6, 64, funcs=synth.SHUTTLE_FUNCS, n_inputs=4,
                                       const_lo=-200.0, const_hi=200.0)
    rng = np.random.default_rng(84)
    x = rng.integers(-100, 101, (4, 97)).astype(np.float32)
    x[:, :5] = np.array([0.0, -0.0, np.nan, np.inf, 1e-45], np.float32)
    for p in progs:
        words, info = gp.encode_tree(p, gp.KIND_SFORM, order)
        got = ref.run_float(words, x)
        exp = oracle.fset_outputs(p, x)
        assert same_bits(got, exp), p.tolist()


def test_encoded_transcendental_programs_inside_enclosures():
    progs = synth.ramped_half_and_half(85, 120, 2, 6, 64, funcs=ALL_SET, n_inputs=2)
    x = synth.uniform_cases(86, 2, 64, -3.0, 3.0)
    for p in progs:
        words, _ = gp.encode_tree(p, gp.KIND_SFORM, gp.ORDER_MIN_DEPTH)
        got = ref.run_float(words, x)
        lo, hi, nan = oracle.fset_enclosure(p, x)
        ok = np.where(np.isnan(got), nan, (lo <= got) & (got <= hi))
        assert ok.all(), p.tolist()


@pytest.mark.parametrize("order", [gp.ORDER_PAPER, gp.ORDER_MIN_DEPTH])
def test_extended_rpn_matches_oracle(order):
    """Extended functions in the RPN form: exact sets bit for bit, the full
    set inside the oracle's enclosures."""
    x = synth.uniform_cases(88, 3, 80, -3.0, 3.0)
    x[:, :3] = np.array([0.0, -0.0, np.nan], np.float32)[None, :]
    exact = synth.ramped_half_and_half(89, 120, 2, 6, 64, funcs=synth.SHUTTLE_FUNCS, n_inputs=3,
                                       full_fallback_to_grow=True)
    for p in exact:
        words, _ = gp.encode_tree(p, gp.KIND_RPN, order)
        assert (int(words[0]) & 0xFF) in (gp.KIND_RPN, gp.KIND_RPN_EXT)
        assert same_bits(ref.run_float(words, x), oracle.fset_outputs(p, x)), p.tolist()
    full = synth.ramped_half_and_half(90, 120, 2, 6, 64, funcs=synth.KDD_FUNCS, n_inputs=3,
                                      full_fallback_to_grow=True)
    for p in full:
        words, _ = gp.encode_tree(p, gp.KIND_RPN, order)
        got = ref.run_float(words, x)
        lo, hi, nan = oracle.fset_enclosure(p, x)
        assert np.where(np.isnan(got), nan, (lo <= got) & (got <= hi)).all(), p.tolist()


def test_nand_is_rejected_in_float_trees():
    with pytest.raises(gp.GPError) as e:
        gp.encode_tree(np.array([synth.NAND, synth.tok(synth.VAR, 0), synth.tok(synth.VAR, 0)],
                                np.uint32), gp.KIND_SFORM)
    assert e.value.code == 2


def test_if_forms_cover_every_operand_mix():
    """IF with each operand an input, a constant or a subtree, in all 27 mixes,
    and every evaluation order of three subtrees."""
    X = synth.tok(synth.VAR, 0)
    Cc = synth.const_tokens(0.75)
    sub = [synth.SUB, X, *synth.const_tokens(0.5)]          # needs one level
    deep = [synth.MUL, *sub, synth.ADD, X, *sub]            # needs two levels
    parts = {"X": [X], "C": Cc, "S": sub, "D": deep}
    x = synth.uniform_cases(87, 1, 33, -2.0, 2.0)
    x[0, :3] = np.array([0.5, 0.0, np.nan], np.float32)
    import itertools
    seen = set()
    for combo in itertools.product("XCSD", repeat=3):
        p = np.array([synth.IF] + parts[combo[0]] + parts[combo[1]] + parts[combo[2]], np.uint32)
        for order in (gp.ORDER_PAPER, gp.ORDER_MIN_DEPTH):
            words, info = gp.encode_tree(p, gp.KIND_SFORM, order)
            seen.add(int(words[4 + 4 * (info["n_instr"] - 1)]))
            assert same_bits(ref.run_float(words, x), oracle.fset_outputs(p, x)), (combo, order)
    assert len(seen) >= 20



def _f32bits(v):
    return int(np.array(v, np.float32).view(np.uint32))


@pytest.mark.parametrize("order", [gp.ORDER_PAPER, gp.ORDER_MIN_DEPTH])
def test_constant_divisors_take_the_reciprocal_forms_inside_the_fast_range(order):
    """A division by a constant in [2^-50, 2^50] (and, for a constant
    numerator, a numerator in that range too) is encoded with the divisor's
    reciprocal, rounded to nearest, in payload c; any other constant divisor
    keeps the plain forms.  Every program still evaluates as the oracle's."""
    x = edge_cases(96, 67)
    recip_seen = plain_seen = 0
    for p in constant_divisor_trees():
        words, info = gp.encode_tree(p, gp.KIND_SFORM, order)
        (code, pa, pb, pc), = ref.instrs(words)[-1:]
        name = ref.SF_FORMS[(code >> 2) // ref.R]
        b = int(pb)
        in_range = ref.DIV_LO <= (b & 0x7FFFFFFF) <= ref.DIV_HI
        numer_const = name[0] == "C"
        want = in_range and (not numer_const or ref.DIV_LO <= (int(pa) & 0x7FFFFFFF) <= ref.DIV_HI)
        assert (name in ref.SF_RECIP) == want, (name, hex(b), hex(int(pa)))
        if want:
            recip_seen += 1
            assert pc == _f32bits(np.float32(1) / np.float32(bitsf32(b)))
        else:
            plain_seen += 1
            assert pc == 0
        assert same_bits(ref.run_float(words, x), oracle.tree_outputs(p, x))
    assert recip_seen >= 20 and plain_seen >= 20


def test_stack_levels_sform_below_rpn_and_min_depth_below_paper_order():
    """The stack-limit table's claims, tree by tree: the S-form never needs
    more stack levels than the RPN form of the same tree, and the
    Sethi-Ullman child order never more than the paper's left-to-right order
    (for both forms); on a population with deep trees the orders differ."""
    import ctypes
    L = gp.lib()
    progs = synth.ramped_half_and_half(71, 300, 2, 9, 511, funcs=synth.SHUTTLE_FUNCS, n_inputs=3,
                                       full_fallback_to_grow=True)

    def depth(p, kind, order):
        cap = 4 + 4 * p.size
        buf = np.zeros(cap, np.uint32)
        info = gp._ProgInfo()
        L.gp_encode_tree(p.ctypes.data_as(ctypes.c_void_p), p.size, kind, order,
                         buf.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(info))
        return info.max_depth

    strict = 0
    for p in progs:
        p = np.ascontiguousarray(p, np.uint32)
        d = {(k, o): depth(p, k, o) for k in (gp.KIND_SFORM, gp.KIND_RPN)
             for o in (gp.ORDER_PAPER, gp.ORDER_MIN_DEPTH)}
        for o in (gp.ORDER_PAPER, gp.ORDER_MIN_DEPTH):
            assert d[(gp.KIND_SFORM, o)] <= d[(gp.KIND_RPN, o)]
        for k in (gp.KIND_SFORM, gp.KIND_RPN):
            assert d[(k, gp.ORDER_MIN_DEPTH)] <= d[(k, gp.ORDER_PAPER)]
        strict += d[(gp.KIND_RPN, gp.ORDER_MIN_DEPTH)] < d[(gp.KIND_RPN, gp.ORDER_PAPER)]
    assert strict > 20
