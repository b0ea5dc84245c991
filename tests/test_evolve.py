"""The device-side encoder and the on-device generation loop.

* gp_encode_population_device writes exactly the host encoder's words (basic
  and extended S-form, both child orders, single terminals, many inputs) and
  marks malformed or oversized trees so that evaluation reports them.
* A run's generations equal the oracle's generations (tournament selection,
  subtree crossover and mutation on the same Philox4x32-10 draws) tree for
  tree and word for word; with classification fitness (exact counts) the
  fitness and therefore every later selection agree exactly too.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import gp_ops
import paper_1601_00221_gb300 as gp
from gpu_util import dev

pytestmark = pytest.mark.gpu


def device_encode(pop, order):
    import torch
    W = dev(pop.words.view(np.int32))
    O = dev(pop.offsets)
    L = dev(pop.lengths)
    out, off, ln = gp.encode_population_device(W, O, L, order)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32), off.cpu().numpy(), ln.cpu().numpy()


@pytest.mark.parametrize("order", [gp.ORDER_PAPER, gp.ORDER_MIN_DEPTH])
@pytest.mark.parametrize("funcs,n_inputs", [(synth.FLOAT_FUNCS, 1), (synth.SEXTIC_FUNCS, 1),
                                            (synth.SHUTTLE_FUNCS, 9), (synth.KDD_FUNCS, 41)])
def test_device_encoder_matches_host(order, funcs, n_inputs):
    progs = synth.ramped_half_and_half(200 + n_inputs, 300, 1, 8, 255, funcs=funcs, n_inputs=n_inputs,
                                       full_fallback_to_grow=True)
    progs += [np.array([synth.tok(synth.VAR, n_inputs - 1)], np.uint32),
              np.array(synth.const_tokens(0.75), np.uint32)]
    pop = synth.pack(progs)
    host = gp.encode_population(pop.words, pop.offsets, pop.lengths, gp.KIND_SFORM, order)
    out, off, ln = device_encode(pop, order)
    assert np.array_equal(ln, host.lengths)
    for p in range(pop.n):
        a = host.words[host.offsets[p]: host.offsets[p] + host.lengths[p]]
        b = out[off[p]: off[p] + ln[p]]
        assert np.array_equal(a, b), p


@pytest.mark.parametrize("order", [gp.ORDER_PAPER, gp.ORDER_MIN_DEPTH])
def test_device_encoder_constant_divisors(order):
    """Divisions by constants at and beyond the edges of the fast range: the
    device encoder chooses the reciprocal forms exactly where the host one
    does and writes the same reciprocal words."""
    from div_trees import constant_divisor_trees
    pop = synth.pack(constant_divisor_trees(1) + constant_divisor_trees(3))
    host = gp.encode_population(pop.words, pop.offsets, pop.lengths, gp.KIND_SFORM, order)
    out, off, ln = device_encode(pop, order)
    assert np.array_equal(ln, host.lengths)
    for p in range(pop.n):
        a = host.words[host.offsets[p]: host.offsets[p] + host.lengths[p]]
        b = out[off[p]: off[p] + ln[p]]
        assert np.array_equal(a, b), p


@pytest.mark.parametrize("order", [gp.ORDER_PAPER, gp.ORDER_MIN_DEPTH])
def test_device_encoder_at_the_node_limit(order):
    """Trees of exactly GP_DEVICE_ENCODE_MAX_NODES = 256 nodes: a chain of 255
    unary functions (255 instructions) and 85 nested IFs whose nested operand
    moves through the three positions beside inputs and constants; every
    word as the host encoder's."""
    x0, x1 = synth.tok(synth.VAR, 0), synth.tok(synth.VAR, 1)
    chain = [synth.SIN, synth.COS, synth.EXP, synth.LOG] * 64
    chain = np.array(chain[:255] + [x0], np.uint32)
    levels = []
    for k in range(85):  # operands of the k-th IF from the root; None: the nested IF
        leaf = [x0] if k % 2 else synth.const_tokens(0.5 + k)
        ops = [leaf, [x1], [x0]]
        ops[k % 3] = None
        levels.append(ops)
    words = [x1]
    for ops in reversed(levels):
        parts = [words if o is None else o for o in ops]
        words = [synth.IF] + parts[0] + parts[1] + parts[2]
    nest = np.array(words, np.uint32)
    progs = [chain, nest]
    pop = synth.pack(progs)
    host = gp.encode_population(pop.words, pop.offsets, pop.lengths, gp.KIND_SFORM, order)
    assert list(host.words[host.offsets + 2]) == [256, 256]
    out, off, ln = device_encode(pop, order)
    assert np.array_equal(ln, host.lengths)
    for p in range(pop.n):
        a = host.words[host.offsets[p]: host.offsets[p] + host.lengths[p]]
        b = out[off[p]: off[p] + ln[p]]
        assert np.array_equal(a, b), p


def test_device_encoder_marks_bad_trees():
    good = np.array([synth.ADD, synth.tok(synth.VAR, 0), synth.tok(synth.VAR, 0)], np.uint32)
    missing = np.array([synth.ADD, synth.tok(synth.VAR, 0)], np.uint32)
    trailing = np.array([synth.tok(synth.VAR, 0), synth.tok(synth.VAR, 0)], np.uint32)
    nand = np.array([synth.NAND, synth.tok(synth.VAR, 0), synth.tok(synth.VAR, 0)], np.uint32)
    big = np.array([synth.ADD] * 200 + [synth.tok(synth.VAR, 0)] * 201, np.uint32)  # 401 nodes
    pop = synth.pack([good, missing, trailing, nand, big, good])
    out, off, ln = device_encode(pop, gp.ORDER_MIN_DEPTH)
    kinds = out[off] & 0xFF
    assert list(kinds) == [gp.KIND_SFORM, 0, 0, 0, 0, gp.KIND_SFORM]
    import torch
    x = dev(np.linspace(-1, 1, 64, dtype=np.float32)[None, :])
    y = dev(np.zeros(64, np.float32))
    f = gp.eval_population(dev(out.view(np.int32)), dev(off), dev(ln), x, y).cpu().numpy()
    assert np.isfinite(f[[0, 5]]).all() and np.isnan(f[1:5]).all()
    assert gp.last_error() == 2


PARAMS = dict(tournament=7, p_crossover=0.95, p_mutation=0.2, mutation_depth=4, p_const=0.5,
              const_lo=-200.0, const_hi=200.0, max_nodes=255)


def oracle_params(funcs, n_inputs, **kw):
    p = dict(PARAMS, funcs=[int(f) for f in funcs], n_inputs=n_inputs)
    p.update(kw)
    return p


def evolve_params(pop_size, funcs, seed, fitness, **kw):
    p = dict(PARAMS)
    p.update(kw)
    return gp.EvolveParams.make(pop_size, list(funcs), max_nodes=p["max_nodes"],
                                tournament=p["tournament"], p_crossover=p["p_crossover"],
                                p_mutation=p["p_mutation"], mutation_depth=p["mutation_depth"],
                                p_const=p["p_const"], const_lo=p["const_lo"], const_hi=p["const_hi"],
                                seed=seed, config=gp.Config(0, 4, 128, 0, fitness))


@pytest.mark.parametrize("seed", [1, (5 << 32) | 77])
def test_generations_match_the_oracle(seed):
    """Shuttle-set trees, classification fitness (exact on both sides): five
    generations, every tree and every fitness value equal."""
    w = synth.shuttle_like_problem(seed=210, n_progs=48, n_cases=400, depth_hi=6, max_nodes=200)
    prm = evolve_params(48, synth.SHUTTLE_FUNCS, seed, gp.FITNESS_CLASS)
    X, Y = dev(w.cases), dev(w.targets)
    op = oracle_params(synth.SHUTTLE_FUNCS, 9)
    pop = [[int(t) for t in w.pop.program(p)] for p in range(w.pop.n)]

    def fitness(trees):
        pk = synth.pack([np.array(t, np.uint32) for t in trees])
        return oracle.fset_population_fitness(pk.words, pk.offsets, pk.lengths, w.cases, w.targets,
                                              oracle.FIT_CLASS)

    with gp.Evolver(prm, w.pop.words, w.pop.offsets, w.pop.lengths, X, Y) as ev:
        trees, fit, g = ev.read()
        exp_fit = fitness(pop)
        assert g == 0 and np.array_equal(fit, exp_fit)
        for gen in range(1, 6):
            ev.run(1)
            trees, fit, g = ev.read()
            pop = gp_ops.generation(pop, exp_fit, gen, seed, op)
            exp_fit = fitness(pop)
            assert g == gen
            for i in range(len(pop)):
                assert trees[i].tolist() == pop[i], (gen, i)
            assert np.array_equal(fit, exp_fit), gen


def test_regression_run_is_consistent():
    """A larger run (1024 quartic-regression trees, sum of absolute errors,
    20 generations): the population after the run, encoded on the host and
    evaluated with the same configuration, has exactly the run's fitness, and
    every tree respects the size cap."""
    w = synth.regression_small(seed=211, n_progs=1024, n_cases=4096)
    cfg = gp.Config(gp.VARIANT_REGISTER, 8, 128, 0, gp.FITNESS_SUM_ABS)
    prm = gp.EvolveParams.make(1024, list(synth.FLOAT_FUNCS), max_nodes=127, seed=9, config=cfg)
    X, Y = dev(w.cases), dev(w.targets)
    with gp.Evolver(prm, w.pop.words, w.pop.offsets, w.pop.lengths, X, Y) as ev:
        n0 = ev.nodes_evaluated()
        assert n0 == int(w.pop.nodes.sum())
        ev.run(20)
        trees, fit, g = ev.read()
        assert ev.nodes_evaluated() > n0 + 19 * 1024
    assert g == 20
    assert all(len(gp_ops.node_starts([int(t) for t in tr])) <= 127 for tr in trees)
    pk = synth.pack(trees)
    enc = gp.encode_population(pk.words, pk.offsets, pk.lengths)
    P, O, L = enc.to_device("cuda")
    again = gp.eval_population(P, O, L, X, Y, config=cfg).cpu().numpy()
    assert np.array_equal(again.view(np.uint64), fit.view(np.uint64))
    exp = oracle.population_fitness(pk.words, pk.offsets, pk.lengths, w.cases, w.targets)
    fin = np.isfinite(exp) & (exp != 0)
    assert np.all(np.abs(fit[fin] - exp[fin]) <= 1e-5 * np.abs(exp[fin]))


def test_run_rejects_malformed_initial_trees():
    import torch
    good = np.array([synth.ADD, synth.tok(synth.VAR, 0), synth.tok(synth.VAR, 0)], np.uint32)
    bad_sets = [
        [synth.ADD, synth.tok(synth.VAR, 0)],                          # missing operand
        [synth.tok(synth.VAR, 0), synth.tok(synth.VAR, 0)],            # trailing tokens
        [synth.NAND, synth.tok(synth.VAR, 0), synth.tok(synth.VAR, 0)],  # not a float function
        [synth.CONST],                                                # constant without its value
    ]
    x = dev(np.zeros((1, 8), np.float32))
    y = dev(np.zeros(8, np.float32))
    for bad in bad_sets:
        pop = synth.pack([good, np.array(bad, np.uint32), good])
        prm = gp.EvolveParams.make(3, list(synth.FLOAT_FUNCS), seed=1)
        with pytest.raises(gp.GPError) as e:
            gp.Evolver(prm, pop.words, pop.offsets, pop.lengths, x, y)
        assert e.value.code == 2


@pytest.mark.parametrize("n", [1, 7, 1024, 1025, 5000])
def test_slot_offsets_are_the_packed_layout(n):
    """gp_encode_slots_device: out_offsets[p] = sum over q < p of
    4 + 4 * max(lengths[q], 0), also with zero and negative lengths (a
    malformed tree gets a header-only slot) and counts that do not fill the
    scan's 1024 threads evenly."""
    import torch
    rng = np.random.default_rng(n)
    ln = rng.integers(-3, 600, n).astype(np.int32)
    got = gp.encode_slots_device(dev(ln)).cpu().numpy()
    slot = 4 + 4 * np.maximum(ln.astype(np.int64), 0)
    want = np.concatenate([[0], np.cumsum(slot)[:-1]]).astype(np.int64)
    torch.cuda.synchronize()
    assert np.array_equal(got, want)
