"""GPU parity of the bit-packed Boolean interpreter: hit counts and output
words bit-exact against the CPU oracle."""
import numpy as np
import pytest

import oracle
import synth
import paper_1601_00221_gb300 as gp
from gpu_util import dev, upload
from synth import AND, OR, NAND, NOR, IF, VAR, tok

pytestmark = pytest.mark.gpu

PROBLEMS = [("parity", 6), ("mux", 6), ("parity", 11), ("mux", 11)]


def run(w, k, block=0, n_cases=None, words=None):
    n_cases = w.n_cases if n_cases is None else n_cases
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_BOOL,
                               gp.ORDER_MIN_DEPTH)
    P, O, L = upload(enc)
    cb = dev(w.case_bits.view(np.int32))
    tb = dev(w.target_bits.view(np.int32))
    cfg = gp.Config(gp.VARIANT_REGISTER, k, block, 0)
    hits = gp.eval_population_bool(P, O, L, cb, n_cases, tb, config=cfg).cpu().numpy()
    import torch
    nw = (n_cases + 31) // 32
    out = torch.zeros((w.pop.n, nw), dtype=torch.int32, device="cuda")
    gp.eval_population_bool(P, O, L, cb, n_cases, tb, hits_out=None, out_words=out, config=cfg)
    return hits.astype(np.uint64), out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("kind,k_inputs", PROBLEMS)
@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_boolean_problems(kind, k_inputs, k):
    w = synth.boolean_problem(kind, k_inputs, n_progs=512)
    hits, out = run(w, k)
    exp = oracle.bool_population_hits(w.pop.words, w.pop.offsets, w.pop.lengths, w.case_bits,
                                      w.n_cases, w.target_bits)
    assert np.array_equal(hits, exp)
    for p in range(0, w.pop.n, 17):
        assert np.array_equal(out[p], oracle.bool_outputs(w.pop.program(p), w.case_bits))


def test_known_correct_programs_score_all_hits():
    from test_oracle_pins import even_parity_program, even_parity_program_if, mux_program_if
    for k_inputs in (6, 11):
        make = even_parity_program if k_inputs == 6 else even_parity_program_if
        progs = [np.array(make(k_inputs), np.uint32)]
        pop = synth.pack(progs)
        w = synth.BooleanWorkload("p", pop, synth.bool_case_bits(k_inputs),
                                  synth.even_parity_target(k_inputs), 1 << k_inputs)
        hits, _ = run(w, 2)
        assert hits[0] == 1 << k_inputs
        pop = synth.pack([np.array(mux_program_if(k_inputs), np.uint32)])
        w = synth.BooleanWorkload("m", pop, synth.bool_case_bits(k_inputs),
                                  synth.mux_target(k_inputs), 1 << k_inputs)
        hits, _ = run(w, 2)
        assert hits[0] == 1 << k_inputs


@pytest.mark.parametrize("n_cases", [1, 5, 31, 33, 100, 1000])
def test_ragged_case_counts(n_cases):
    """Cases that do not fill the last word: the unused bits never count."""
    k_inputs = 10
    w = synth.boolean_problem("parity", k_inputs, seed=81, n_progs=64)
    nw = (n_cases + 31) // 32
    cb = np.ascontiguousarray(w.case_bits[:, :nw])
    tb = np.ascontiguousarray(w.target_bits[:nw])
    w2 = synth.BooleanWorkload("r", w.pop, cb, tb, n_cases)
    for k in (1, 4):
        hits, out = run(w2, k, n_cases=n_cases)
        exp = oracle.bool_population_hits(w.pop.words, w.pop.offsets, w.pop.lengths, cb, n_cases, tb)
        assert np.array_equal(hits, exp)


def test_large_multiplexer_sampled():
    """20-multiplexer shape of the paper (2^20 cases = 32768 words)."""
    w = synth.boolean_problem("mux", 20, n_progs=256)
    hits, _ = run(w, 4)
    for p in range(0, 256, 16):
        exp = oracle.bool_hits(w.pop.program(p), w.case_bits, w.n_cases, w.target_bits)
        assert hits[p] == exp


def test_malformed_bool_program():
    w = synth.boolean_problem("mux", 6, n_progs=4)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_BOOL)
    words = enc.words.copy()
    words[int(enc.offsets[1]) + 4] = 9999
    P = dev(words.view(np.int32))
    gp.last_error()
    hits = gp.eval_population_bool(P, dev(enc.offsets), dev(enc.lengths),
                                   dev(w.case_bits.view(np.int32)), w.n_cases,
                                   dev(w.target_bits.view(np.int32))).cpu().numpy().view(np.uint64)
    assert hits[1] == np.uint64(0xFFFFFFFFFFFFFFFF)
    assert gp.last_error() == 2


@pytest.mark.parametrize("kind,k_inputs", [("parity", 5), ("mux", 6), ("parity", 6), ("parity", 7)])
def test_program_per_lane_variant(kind, k_inputs):
    """Tiny case sets (<= 4 words): one program per lane, bit-exact hits and words."""
    if kind == "mux":
        w = synth.boolean_problem(kind, k_inputs, seed=121, n_progs=1000)
    else:
        progs = synth.ramped_half_and_half(122 + k_inputs, 1000, 2, 8, 256,
                                           funcs=synth.BOOL_FUNCS + (IF,), n_inputs=k_inputs,
                                           p_const=0.0, full_fallback_to_grow=True)
        w = synth.BooleanWorkload("p", synth.pack(progs), synth.bool_case_bits(k_inputs),
                                  synth.even_parity_target(k_inputs), 1 << k_inputs)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_BOOL)
    P, O, L = upload(enc)
    cb = dev(w.case_bits.view(np.int32))
    tb = dev(w.target_bits.view(np.int32))
    import torch
    nw = (w.n_cases + 31) // 32
    for cfg in (gp.Config(gp.VARIANT_LANES, 0, 0, 0), None):  # forced, and chosen automatically
        hits = gp.eval_population_bool(P, O, L, cb, w.n_cases, tb, config=cfg).cpu().numpy()
        exp = oracle.bool_population_hits(w.pop.words, w.pop.offsets, w.pop.lengths, w.case_bits,
                                          w.n_cases, w.target_bits)
        assert np.array_equal(hits.astype(np.uint64), exp)
        out = torch.zeros((w.pop.n, nw), dtype=torch.int32, device="cuda")
        gp.eval_population_bool(P, O, L, cb, w.n_cases, tb, hits_out=None, out_words=out, config=cfg)
        out = out.cpu().numpy().view(np.uint32)
        for p in range(0, w.pop.n, 37):
            exp_w = oracle.bool_outputs(w.pop.program(p), w.case_bits)
            if w.n_cases % 32:
                m = np.uint32((1 << (w.n_cases % 32)) - 1)
                assert np.array_equal(out[p][:-1], exp_w[:-1]) and (out[p][-1] & m) == (exp_w[-1] & m)
            else:
                assert np.array_equal(out[p], exp_w)


@pytest.mark.parametrize("n_cases", [1, 17, 32, 33, 64, 100, 128])
def test_program_per_lane_ragged(n_cases):
    w = synth.boolean_problem("parity", 7, seed=123, n_progs=300)
    nw = (n_cases + 31) // 32
    cb = np.ascontiguousarray(w.case_bits[:, :nw])
    tb = np.ascontiguousarray(w.target_bits[:nw])
    w2 = synth.BooleanWorkload("r", w.pop, cb, tb, n_cases)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_BOOL)
    P, O, L = upload(enc)
    hits = gp.eval_population_bool(P, O, L, dev(cb.view(np.int32)), n_cases, dev(tb.view(np.int32)),
                                   config=gp.Config(gp.VARIANT_LANES, 0, 0, 0)).cpu().numpy()
    exp = oracle.bool_population_hits(w.pop.words, w.pop.offsets, w.pop.lengths, cb, n_cases, tb)
    assert np.array_equal(hits.astype(np.uint64), exp)


@pytest.mark.parametrize("k", [2, 8])
def test_program_buffer_sized_to_the_population(k):
    """gp_config.max_instructions: with the population's largest instruction
    count the hits equal those with the full program buffer, and the oracle's;
    a program longer than the buffer is reported malformed, the others are
    unaffected."""
    w = synth.boolean_problem("mux", 11, n_progs=400)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_BOOL)
    P, O, L = upload(enc)
    cb, tb = dev(w.case_bits.view(np.int32)), dev(w.target_bits.view(np.int32))
    n_instr = enc.info["n_instr"]
    exp = oracle.bool_population_hits(w.pop.words, w.pop.offsets, w.pop.lengths, w.case_bits,
                                      w.n_cases, w.target_bits)
    full = gp.eval_population_bool(P, O, L, cb, w.n_cases, tb,
                                   config=gp.Config(gp.VARIANT_REGISTER, k, 64, 0)).cpu().numpy()
    tight = gp.eval_population_bool(P, O, L, cb, w.n_cases, tb,
                                    config=gp.Config(gp.VARIANT_REGISTER, k, 64, 0, 0, 0, 0,
                                                     enc.max_instructions)).cpu().numpy()
    assert np.array_equal(full.view(np.uint64), exp) and np.array_equal(tight.view(np.uint64), exp)
    cap = int(n_instr.max()) - 1  # the longest programs no longer fit
    gp.last_error()
    short = gp.eval_population_bool(P, O, L, cb, w.n_cases, tb,
                                    config=gp.Config(gp.VARIANT_REGISTER, k, 64, 0, 0, 0, 0, cap)
                                    ).cpu().numpy().view(np.uint64)
    over = n_instr > cap
    assert over.sum() >= 1 and np.all(short[over] == np.uint64(0xFFFFFFFFFFFFFFFF))
    assert np.array_equal(short[~over], exp[~over])
    assert gp.last_error() == 2


@pytest.mark.parametrize("k,block", [(4, 128), (2, 64), (8, 32)])
def test_input_listing_matches_the_oracle(k, block):
    """Blocks of at least four passes stage only the inputs their tree reads
    (payloads rewritten to slots); blocks of fewer stage every input.  Trees
    over 16 inputs that each read a few of them, at a chunk of eight passes
    (listed) and of one pass (every input): both give the oracle's hits and
    output words."""
    import torch
    progs = synth.ramped_half_and_half(190 + k, 200, 2, 6, 63, funcs=synth.BOOL_FUNCS + (IF,),
                                       n_inputs=16, p_const=0.0, full_fallback_to_grow=True)
    pop = synth.pack(progs)
    n_cases = 1 << 16
    w = synth.BooleanWorkload("l", pop, synth.bool_case_bits(16), synth.even_parity_target(16), n_cases)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_BOOL)
    P, O, L = upload(enc)
    cb, tb = dev(w.case_bits.view(np.int32)), dev(w.target_bits.view(np.int32))
    exp = oracle.bool_population_hits(w.pop.words, w.pop.offsets, w.pop.lengths, w.case_bits,
                                      w.n_cases, w.target_bits)
    nw = n_cases // 32
    for passes in (8, 1):
        cfg = gp.Config(gp.VARIANT_REGISTER, k, block, passes * k * block, 0, 0, 0, enc.max_instructions)
        hits = gp.eval_population_bool(P, O, L, cb, n_cases, tb, config=cfg).cpu().numpy()
        assert np.array_equal(hits.astype(np.uint64), exp), passes
        out = torch.zeros((w.pop.n, nw), dtype=torch.int32, device="cuda")
        gp.eval_population_bool(P, O, L, cb, n_cases, tb, hits_out=None, out_words=out, config=cfg)
        out = out.cpu().numpy().view(np.uint32)
        for p in range(0, w.pop.n, 29):
            assert np.array_equal(out[p], oracle.bool_outputs(w.pop.program(p), w.case_bits)), (passes, p)
