"""GPU parity of the Boolean interpreter with a warp per program
(GP_VARIANT_WARPS: several programs per block over one staged copy of the
case set): hit counts and output words bit-exact against the CPU oracle."""
import numpy as np
import pytest

import oracle
import synth
import paper_1601_00221_gb300 as gp
from gpu_util import dev, upload

pytestmark = pytest.mark.gpu

ALL_ONES = np.uint64(0xFFFFFFFFFFFFFFFF)


def _workload(kind, k_inputs, n_progs, seed=3, n_cases=None):
    w = synth.boolean_problem(kind, k_inputs, seed=seed, n_progs=n_progs)
    if n_cases is None:
        return w
    nw = (n_cases + 31) // 32
    cb = np.ascontiguousarray(w.case_bits[:, :nw])
    tb = np.ascontiguousarray(w.target_bits[:nw])
    return synth.BooleanWorkload(w.name, w.pop, cb, tb, n_cases)


def _eval(w, cfg, out=False):
    import torch
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_BOOL,
                               gp.ORDER_MIN_DEPTH)
    P, O, L = upload(enc)
    cb = dev(w.case_bits.view(np.int32))
    tb = dev(w.target_bits.view(np.int32))
    hits = gp.eval_population_bool(P, O, L, cb, w.n_cases, tb, config=cfg).cpu().numpy().view(np.uint64)
    if not out:
        return hits, None
    nw = (w.n_cases + 31) // 32
    words = torch.zeros((w.pop.n, nw), dtype=torch.int32, device="cuda")
    gp.eval_population_bool(P, O, L, cb, w.n_cases, tb, hits_out=None, out_words=words, config=cfg)
    return hits, words.cpu().numpy().view(np.uint32)


def _expected(w):
    return oracle.bool_population_hits(w.pop.words, w.pop.offsets, w.pop.lengths, w.case_bits,
                                       w.n_cases, w.target_bits)


def _check_words(w, words, step):
    for p in range(0, w.pop.n, step):
        exp = oracle.bool_outputs(w.pop.program(p), w.case_bits)
        if w.n_cases % 32:
            m = np.uint32((1 << (w.n_cases % 32)) - 1)
            assert np.array_equal(words[p][:-1], exp[:-1]) and (words[p][-1] & m) == (exp[-1] & m), p
        else:
            assert np.array_equal(words[p], exp), p


@pytest.mark.parametrize("kind,k_inputs", [("parity", 11), ("mux", 11), ("parity", 9), ("parity", 13)])
@pytest.mark.parametrize("k", [1, 2, 4, 8])
@pytest.mark.parametrize("block", [64, 256])
def test_warps_variant_problems(kind, k_inputs, k, block):
    """16, 64 and 256 words: one pass (k words per lane cover the set) or
    several (k = 1 and 2 at 256 words); every program's hits exact."""
    w = _workload(kind, k_inputs, 300)
    hits, words = _eval(w, gp.Config(gp.VARIANT_WARPS, k, block, 0), out=(block == 64))
    assert np.array_equal(hits, _expected(w))
    if words is not None:
        _check_words(w, words, 23)


@pytest.mark.parametrize("n_cases", [129, 200, 1000, 2047, 2049, 3000])
@pytest.mark.parametrize("k", [1, 2, 8])
def test_warps_ragged_case_counts(n_cases, k):
    """A ragged last word and a ragged last pass: bits past n_cases never
    count, the padded words of the staged set are zero."""
    w = _workload("parity", 12, 97, seed=141, n_cases=n_cases)
    hits, words = _eval(w, gp.Config(gp.VARIANT_WARPS, k, 128, 0), out=True)
    assert np.array_equal(hits, _expected(w))
    _check_words(w, words, 11)


def test_warps_chosen_automatically():
    """Up to 256 words go to the per-warp kernel by default; the result is the
    oracle's either way, and equals the forced variant's and the register
    variant's."""
    for k_inputs in (5, 6, 8, 11, 13):  # 1 to 256 words
        w = _workload("parity", k_inputs, 150, seed=150 + k_inputs)
        auto, _ = _eval(w, None)
        forced, _ = _eval(w, gp.Config(gp.VARIANT_WARPS, 0, 0, 0))
        blocks, _ = _eval(w, gp.Config(gp.VARIANT_REGISTER, 2, 64, 0))
        exp = _expected(w)
        assert np.array_equal(auto, exp) and np.array_equal(forced, exp) and np.array_equal(blocks, exp)


@pytest.mark.parametrize("n_progs", [1, 7, 9, 33])
def test_warps_partial_last_block(n_progs):
    """Populations that do not fill the last block's warps."""
    w = _workload("mux", 11, n_progs, seed=160 + n_progs)
    hits, _ = _eval(w, gp.Config(gp.VARIANT_WARPS, 2, 256, 0))
    assert np.array_equal(hits, _expected(w))


def test_warps_malformed_program():
    """An unknown code in one program: its hits are all ones and the status
    reports a program error; the programs beside it in the block are exact."""
    w = _workload("mux", 11, 16, seed=170)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_BOOL)
    words = enc.words.copy()
    words[int(enc.offsets[5]) + 4] = 9999
    gp.last_error()
    hits = gp.eval_population_bool(dev(words.view(np.int32)), dev(enc.offsets), dev(enc.lengths),
                                   dev(w.case_bits.view(np.int32)), w.n_cases,
                                   dev(w.target_bits.view(np.int32)),
                                   config=gp.Config(gp.VARIANT_WARPS, 2, 128, 0)).cpu().numpy().view(np.uint64)
    assert gp.last_error() == 2
    exp = _expected(w)
    assert hits[5] == ALL_ONES
    others = np.arange(w.pop.n) != 5
    assert np.array_equal(hits[others], exp[others])


def test_warps_program_longer_than_the_buffer():
    """max_instructions below the longest program: those programs are
    reported malformed, the rest are exact."""
    w = _workload("mux", 11, 200, seed=180)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_BOOL)
    n_instr = enc.info["n_instr"]
    cap = int(n_instr.max()) - 1
    P, O, L = upload(enc)
    gp.last_error()
    hits = gp.eval_population_bool(P, O, L, dev(w.case_bits.view(np.int32)), w.n_cases,
                                   dev(w.target_bits.view(np.int32)),
                                   config=gp.Config(gp.VARIANT_WARPS, 2, 128, 0, 0, 0, 0, cap)
                                   ).cpu().numpy().view(np.uint64)
    over = n_instr > cap
    exp = _expected(w)
    assert over.sum() >= 1 and np.all(hits[over] == ALL_ONES)
    assert np.array_equal(hits[~over], exp[~over])
    assert gp.last_error() == 2


def test_warps_no_cases_and_too_large():
    """No cases: every program scores 0.  A case set larger than the shared
    memory the variant may use is an argument error, raised before any
    launch."""
    w = _workload("parity", 11, 40, seed=190)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_BOOL)
    P, O, L = upload(enc)
    cb = dev(w.case_bits.view(np.int32))
    tb = dev(w.target_bits.view(np.int32))
    hits = gp.eval_population_bool(P, O, L, cb, 0, tb, config=gp.Config(gp.VARIANT_WARPS, 2, 128, 0))
    assert np.all(hits.cpu().numpy() == 0)
    big = _workload("parity", 20, 4, seed=191)  # 32768 words x 20 inputs
    enc = gp.encode_population(big.pop.words, big.pop.offsets, big.pop.lengths, gp.KIND_BOOL)
    P, O, L = upload(enc)
    with pytest.raises(gp.GPError) as e:
        gp.eval_population_bool(P, O, L, dev(big.case_bits.view(np.int32)), big.n_cases,
                                dev(big.target_bits.view(np.int32)), config=gp.Config(gp.VARIANT_WARPS, 8, 128, 0))
    assert e.value.code == 1  # GP_ERR_INVALID_ARG


def test_warps_known_correct_programs():
    """The 11-input even-parity and multiplexer programs built from the
    definitions score every case."""
    from test_oracle_pins import even_parity_program_if, mux_program_if
    for make, target in ((even_parity_program_if, synth.even_parity_target),
                         (mux_program_if, synth.mux_target)):
        pop = synth.pack([np.array(make(11), np.uint32)] * 3)
        w = synth.BooleanWorkload("k", pop, synth.bool_case_bits(11), target(11), 1 << 11)
        for k in (1, 2):
            hits, _ = _eval(w, gp.Config(gp.VARIANT_WARPS, k, 64, 0))
            assert np.all(hits == np.uint64(1 << 11))


@pytest.mark.parametrize("variant,k,block", [(gp.VARIANT_WARPS, 2, 128), (gp.VARIANT_WARPS, 1, 64),
                                             (gp.VARIANT_REGISTER, 4, 64)])
def test_case_bits_not_16_byte_aligned(variant, k, block):
    """Case bits and targets that start one word past a 16-byte boundary (the
    staging then loads word by word): hits exact for the per-warp and the
    block kernels."""
    import torch
    w = _workload("mux", 11, 120, seed=200)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_BOOL)
    P, O, L = upload(enc)
    nin, nw = w.case_bits.shape
    buf = torch.zeros(nin * nw + 1, dtype=torch.int32, device="cuda")
    buf[1:] = torch.from_numpy(w.case_bits.reshape(-1).view(np.int32)).cuda()
    cb = buf[1:].view(nin, nw)
    tbuf = torch.zeros(nw + 1, dtype=torch.int32, device="cuda")
    tbuf[1:] = torch.from_numpy(w.target_bits.view(np.int32)).cuda()
    tb = tbuf[1:]
    assert cb.data_ptr() % 16 != 0 and tb.data_ptr() % 16 != 0
    hits = gp.eval_population_bool(P, O, L, cb, w.n_cases, tb, config=gp.Config(variant, k, block, 0))
    assert np.array_equal(hits.cpu().numpy().view(np.uint64), _expected(w))
