"""GPU parity of the binary32 interpreters against the CPU oracle.

Per-case outputs must match bit for bit (any NaN equals any NaN); fitness must
lie within 1e-5 relative of the binary64 oracle (exactly equal when the oracle
gives 0 or +inf).  Calls go through the C ABI (ctypes binding).
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1601_00221_gb300 as gp
from gpu_util import dev, upload, assert_bits, assert_fitness, oracle_outputs, rel_errors
from synth import ADD, SUB, MUL, DIV, VAR, tok, const_tokens

pytestmark = pytest.mark.gpu

KS = [1, 2, 4, 8]


@pytest.fixture(scope="module")
def small():
    w = synth.regression_small()  # 256 trees, depth 2-6, 1024 cases
    x = w.cases.copy()
    x[0, :4] = [0.0, -0.0, 1e-40, -1.0]  # protected division and subnormals
    y = synth.quartic_target(x[0])
    ref = oracle_outputs(w.pop, x)
    fit = oracle.population_fitness(w.pop.words, w.pop.offsets, w.pop.lengths, x, y)
    return w, x, y, ref, fit


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("kind", [gp.KIND_SFORM, gp.KIND_RPN])
@pytest.mark.parametrize("order", [gp.ORDER_PAPER, gp.ORDER_MIN_DEPTH])
def test_small_regression_all_k(small, k, kind, order):
    w, x, y, ref, fit = small
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, kind, order)
    P, O, L = upload(enc)
    X, Y = dev(x), dev(y)
    for block in (32, 128):
        cfg = gp.Config(gp.VARIANT_REGISTER, k, block, 0)
        out = gp.eval_outputs(P, O, L, X, config=cfg)
        assert_bits(out.cpu().numpy(), ref, f"outputs k={k} block={block}")
        f = gp.eval_population(P, O, L, X, Y, config=cfg)
        assert_fitness(f.cpu().numpy(), fit, f"fitness k={k} block={block}")
    assert gp.last_error() == 0


def test_blockgp_local_stack(small):
    w, x, y, ref, fit = small
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_RPN,
                               gp.ORDER_PAPER)
    P, O, L = upload(enc)
    cfg = gp.Config(gp.VARIANT_LOCAL, 1, 256, 0)
    out = gp.eval_outputs(P, O, L, dev(x), config=cfg)
    assert_bits(out.cpu().numpy(), ref, "blockgp outputs")
    f = gp.eval_population(P, O, L, dev(x), dev(y), config=cfg)
    assert_fitness(f.cpu().numpy(), fit, "blockgp fitness")


@pytest.mark.parametrize("n_cases", [0, 1, 3, 31, 1000, 1027, 4099])
@pytest.mark.parametrize("k", [1, 4, 8])
def test_ragged_case_counts_and_chunks(n_cases, k):
    w = synth.regression_small(seed=71, n_progs=40, n_cases=max(n_cases, 1))
    x = w.cases[:, :n_cases].copy()
    y = synth.quartic_target(x[0])
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths)
    P, O, L = upload(enc)
    # small chunks force many blocks per program and the fused cross-block sum
    for chunk in (0, 64 * k):
        cfg = gp.Config(gp.VARIANT_REGISTER, k, 64, chunk)
        f = gp.eval_population(P, O, L, dev(x), dev(y), config=cfg).cpu().numpy()
        exp = oracle.population_fitness(w.pop.words, w.pop.offsets, w.pop.lengths, x, y)
        assert_fitness(f, exp, f"n_cases={n_cases} chunk={chunk}")
        if n_cases:
            out = gp.eval_outputs(P, O, L, dev(x), config=cfg).cpu().numpy()
            assert_bits(out, oracle_outputs(w.pop, x), f"outputs n_cases={n_cases}")


@pytest.mark.parametrize("k", KS)
def test_multi_input_programs(k):
    progs = synth.ramped_half_and_half(72, 96, 2, 7, 127, n_inputs=5)
    progs.append(np.array([tok(VAR, 4)], np.uint32))
    progs.append(np.array(const_tokens(-0.375), np.uint32))
    pop = synth.pack(progs)
    x = synth.uniform_cases(73, 5, 2053)
    y = synth.uniform_cases(74, 1, 2053)[0]
    for kind in (gp.KIND_SFORM, gp.KIND_RPN):
        enc = gp.encode_population(pop.words, pop.offsets, pop.lengths, kind, gp.ORDER_MIN_DEPTH)
        P, O, L = upload(enc)
        cfg = gp.Config(gp.VARIANT_REGISTER, k, 128, 0)
        out = gp.eval_outputs(P, O, L, dev(x), config=cfg).cpu().numpy()
        assert_bits(out, oracle_outputs(pop, x), f"multi-input kind={kind}")
        f = gp.eval_population(P, O, L, dev(x), dev(y), config=cfg).cpu().numpy()
        assert_fitness(f, oracle.population_fitness(pop.words, pop.offsets, pop.lengths, x, y))


def test_nonfinite_and_special_values():
    big = const_tokens(3e38)
    progs = [
        [tok(MUL)] + big + big,                               # +inf everywhere
        [tok(SUB), tok(MUL)] + big + big + [tok(MUL)] + big + big,  # NaN
        [tok(DIV), tok(VAR, 0), tok(VAR, 0)],                  # 1 everywhere (protected at 0)
        [tok(DIV)] + const_tokens(1.0) + [tok(VAR, 0)],        # 1/x: protected at +-0, +inf at 1e-45
        [tok(SUB), tok(VAR, 0), tok(VAR, 0)],
        list(synth.quartic_program()),
    ]
    pop = synth.pack([np.array(p, np.uint32) for p in progs])
    x = synth.uniform_cases(75, 1, 777)
    x[0, :5] = [0.0, -0.0, 1e-45, -1e-45, 3.4e38]
    y = synth.quartic_target(x[0])
    exp_out = oracle_outputs(pop, x)
    exp_fit = oracle.population_fitness(pop.words, pop.offsets, pop.lengths, x, y)
    assert np.isinf(exp_fit[0]) and np.isinf(exp_fit[1])
    for k in KS:
        enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
        P, O, L = upload(enc)
        cfg = gp.Config(gp.VARIANT_REGISTER, k, 64, 0)
        assert_bits(gp.eval_outputs(P, O, L, dev(x), config=cfg).cpu().numpy(), exp_out, f"k={k}")
        f = gp.eval_population(P, O, L, dev(x), dev(y), config=cfg).cpu().numpy()
        assert_fitness(f, exp_fit, f"k={k}")


@pytest.mark.parametrize("fitness", [gp.FITNESS_SUM_ABS, gp.FITNESS_MSE])
def test_error_sum_past_binary32_is_inf(fitness):
    """Every per-case error finite, their sum beyond binary32 (reading r29):
    the fitness is +inf, whether the sum overflows inside a pass, across the
    passes of a thread or across blocks.  The binary64 oracle's value is
    finite there; it is checked to be beyond the binary32 range."""
    c = 2e38 if fitness == gp.FITNESS_SUM_ABS else 1.5e19   # error 2e38 (or its square 2.25e38)
    progs = [np.array(const_tokens(c), np.uint32), np.array(synth.quartic_program(), np.uint32)]
    pop = synth.pack(progs)
    for n_cases in (2, 40, 5000):
        x = synth.uniform_cases(76, 1, n_cases)
        y = np.zeros(n_cases, np.float32)
        exp = oracle.fset_population_fitness(pop.words, pop.offsets, pop.lengths, x, y,
                                             oracle.FIT_MSE if fitness == gp.FITNESS_MSE else oracle.FIT_ABS)
        assert np.isfinite(exp[0]) and exp[0] * (n_cases if fitness == gp.FITNESS_MSE else 1) > 3.5e38
        for k in KS:
            enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
            P, O, L = upload(enc)
            for chunk in (0, 32 * k):
                cfg = gp.Config(gp.VARIANT_REGISTER, k, 32, chunk, fitness)
                f = gp.eval_population(P, O, L, dev(x), dev(y), config=cfg).cpu().numpy()
                assert f[0] == np.inf, (n_cases, k, chunk, f[0])
                assert np.isfinite(f[1]) and abs(f[1] - exp[1]) <= 1e-5 * abs(exp[1]), (n_cases, k, chunk)


@pytest.mark.parametrize("chunk_per_pass", [8, 40])
def test_block_order_changes_nothing(chunk_per_pass):
    """Populations of at least two programs per SM are taken longest first
    (a counting sort of the instruction counts on the device).  1200 trees of
    1 to 255 nodes (many of equal size, a few identical): every fitness equals
    the same programs evaluated 100 at a time (too few to be reordered) bit for
    bit, and the oracle's within the bound; with several chunks per program the
    cross-block sums stay in chunk order.  (The chunk is given: a chosen one
    depends on the population's size, and with it the summation order.)"""
    progs = synth.ramped_half_and_half(313, 1200, 1, 8, 255, full_fallback_to_grow=True)
    progs[700] = progs[3]
    pop = synth.pack(progs)
    x = synth.uniform_cases(77, 1, 20000)   # (enough cases per program to be ordered)
    y = synth.quartic_target(x[0])
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    P, O, L = upload(enc)
    k, block = 8, 64
    cfg = gp.Config(gp.VARIANT_REGISTER, k, block, chunk_per_pass * k * block)
    f_all = gp.eval_population(P, O, L, dev(x), dev(y), config=cfg).cpu().numpy()
    parts = []
    for i in range(0, pop.n, 100):
        sub = synth.pack(progs[i:i + 100])
        e2 = gp.encode_population(sub.words, sub.offsets, sub.lengths)
        P2, O2, L2 = upload(e2)
        parts.append(gp.eval_population(P2, O2, L2, dev(x), dev(y), config=cfg).cpu().numpy())
    f_parts = np.concatenate(parts)
    assert np.array_equal(f_all.view(np.uint64), f_parts.view(np.uint64))
    assert f_all[700] == f_all[3]
    assert_fitness(f_all, oracle.population_fitness(pop.words, pop.offsets, pop.lengths, x, y))
    # the 1200 were ordered (two launches), the groups of 100 were not
    assert gp.eval_launches(pop.n, 20000) == 2 and gp.eval_launches(100, 20000) == 1
    assert gp.eval_launches(pop.n, 2000) == 1


@pytest.mark.parametrize("variant,kind", [(gp.VARIANT_REGISTER, gp.KIND_SFORM), (gp.VARIANT_REGISTER, gp.KIND_RPN),
                                          (gp.VARIANT_LOCAL, gp.KIND_RPN)])
def test_program_buffer_sized_to_the_population(variant, kind):
    """gp_config.max_instructions: with the population's largest instruction
    count the fitness equals the full-buffer fitness bit for bit; a program
    longer than the buffer is reported malformed (NaN, status 2), the others
    are unaffected; values outside 0..GP_MAX_INSTR are rejected."""
    w = synth.regression_small(seed=317, n_progs=400, n_cases=4096)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, kind)
    P, O, L = upload(enc)
    X, Y = dev(w.cases), dev(w.targets)
    k = 1 if variant == gp.VARIANT_LOCAL else 8
    base = gp.Config(variant, k, 128, 0)
    full = gp.eval_population(P, O, L, X, Y, config=base).cpu().numpy()
    tight_cfg = gp.Config(variant, k, 128, 0, 0, 0, 0, enc.max_instructions)
    tight = gp.eval_population(P, O, L, X, Y, config=tight_cfg).cpu().numpy()
    assert np.array_equal(full.view(np.uint64), tight.view(np.uint64))
    n_instr = enc.info["n_instr"]
    cap = int(n_instr.max()) - 1
    gp.last_error()
    short = gp.eval_population(P, O, L, X, Y, config=gp.Config(variant, k, 128, 0, 0, 0, 0, cap)).cpu().numpy()
    over = n_instr > cap
    assert over.sum() >= 1 and np.isnan(short[over]).all()
    assert np.array_equal(short[~over].view(np.uint64), full[~over].view(np.uint64))
    assert gp.last_error() == 2
    for bad in (-1, 1025):
        with pytest.raises(gp.GPError):
            gp.eval_population(P, O, L, X, Y, config=gp.Config(variant, k, 128, 0, 0, 0, 0, bad))


def test_malformed_device_program_gives_nan_and_status():
    w = synth.regression_small(n_progs=8, n_cases=256)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths)
    words = enc.words.copy()
    o = int(enc.offsets[3])
    words[o + 4] = 0xFFFF          # unknown instruction code in program 3
    o5 = int(enc.offsets[5])
    words[o5 + 1] = 5000            # header claims more instructions than fit
    P = dev(words.view(np.int32))
    O, L = dev(enc.offsets), dev(enc.lengths)
    gp.last_error()  # clear
    f = gp.eval_population(P, O, L, dev(w.cases), dev(w.targets)).cpu().numpy()
    assert np.isnan(f[3]) and np.isnan(f[5])
    good = [p for p in range(8) if p not in (3, 5)]
    exp = oracle.population_fitness(w.pop.words, w.pop.offsets, w.pop.lengths, w.cases, w.targets)
    assert_fitness(f[good], exp[good])
    assert gp.last_error() == 2
    assert gp.last_error() == 0  # cleared by the read


def test_input_index_beyond_n_inputs_is_rejected_on_device():
    pop = synth.pack([np.array([tok(ADD), tok(VAR, 0), tok(VAR, 3)], np.uint32)])
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    P, O, L = upload(enc)
    x = synth.uniform_cases(76, 2, 64)   # only 2 inputs
    gp.last_error()
    f = gp.eval_population(P, O, L, dev(x), dev(x[0])).cpu().numpy()
    assert np.isnan(f[0])
    assert gp.last_error() == 2


@pytest.mark.parametrize("k", KS)
def test_register_linear_gp(k):
    w = synth.linear_workload(seed=77, n_progs=128, n_cases=4099)
    x = w.cases.copy()
    x[:, :2] = 0.0
    enc = gp.encode_linear_population(w.pop.instr, w.pop.offsets, w.pop.lengths)
    P, O, L = upload(enc)
    cfg = gp.Config(gp.VARIANT_REGISTER, k, 128, 0)
    out = gp.eval_outputs(P, O, L, dev(x), config=cfg).cpu().numpy()
    exp = np.stack([oracle.linear_outputs(w.pop.program(p), x) for p in range(w.pop.n)])
    assert_bits(out, exp, "linear outputs")
    f = gp.eval_population(P, O, L, dev(x), dev(w.targets), config=cfg).cpu().numpy()
    fit = oracle.linear_population_fitness(w.pop.instr, w.pop.offsets, w.pop.lengths, x, w.targets)
    assert_fitness(f, fit, "linear fitness")


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("n_inputs,n_cases", [(8, 4099), (3, 1000), (11, 2052), (8, 7)])
def test_register_file_in_shared_memory(k, n_inputs, n_cases):
    """The register-file variant (registers in shared memory, one jump per
    instruction): per-case outputs bit for bit and fitness against the
    oracle, with fewer inputs than registers (the rest start at 0), more
    (only the first eight are registers), ragged and unaligned case counts
    (the scalar staging path) and several chunks per program."""
    pop = synth.linear_programs(80 + n_inputs, 96, 1, 128)
    x = synth.normal_cases(81, n_inputs, n_cases)
    x[:, :2] = 0.0
    y = synth.normal_cases(82, 1, n_cases)[0]
    enc = gp.encode_linear_population(pop.instr, pop.offsets, pop.lengths)
    P, O, L = upload(enc)
    exp = np.stack([oracle.linear_outputs(pop.program(p), x) for p in range(pop.n)])
    fit = oracle.linear_population_fitness(pop.instr, pop.offsets, pop.lengths, x, y)
    for block, chunk in ((64, 0), (256, 0), (128, 128 * k)):
        cfg = gp.Config(gp.VARIANT_REGISTER_FILE, k, block, chunk)
        out = gp.eval_outputs(P, O, L, dev(x), config=cfg).cpu().numpy()
        assert_bits(out, exp, f"register file k={k} block={block}")
        f = gp.eval_population(P, O, L, dev(x), dev(y), config=cfg).cpu().numpy()
        assert_fitness(f, fit, f"register file k={k} block={block} chunk={chunk}")
    assert gp.last_error() == 0


def test_register_file_rejects_tree_programs():
    w = synth.regression_small(seed=83, n_progs=8, n_cases=100)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths)
    P, O, L = upload(enc)
    f = gp.eval_population(P, O, L, dev(w.cases), dev(w.targets),
                           config=gp.Config(gp.VARIANT_REGISTER_FILE, 4, 64, 0)).cpu().numpy()
    assert np.all(np.isnan(f))
    assert gp.last_error() == 2


def test_mixed_kinds_in_one_launch():
    w = synth.regression_small(seed=78, n_progs=30, n_cases=515)
    sf = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_SFORM)
    rp = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_RPN)
    words = np.concatenate([sf.words, rp.words])
    offs = np.concatenate([sf.offsets, rp.offsets + sf.words.size])
    lens = np.concatenate([sf.lengths, rp.lengths])
    P = dev(words.view(np.int32))
    f = gp.eval_population(P, dev(offs), dev(lens), dev(w.cases), dev(w.targets)).cpu().numpy()
    exp = oracle.population_fitness(w.pop.words, w.pop.offsets, w.pop.lengths, w.cases, w.targets)
    assert_fitness(f, np.concatenate([exp, exp]))
    assert np.array_equal(f[:30], f[30:])  # same order of summation for both kinds


def test_fitness_bit_identical_across_runs_and_streams():
    import torch
    w = synth.regression_small(seed=79, n_progs=64, n_cases=3000)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths)
    P, O, L = upload(enc)
    X, Y = dev(w.cases), dev(w.targets)
    f0 = gp.eval_population(P, O, L, X, Y).cpu().numpy()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        f1 = gp.eval_population(P, O, L, X, Y, stream=s)
    s.synchronize()
    assert np.array_equal(f0, f1.cpu().numpy())


@pytest.mark.parametrize("k,block,chunk", [(1, 128, 0), (8, 256, 65536), (8, 256, 16384), (8, 512, 0),
                                           (4, 512, 0), (4, 256, 65536), (2, 512, 0), (1, 512, 0)])
def test_full_size_regression_sampled(k, block, chunk):
    """4096 trees (depth 2-8, <= 256 nodes) x 65536 cases, the benchmark's
    workload, in the launch shape the benchmark times (K = 8, block 256,
    all 65536 cases per block) and others, among them the register-capped
    K = 1, 2, 4 kernels at their largest blocks; the oracle checks a sample
    of 48 programs entirely."""
    w = synth.regression_large()
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_SFORM,
                               gp.ORDER_MIN_DEPTH)
    P, O, L = upload(enc)
    X, Y = dev(w.cases), dev(w.targets)
    cfg = gp.Config(gp.VARIANT_REGISTER, k, block, chunk)
    f = gp.eval_population(P, O, L, X, Y, config=cfg).cpu().numpy()
    rng = np.random.default_rng(5)
    sample = np.sort(rng.choice(w.pop.n, 48, replace=False))
    exp = np.array([oracle.tree_fitness(w.pop.program(int(p)), w.cases, w.targets)
                    for p in sample])
    assert_fitness(f[sample], exp, "full-size sample")
    # per-case outputs of a few sampled programs
    for p in sample[:6]:
        sub = gp.EncodedPopulation(enc.words, enc.offsets[p:p + 1], enc.lengths[p:p + 1],
                                   0, enc.kind, enc.order)
        Pp, Op, Lp = upload(sub)
        out = gp.eval_outputs(Pp, Op, Lp, X, config=cfg).cpu().numpy()[0]
        assert_bits(out, oracle.tree_outputs(w.pop.program(int(p)), w.cases), f"program {p}")
    assert np.all(np.isfinite(f) | np.isinf(f))


@pytest.mark.parametrize("variant,k,block,chunk", [(gp.VARIANT_REGISTER_FILE, 4, 256, 131072),
                                                   (gp.VARIANT_REGISTER_FILE, 8, 128, 0),
                                                   (gp.VARIANT_REGISTER, 8, 256, 0)])
def test_full_size_register_gp_sampled(variant, k, block, chunk):
    """The register-GP workload at its full size, 8192 programs of 16-128
    instructions x 262144 cases x 8 inputs, in the launch shape the
    benchmark's tuner picks (the register file in shared memory, K = 4,
    block 256, 131072 cases per block) and others; the oracle checks the
    fitness of 24 sampled programs over every case and the per-case outputs
    of 3 of them."""
    w = synth.linear_workload(n_progs=8192)
    enc = gp.encode_linear_population(w.pop.instr, w.pop.offsets, w.pop.lengths)
    P, O, L = upload(enc)
    X, Y = dev(w.cases), dev(w.targets)
    cfg = gp.Config(variant, k, block, chunk, 0, 0, 0, enc.max_instructions)
    f = gp.eval_population(P, O, L, X, Y, config=cfg).cpu().numpy()
    sample = np.sort(np.random.default_rng(6).choice(w.pop.n, 24, replace=False))
    exp = np.array([oracle.linear_population_fitness(w.pop.instr, w.pop.offsets, w.pop.lengths, w.cases,
                                                     w.targets, p_range=(int(p), int(p) + 1))[int(p)]
                    for p in sample])
    assert_fitness(f[sample], exp, "register GP full-size sample")
    for p in sample[:3]:
        sub = gp.EncodedPopulation(enc.words, enc.offsets[p:p + 1], enc.lengths[p:p + 1], 0, enc.kind, enc.order)
        Pp, Op, Lp = upload(sub)
        out = gp.eval_outputs(Pp, Op, Lp, X, config=cfg).cpu().numpy()[0]
        assert_bits(out, oracle.linear_outputs(w.pop.program(int(p)), w.cases), f"program {p}")
    assert gp.last_error() == 0


@pytest.mark.parametrize("n_inputs", [1, 3])
def test_stack_levels_in_shared_memory(n_inputs):
    """gp_config.stack_registers = 4 (levels 4..7 in shared memory): deep
    S-form programs (full trees needing up to 7 levels) bit-exact; an RPN
    program is refused by this kernel (malformed)."""
    progs = synth.ramped_half_and_half(60 + n_inputs, 200, 2, 8, 255, n_inputs=n_inputs)
    pop = synth.pack(progs)
    x = synth.uniform_cases(61, n_inputs, 3001)
    x[0, :3] = [0.0, -0.0, 1e-40]
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    assert enc.info["max_depth"].max() >= 6
    P, O, L = upload(enc)
    ref = np.stack([oracle.tree_outputs(pop.program(p), x) for p in range(pop.n)])
    for block in (64, 256, 512):
        out = gp.eval_outputs(P, O, L, dev(x), config=gp.Config(gp.VARIANT_REGISTER, 8, block, 0, 0, 0, 4))
        assert_bits(out.cpu().numpy(), ref, f"block={block}")
    assert gp.last_error() == 0
    rpn = gp.encode_population(pop.words, pop.offsets, pop.lengths, gp.KIND_RPN)
    P, O, L = upload(rpn)
    y = dev(np.zeros(3001, np.float32))
    f = gp.eval_population(P, O, L, dev(x), y, config=gp.Config(gp.VARIANT_REGISTER, 8, 256, 0, 0, 0, 4))
    assert np.all(np.isnan(f.cpu().numpy()))
    assert gp.last_error() == 2
    with pytest.raises(gp.GPError):
        gp.eval_population(P, O, L, dev(x), y, config=gp.Config(gp.VARIANT_REGISTER, 4, 256, 0, 0, 0, 4))


@pytest.mark.parametrize("fitness", [gp.FITNESS_SUM_ABS, gp.FITNESS_MSE, gp.FITNESS_CLASS])
@pytest.mark.parametrize("chunk", [0, 4096])
def test_pass_loop_inside_the_interpreter_changes_nothing(fitness, chunk):
    """K = 8 with the input in registers runs a warp's full passes inside one
    interpreter call; asking for per-case outputs takes the per-pass path.
    The fitness is the same to the bit under every measure, with a ragged tail
    (20000 cases: the last passes partial) and with chunks of cases."""
    w = synth.regression_small(seed=77, n_progs=300, n_cases=20000)
    y = w.targets if fitness != gp.FITNESS_CLASS else np.rint(w.targets * 3.0).astype(np.float32)
    P, O, L = upload(gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths))
    X, Y = dev(w.cases), dev(y)
    cfg = gp.Config(gp.VARIANT_REGISTER, 8, 256, chunk, fitness)
    loop = gp.eval_population(P, O, L, X, Y, config=cfg).cpu().numpy()
    import torch
    outs = torch.empty((w.pop.n, w.cases.shape[1]), dtype=torch.float32, device=X.device)
    per_pass = gp.eval_population(P, O, L, X, Y, outputs=outs, config=cfg).cpu().numpy()
    assert np.array_equal(loop.view(np.uint64), per_pass.view(np.uint64))
    assert np.isfinite(loop).sum() > w.pop.n // 2


# ---------------------------------------------------------------------------
# divisions by constants: the reciprocal forms (divisor in the fast range,
# one remainder correction) and the plain forms beside them, with numerators
# that send some warps to the slow path
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("n_inputs", [1, 2])
@pytest.mark.parametrize("order", [gp.ORDER_PAPER, gp.ORDER_MIN_DEPTH])
def test_constant_divisors_bit_exact(k, n_inputs, order):
    from div_trees import constant_divisor_trees, edge_cases
    pop = synth.pack(constant_divisor_trees(n_inputs))
    x = edge_cases(3001, 76, n_inputs)
    y = synth.uniform_cases(77, 1, 3001)[0]
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths, gp.KIND_SFORM, order)
    P, O, L = upload(enc)
    ref = oracle_outputs(pop, x)
    exp = oracle.population_fitness(pop.words, pop.offsets, pop.lengths, x, y)
    for block in (32, 128):
        cfg = gp.Config(gp.VARIANT_REGISTER, k, block, 0)
        out = gp.eval_outputs(P, O, L, dev(x), config=cfg).cpu().numpy()
        assert_bits(out, ref, f"k={k} inputs={n_inputs} block={block}")
        f = gp.eval_population(P, O, L, dev(x), dev(y), config=cfg).cpu().numpy()
        assert_fitness(f, exp, f"k={k} inputs={n_inputs} block={block}")
    # the interpreters that take the plain division for these forms: the
    # extended one and the one with levels 4..7 in shared memory
    out = gp.eval_outputs(P, O, L, dev(x), config=gp.Config(gp.VARIANT_EXTENDED, k, 64, 0)).cpu().numpy()
    assert_bits(out, ref, f"extended k={k}")
    if k == 8:
        out = gp.eval_outputs(P, O, L, dev(x), config=gp.Config(gp.VARIANT_REGISTER, 8, 64, 0, 0, 0, 4)).cpu().numpy()
        assert_bits(out, ref, "levels 4..7 in shared memory")
    assert gp.last_error() == 0


def test_reciprocal_payload_is_checked_when_staged():
    """An S-form division by a constant whose payload c is not the divisor's
    reciprocal rounded to nearest is malformed (NaN fitness, status
    GP_ERR_PROGRAM): the interpreter never runs with a wrong reciprocal."""
    import torch
    from div_trees import constant_divisor_trees
    trees = constant_divisor_trees()[:2]  # x / 2^-50 and (x*x) / 2^-50: reciprocal forms
    pop = synth.pack(trees)
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    words = enc.words.copy()
    last = enc.offsets[1] + enc.lengths[1] - 1   # payload c of program 1's last instruction
    assert words[last] != 0
    words[last] ^= 1
    P = torch.from_numpy(words.view(np.int32)).cuda()
    O, L = dev(enc.offsets), dev(enc.lengths)
    x = synth.uniform_cases(78, 1, 512)
    f = gp.eval_population(P, O, L, dev(x), dev(np.zeros(512, np.float32))).cpu().numpy()
    assert not np.isnan(f[0]) and np.isnan(f[1])
    assert gp.last_error() == 2


def test_register_file_rejects_flags_that_do_not_match():
    """The register-file kernel replays the encoder's rules for what A and B
    hold: a program whose flags claim an operand from B that B does not
    hold, or both operands held, or a source that does not exist, is
    malformed (NaN fitness, program-error status); the programs beside it are
    exact."""
    pop = synth.linear_programs(84, 12, 8, 40)
    x = synth.normal_cases(85, 8, 700)
    y = synth.normal_cases(86, 1, 700)[0]
    enc = gp.encode_linear_population(pop.instr, pop.offsets, pop.lengths)
    fit = oracle.linear_population_fitness(pop.instr, pop.offsets, pop.lengths, x, y)
    cfg = gp.Config(gp.VARIANT_REGISTER_FILE, 4, 64, 0)
    for p, change in ((3, "from_b"), (5, "both"), (7, "three")):
        words = enc.words.copy()
        base = int(enc.offsets[p]) + 4
        n = int(pop.lengths[p])
        # the first instruction: nothing is held yet
        f = int(words[base + 2])
        if change == "from_b":
            words[base + 2] = (f & ~3) | 2
        elif change == "both":
            words[base + 2] = (f & ~15) | 1 | (2 << 2)
        else:
            words[base + 2] = (f & ~3) | 3
        assert n >= 1
        gp.last_error()
        got = gp.eval_population(dev(words.view(np.int32)), dev(enc.offsets), dev(enc.lengths), dev(x), dev(y),
                                 config=cfg).cpu().numpy()
        assert np.isnan(got[p]) and gp.last_error() == 2, change
        others = np.arange(pop.n) != p
        assert_fitness(got[others], fit[others], change)
