"""GPU parity of the extended S-form interpreter (the full float function sets
of Sec. 4.2) and of the fitness measures, against the CPU oracle.

* Programs without a transcendental function (the Shuttle set: *, /, +, -,
  >, <, ==, AND, OR, IF): per-case outputs bit-exact (any NaN equals any NaN).
* Programs with SIN, COS, EXP, LOG: there is no unique binary32 answer, so
  every per-case output must lie inside the oracle's enclosure of all
  admissible implementations (CUDA's documented bounds: sinf, cosf, expf
  2 ulp, logf 1 ulp), and most enclosures must be tight (so that the check
  has teeth); each single function is also held to its documented bound
  directly.
* Fitness: sum |e|, mean squared error, classification errors; within 1e-5
  relative of the binary64 oracle (classification counts exactly) for exact
  programs, inside the oracle's fitness enclosure widened by 1e-5 otherwise.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1601_00221_gb300 as gp
from gpu_util import dev, upload, assert_bits, assert_fitness, REL_TOL
from synth import SIN, COS, EXP, LOG, VAR, tok

pytestmark = pytest.mark.gpu

KS = [1, 2, 4, 8]
FITS = [gp.FITNESS_SUM_ABS, gp.FITNESS_MSE, gp.FITNESS_CLASS]


def ext_cfg(k, block=128, chunk=0, fitness=gp.FITNESS_SUM_ABS, kind=gp.KIND_SFORM):
    variant = gp.VARIANT_EXTENDED_RPN if kind == gp.KIND_RPN else gp.VARIANT_EXTENDED
    return gp.Config(variant, k, block, chunk, fitness)


def oracle_fset_outputs(pop, x):
    return np.stack([oracle.fset_outputs(pop.program(p), x) for p in range(pop.n)])


def enclosures(pop, x):
    lo, hi, nan = zip(*(oracle.fset_enclosure(pop.program(p), x) for p in range(pop.n)))
    return np.stack(lo), np.stack(hi), np.stack(nan)


def assert_inside(got, lo, hi, nan, what):
    ok = np.where(np.isnan(got), nan, (lo <= got) & (got <= hi))
    if not ok.all():
        i = np.argwhere(~ok)[0]
        raise AssertionError(f"{what}: {int((~ok).sum())} outputs outside, first {i.tolist()}: "
                             f"{got[tuple(i)]!r} not in [{lo[tuple(i)]!r}, {hi[tuple(i)]!r}]")


def tight_fraction(lo, hi):
    fin = lo <= hi
    mag = np.maximum(np.abs(lo), np.abs(hi)).astype(np.float32)
    with np.errstate(invalid="ignore"):
        w = (hi.astype(np.float64) - lo) / np.maximum(np.spacing(mag), 1e-45)
    return float(np.mean(fin & (w <= 64)))


def assert_fitness_inside(got, pop, x, y, kind, lo, hi, nan, what):
    for p in range(pop.n):
        f_lo, f_hi, may_inf, must_inf = oracle.fitness_enclosure(lo[p], hi[p], nan[p], y, kind)
        g = float(got[p])
        if g == np.inf:
            assert may_inf, f"{what} program {p}: +inf not admissible"
            continue
        assert not must_inf, f"{what} program {p}: got {g}, must be +inf"
        if kind == gp.FITNESS_CLASS:
            assert f_lo <= g <= f_hi, f"{what} program {p}: {g} not in [{f_lo}, {f_hi}]"
        else:
            assert f_lo * (1 - REL_TOL) - 1e-30 <= g <= f_hi * (1 + REL_TOL) + 1e-30, \
                f"{what} program {p}: {g} not in [{f_lo}, {f_hi}]"


# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def exact_set():
    """Shuttle-set trees on 9 integer inputs (zeros, so protected division and
    false conditions occur), ragged case count, with specials."""
    w = synth.shuttle_like_problem(seed=101, n_progs=96, n_cases=1500)
    x = w.cases.copy()
    x[:, :6] = np.array([0.0, -0.0, np.nan, np.inf, -np.inf, 1e-45], np.float32)[None, :]
    return w, x, oracle_fset_outputs(w.pop, x)


@pytest.mark.parametrize("kind", [gp.KIND_SFORM, gp.KIND_RPN])
@pytest.mark.parametrize("k", KS)
def test_exact_extended_programs_bit_exact(exact_set, k, kind):
    w, x, ref = exact_set
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, kind)
    assert enc.extended
    P, O, L = upload(enc)
    for block in (64, 256):
        out = gp.eval_outputs(P, O, L, dev(x), config=ext_cfg(k, block, kind=kind))
        assert_bits(out.cpu().numpy(), ref, f"k={k} block={block}")
    assert gp.last_error() == 0


@pytest.mark.parametrize("k", KS)
def test_exact_extended_single_input_in_registers(k):
    progs = synth.ramped_half_and_half(102, 80, 2, 7, 128, funcs=synth.SHUTTLE_FUNCS,
                                       const_lo=-2.0, const_hi=2.0, full_fallback_to_grow=True)
    pop = synth.pack(progs)
    x = synth.uniform_cases(103, 1, 2051, -2.0, 2.0)
    x[0, :4] = np.array([0.0, -0.0, np.nan, 1.0], np.float32)
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    P, O, L = upload(enc)
    out = gp.eval_outputs(P, O, L, dev(x), config=ext_cfg(k))
    assert_bits(out.cpu().numpy(), oracle_fset_outputs(pop, x), f"k={k}")


@pytest.fixture(scope="module")
def trans_set():
    """All fourteen functions (the KDDcup set) on 3 inputs, x ~ U[-3, 3]."""
    progs = synth.ramped_half_and_half(104, 120, 2, 8, 256, funcs=synth.KDD_FUNCS, n_inputs=3,
                                       const_lo=-2.0, const_hi=2.0, full_fallback_to_grow=True)
    pop = synth.pack(progs)
    x = synth.uniform_cases(105, 3, 777, -3.0, 3.0)
    x[:, :3] = np.array([0.0, 1e-45, np.nan], np.float32)[None, :]
    lo, hi, nan = enclosures(pop, x)
    return pop, x, lo, hi, nan


@pytest.mark.parametrize("kind", [gp.KIND_SFORM, gp.KIND_RPN])
@pytest.mark.parametrize("k", KS)
def test_transcendental_outputs_inside_enclosures(trans_set, k, kind):
    pop, x, lo, hi, nan = trans_set
    assert tight_fraction(lo, hi) >= 0.8
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths, kind)
    P, O, L = upload(enc)
    out = gp.eval_outputs(P, O, L, dev(x), config=ext_cfg(k, kind=kind)).cpu().numpy()
    assert_inside(out, lo, hi, nan, f"k={k}")
    assert gp.last_error() == 0


@pytest.mark.parametrize("k", [2, 8])
def test_sextic_single_input_inside_enclosures(k):
    w = synth.sextic_problem(seed=106, n_progs=100, n_cases=3000)
    lo, hi, nan = enclosures(w.pop, w.cases)
    assert tight_fraction(lo, hi) >= 0.8
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths)
    P, O, L = upload(enc)
    X, Y = dev(w.cases), dev(w.targets)
    out = gp.eval_outputs(P, O, L, X, config=ext_cfg(k)).cpu().numpy()
    assert_inside(out, lo, hi, nan, f"sextic k={k}")
    f = gp.eval_population(P, O, L, X, Y, config=ext_cfg(k, fitness=gp.FITNESS_MSE)).cpu().numpy()
    assert_fitness_inside(f, w.pop, w.cases, w.targets, gp.FITNESS_MSE, lo, hi, nan, "sextic MSE")


def _ulps(a, b):
    """Distance in binary32 steps between finite a and b."""
    def key(v):
        i = v.view(np.int32).astype(np.int64)
        return np.where(i < 0, -(i & 0x7FFFFFFF), i)
    return np.abs(key(a) - key(b))


@pytest.mark.parametrize("op,bound", [(SIN, 2), (COS, 2), (EXP, 2), (LOG, 1)])
def test_unary_functions_within_documented_ulps(op, bound):
    rng = np.random.default_rng(110 + op)
    n = 1 << 18
    bits = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32).copy()
    x[: n // 2] = rng.uniform(-100, 100, n // 2).astype(np.float32)   # the common range
    x[:8] = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, 88.7, -103.0], np.float32)
    X = x[None, :]
    pop = synth.pack([np.array([op, tok(VAR, 0)], np.uint32)])
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    P, O, L = upload(enc)
    got = gp.eval_outputs(P, O, L, dev(X), config=ext_cfg(8)).cpu().numpy()[0]
    lo, hi, nan = oracle.fset_enclosure(pop.program(0), X)
    assert_inside(got[None], lo[None], hi[None], nan[None], f"op {op}")
    ref = oracle.fset_outputs(pop.program(0), X)        # nearest binary32 to the binary64 value
    both = np.isfinite(got) & np.isfinite(ref)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.array_equal(got[np.isinf(ref)], ref[np.isinf(ref)]) or op == EXP
    assert _ulps(got[both], ref[both]).max() <= bound


@pytest.mark.parametrize("kind", [gp.KIND_SFORM, gp.KIND_RPN])
def test_basic_programs_identical_on_both_interpreters(kind):
    w = synth.regression_small(seed=107, n_progs=128, n_cases=999)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, kind)
    assert not enc.extended
    P, O, L = upload(enc)
    X = dev(w.cases)
    for k in KS:
        a = gp.eval_outputs(P, O, L, X, config=gp.Config(gp.VARIANT_REGISTER, k, 128, 0)).cpu().numpy()
        b = gp.eval_outputs(P, O, L, X, config=ext_cfg(k, kind=kind)).cpu().numpy()
        assert_bits(b, a, f"k={k}")


def test_extended_program_needs_the_extended_variant(exact_set):
    w, x, ref = exact_set
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths)
    P, O, L = upload(enc)
    kinds = enc.words[enc.offsets] & 0xFF
    f = gp.eval_population(P, O, L, dev(x), dev(w.targets), config=gp.Config(gp.VARIANT_REGISTER, 8, 128, 0))
    f = f.cpu().numpy()
    assert np.all(np.isnan(f[kinds == gp.KIND_SFORM_EXT]))
    assert gp.last_error() == 2
    assert gp.last_error() == 0


# ---------------------------------------------------------------------------
# fitness measures
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fit", FITS)
@pytest.mark.parametrize("variant,kind", [(gp.VARIANT_REGISTER, gp.KIND_SFORM),
                                          (gp.VARIANT_REGISTER, gp.KIND_RPN),
                                          (gp.VARIANT_LOCAL, gp.KIND_RPN),
                                          (gp.VARIANT_EXTENDED, gp.KIND_SFORM)])
def test_fitness_measures_basic_programs(fit, variant, kind):
    w = synth.regression_small(seed=108, n_progs=96, n_cases=3001)
    x = w.cases.copy()
    y = w.targets.copy()
    if fit == gp.FITNESS_CLASS:
        y = np.rint(y * 2).astype(np.float32)      # integer labels in -2..8
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, kind)
    P, O, L = upload(enc)
    exp = oracle.fset_population_fitness(w.pop.words, w.pop.offsets, w.pop.lengths, x, y, fit)
    for chunk in (0, 512):
        k = 1 if variant == gp.VARIANT_LOCAL else 4
        cfg = gp.Config(variant, k, 128 if variant != gp.VARIANT_LOCAL else 256, chunk, fit)
        got = gp.eval_population(P, O, L, dev(x), dev(y), config=cfg).cpu().numpy()
        if fit == gp.FITNESS_CLASS:
            assert np.array_equal(got, exp), f"chunk={chunk}"
        else:
            assert_fitness(got, exp, f"fit={fit} chunk={chunk}")


@pytest.mark.parametrize("fit", FITS)
def test_fitness_measures_extended_programs(trans_set, fit):
    pop, x, lo, hi, nan = trans_set
    y = np.rint(np.random.default_rng(109).uniform(-1, 3, x.shape[1])).astype(np.float32)
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    P, O, L = upload(enc)
    for chunk in (0, 256):
        got = gp.eval_population(P, O, L, dev(x), dev(y), config=ext_cfg(4, 64, chunk, fit)).cpu().numpy()
        assert_fitness_inside(got, pop, x, y, fit, lo, hi, nan, f"fit={fit} chunk={chunk}")


def test_fitness_measures_no_cases():
    w = synth.regression_small(seed=111, n_progs=16, n_cases=0)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths)
    P, O, L = upload(enc)
    X = dev(np.zeros((1, 0), np.float32))
    Y = dev(np.zeros(0, np.float32))
    for fit in FITS:
        f = gp.eval_population(P, O, L, X, Y, config=gp.Config(gp.VARIANT_REGISTER, 8, 128, 0, fit))
        assert np.all(f.cpu().numpy() == 0)


# ---------------------------------------------------------------------------
# staged-input compaction: a tree stages only the inputs it reads
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def wide():
    """Shuttle-set trees over 41 inputs (the KDDcup shape), ragged cases."""
    progs = synth.ramped_half_and_half(120, 128, 2, 7, 128, funcs=synth.SHUTTLE_FUNCS, n_inputs=41,
                                       const_lo=-50.0, const_hi=50.0, full_fallback_to_grow=True)
    pop = synth.pack(progs)
    rng = np.random.default_rng(121)
    x = rng.integers(-20, 21, (41, 2999)).astype(np.float32)
    return pop, x, oracle_fset_outputs(pop, x)


@pytest.mark.parametrize("k,block", [(8, 256), (4, 128), (1, 64)])
def test_compacted_tiles_bit_exact(wide, k, block):
    pop, x, ref = wide
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    used = enc.info["inputs_used"]
    assert 0 < enc.max_inputs_used < 41
    P, O, L = upload(enc)
    cfg = enc.config(k=k, block=block)
    assert cfg.tile_inputs == enc.max_inputs_used
    out = gp.eval_outputs(P, O, L, dev(x), config=cfg)
    assert_bits(out.cpu().numpy(), ref, f"k={k} block={block}")
    assert gp.last_error() == 0


def test_tile_smaller_than_a_program_needs(wide):
    pop, x, ref = wide
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    used = enc.info["inputs_used"]
    cap = int(np.median(used))
    P, O, L = upload(enc)
    cfg = enc.config(k=4, block=128)
    cfg.tile_inputs = cap
    y = np.zeros(x.shape[1], np.float32)
    f = gp.eval_population(P, O, L, dev(x), dev(y), config=cfg).cpu().numpy()
    assert np.all(np.isnan(f[used > cap]))
    assert not np.any(np.isnan(f[used <= cap]))
    assert gp.last_error() == 2
    out = gp.eval_outputs(P, O, L, dev(x), config=cfg).cpu().numpy()
    assert_bits(out[used <= cap], ref[used <= cap], "programs that fit")
    gp.last_error()


def test_tree_reading_more_inputs_than_the_list_holds():
    """A chain over 300 distinct inputs (more than the 256 a block lists):
    every input is staged in order, and the outputs stay exact."""
    n_in = 300
    chain = []
    for v in range(n_in - 1):
        chain += [synth.ADD, tok(VAR, v)]
    chain.append(tok(VAR, n_in - 1))
    other = [synth.MUL, tok(VAR, 7), tok(VAR, 299)]
    pop = synth.pack([np.array(chain, np.uint32), np.array(other, np.uint32)])
    x = synth.uniform_cases(130, n_in, 100, -1.0, 1.0)
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    assert enc.max_inputs_used == n_in
    P, O, L = upload(enc)
    for k in (1, 2):
        out = gp.eval_outputs(P, O, L, dev(x), config=gp.Config(gp.VARIANT_REGISTER, k, 32, 0))
        exp = np.stack([oracle.tree_outputs(pop.program(p), x) for p in range(2)])
        assert_bits(out.cpu().numpy(), exp, f"k={k}")
    assert gp.last_error() == 0



@pytest.mark.parametrize("name", ["sextic", "shuttle-like", "kdd-like"])
def test_full_size_function_set_problems_sampled(name):
    """The benchmark's function-set workloads at full size, in the launch
    shapes it times (the population's own configuration); sampled trees are
    checked case by case against the oracle's enclosures (bit for bit where no
    transcendental function occurs), and their fitness too."""
    make = {"sextic": synth.sextic_problem, "shuttle-like": synth.shuttle_like_problem,
            "kdd-like": synth.kdd_like_problem}[name]
    w = make()
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths)
    k = 2 if name == "kdd-like" else 8
    cfg = enc.config(fitness=w.fitness, k=k, block=256)
    P, O, L = upload(enc)
    X, Y = dev(w.cases), dev(w.targets)
    f = gp.eval_population(P, O, L, X, Y, config=cfg).cpu().numpy()
    sample = np.arange(0, w.pop.n, w.pop.n // 5)[:5]
    import torch
    out = gp.eval_outputs(P, O, L, X, config=cfg)[torch.from_numpy(sample).cuda()].cpu().numpy()
    for i, p in enumerate(sample):
        lo, hi, nan = oracle.fset_enclosure(w.pop.program(int(p)), w.cases)
        assert_inside(out[i][None], lo[None], hi[None], nan[None], f"{name} program {p}")
        f_lo, f_hi, may_inf, must_inf = oracle.fitness_enclosure(lo, hi, nan, w.targets, w.fitness)
        g = float(f[p])
        if g == np.inf:
            assert may_inf
        elif w.fitness == gp.FITNESS_CLASS:
            assert f_lo <= g <= f_hi
        else:
            assert f_lo * (1 - REL_TOL) <= g <= f_hi * (1 + REL_TOL)
    assert gp.last_error() == 0



def test_each_extended_kernel_runs_its_own_form(exact_set):
    """The extended S-form kernel refuses RPN programs and the extended RPN
    kernel S-form ones (malformed for that kernel, fitness NaN)."""
    w, x, ref = exact_set
    y = dev(w.targets)
    for kind, wrong in ((gp.KIND_SFORM, gp.VARIANT_EXTENDED_RPN), (gp.KIND_RPN, gp.VARIANT_EXTENDED)):
        enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, kind)
        P, O, L = upload(enc)
        f = gp.eval_population(P, O, L, dev(x), y, config=gp.Config(wrong, 4, 128, 0)).cpu().numpy()
        assert np.isnan(f).all()
        assert gp.last_error() == 2



def test_blockgp_runs_the_extended_functions(exact_set, trans_set):
    """The BlockGP-style local-memory interpreter (the paper's baseline) on
    extended RPN programs: exact sets bit for bit, the full set inside the
    enclosures."""
    cfg = gp.Config(gp.VARIANT_LOCAL, 1, 256, 0)
    w, x, ref = exact_set
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_RPN)
    P, O, L = upload(enc)
    assert_bits(gp.eval_outputs(P, O, L, dev(x), config=cfg).cpu().numpy(), ref, "exact set")
    pop, xt, lo, hi, nan = trans_set
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths, gp.KIND_RPN)
    P, O, L = upload(enc)
    assert_inside(gp.eval_outputs(P, O, L, dev(xt), config=cfg).cpu().numpy(), lo, hi, nan, "full set")
    assert gp.last_error() == 0


# ---------------------------------------------------------------------------
# width split: narrow programs under one configuration, wide ones under another
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("split", [2, 6, 40])
def test_width_split_matches_each_class_alone(wide, split):
    """Each program's fitness under gp_eval_population_split equals its
    fitness under its class's configuration evaluated alone (bit for bit),
    and the oracle's."""
    import torch
    pop, x, ref = wide
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    used = enc.info["inputs_used"]
    y = np.rint(np.random.default_rng(131).uniform(-1, 3, x.shape[1])).astype(np.float32)
    P, O, L = upload(enc)
    X, Y = dev(x), dev(y)
    narrow = ext_cfg(8, 128, 0, gp.FITNESS_CLASS)
    narrow.tile_inputs = split
    narrow.max_instructions = enc.max_instructions
    widecfg = enc.config(fitness=gp.FITNESS_CLASS, k=2, block=256)
    got = gp.eval_population_split(P, O, L, X, Y, split, narrow, widecfg).cpu().numpy()
    a = gp.eval_population(P, O, L, X, Y, config=narrow).cpu().numpy()
    b = gp.eval_population(P, O, L, X, Y, config=widecfg).cpu().numpy()
    gp.last_error()  # (the narrow tile cannot hold the wide programs alone)
    exp_cls = np.where(used <= split, a, b)
    assert np.array_equal(got.view(np.uint64), exp_cls.view(np.uint64))
    exp = oracle.fset_population_fitness(pop.words, pop.offsets, pop.lengths, x, y, oracle.FIT_CLASS)
    assert np.array_equal(got, exp)
    assert gp.last_error() == 0


@pytest.mark.parametrize("fit", [gp.FITNESS_CLASS, gp.FITNESS_SUM_ABS])
def test_recorded_width_split_runs_for_automatic_configurations(wide, tmp_path, fit):
    """A width split recorded for the population's shape (as the float tuner
    records one) runs when the configuration leaves k and block at 0: the
    fitness equals that of gp_eval_population_split with the record's
    classes, bit for bit, and the oracle's (exactly for classification,
    within the tolerance for absolute errors); a request for outputs ignores
    the record."""
    pop, x, ref = wide
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    y = np.rint(np.random.default_rng(132).uniform(-1, 3, x.shape[1])).astype(np.float32)
    P, O, L = upload(enc)
    X, Y = dev(x), dev(y)
    n_cases = x.shape[1]
    key = (gp.VARIANT_EXTENDED, 1, int(np.log2(n_cases)), int(np.log2(pop.n)))
    gp.autotune_clear()
    rec = tmp_path / "split.txt"
    rec.write_text("split %d %d %d %d 6 %d 8 256 0 %d 2 128 0\n" % (key + (gp.VARIANT_EXTENDED, gp.VARIANT_EXTENDED)))
    gp.autotune_load(str(rec))
    assert gp.autotune_split_record(gp.VARIANT_EXTENDED, 41, n_cases, pop.n)[0] == 6
    auto = enc.config(fitness=fit)  # k = block = 0: the library's choice
    assert auto.k == 0 and auto.block == 0
    got = gp.eval_population(P, O, L, X, Y, config=auto).cpu().numpy()
    narrow = enc.config(fitness=fit, k=8, block=256)
    narrow.tile_inputs = 6
    widecfg = enc.config(fitness=fit, k=2, block=128)
    split = gp.eval_population_split(P, O, L, X, Y, 6, narrow, widecfg).cpu().numpy()
    assert np.array_equal(got.view(np.uint64), split.view(np.uint64))
    ofit = oracle.FIT_CLASS if fit == gp.FITNESS_CLASS else oracle.FIT_ABS
    exp = oracle.fset_population_fitness(pop.words, pop.offsets, pop.lengths, x, y, ofit)
    if fit == gp.FITNESS_CLASS:
        assert np.array_equal(got, exp)
    else:
        assert_fitness(got, exp, "recorded split, absolute errors")
    outs = gp.eval_outputs(P, O, L, X, config=auto).cpu().numpy()  # outputs: one launch
    assert_bits(outs, ref, "outputs under a recorded split")
    gp.autotune_clear()
    assert gp.last_error() == 0


def test_tuner_records_a_width_split_only_when_faster(wide):
    """The float tuner on a 41-input population: whatever it records (a split
    or none), the automatic evaluation afterwards gives the oracle's
    classification fitness; a recorded split names one of the thresholds it
    tries."""
    pop, x, ref = wide
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    y = np.rint(np.random.default_rng(133).uniform(-1, 3, x.shape[1])).astype(np.float32)
    P, O, L = upload(enc)
    X, Y = dev(x), dev(y)
    gp.autotune_clear()
    gp.autotune_population_ex(P, O, L, X, Y, base=enc.config(fitness=gp.FITNESS_CLASS), repeats=1)
    th = gp.autotune_split_record(gp.VARIANT_EXTENDED, 41, x.shape[1], pop.n)[0]
    assert th in (0, 6, 8, 12, 16)
    got = gp.eval_population(P, O, L, X, Y, config=enc.config(fitness=gp.FITNESS_CLASS)).cpu().numpy()
    exp = oracle.fset_population_fitness(pop.words, pop.offsets, pop.lengths, x, y, oracle.FIT_CLASS)
    assert np.array_equal(got, exp)
    gp.autotune_clear()
