"""Several populations in one launch (gp_eval_segments): each segment's
fitness is bit-identical to evaluating its population alone with the same
configuration and chunk, and within the tolerance of the oracle; Boolean hit
counts are exact.  Segments differ in size, program lengths, case counts and
input counts, and share one kernel launch."""
import numpy as np
import pytest

import oracle
import synth
import paper_1601_00221_gb300 as gp
from gpu_util import dev, assert_fitness

pytestmark = pytest.mark.gpu


def concat(encs):
    """Concatenated encoded programs of several populations; the first
    program of each."""
    words, offs, lens, begins = [], [], [], []
    base_w = base_p = 0
    for e in encs:
        words.append(e.words)
        offs.append(e.offsets + base_w)
        lens.append(e.lengths)
        begins.append(base_p)
        base_w += e.words.size
        base_p += e.lengths.size
    import torch
    W = np.concatenate(words)
    return (torch.from_numpy(W.view(np.int32)).cuda(), dev(np.concatenate(offs)), dev(np.concatenate(lens)),
            begins)


def float_runs(spec, seed):
    runs = []
    for i, (n_progs, n_cases, n_inputs) in enumerate(spec):
        progs = synth.ramped_half_and_half(seed + i, n_progs, 2, 8, 255, n_inputs=n_inputs)
        pop = synth.pack(progs)
        x = synth.uniform_cases(seed + 100 + i, n_inputs, n_cases)
        y = synth.uniform_cases(seed + 200 + i, 1, n_cases)[0]
        runs.append((pop, x, y))
    return runs


@pytest.mark.parametrize("k,block", [(8, 128), (4, 256), (1, 64)])
@pytest.mark.parametrize("spec", [
    [(50, 1000, 1), (300, 70000, 1), (120, 5003, 1)],            # single input: registers
    [(50, 1000, 1), (300, 70000, 8), (120, 5003, 3), (7, 33, 1)],  # mixed: staged tile
])
def test_float_segments_bit_identical_to_alone_and_oracle(k, block, spec):
    import torch
    runs = float_runs(spec, 300 + k)
    encs = [gp.encode_population(p.words, p.offsets, p.lengths) for p, _, _ in runs]
    P, O, L, begins = concat(encs)
    cfg = gp.Config(gp.VARIANT_REGISTER, k, block, 0)
    chunks = [0, 2 * k * block, 0, 0][:len(runs)]
    segs, outs = [], []
    for (pop, x, y), b, ch in zip(runs, begins, chunks):
        out = torch.full((pop.n,), float("nan"), dtype=torch.float64, device="cuda")
        outs.append(out)
        segs.append(dict(prog_begin=b, n_progs=pop.n, cases=dev(x), targets=dev(y), out=out, chunk=ch))
    for _ in range(2):  # twice: the arrival counters must be back at zero
        gp.eval_segments(P, O, L, segs, config=cfg)
        torch.cuda.synchronize()
        for (pop, x, y), e, out, ch, g in zip(runs, encs, outs, chunks, segs):
            Pa, Oa, La = e.to_device("cuda")
            alone = gp.eval_population(Pa, Oa, La, g["cases"], g["targets"],
                                       config=gp.Config(gp.VARIANT_REGISTER, k, block, ch)).cpu().numpy()
            got = out.cpu().numpy()
            assert np.array_equal(got.view(np.uint64), alone.view(np.uint64)), "segment differs from alone"
            exp = oracle.population_fitness(pop.words, pop.offsets, pop.lengths, x, y)
            assert_fitness(got, exp, f"segment of {pop.n} x {x.shape}")
    assert gp.last_error() == 0


def test_float_segments_ordered_longest_first():
    """Enough programs for the block order (two blocks per multiprocessor):
    every segment's programs are taken longest first inside the segment."""
    import torch
    runs = float_runs([(400, 20000, 1), (500, 40000, 1), (300, 17, 1)], 400)
    encs = [gp.encode_population(p.words, p.offsets, p.lengths) for p, _, _ in runs]
    P, O, L, begins = concat(encs)
    segs, outs = [], []
    for (pop, x, y), b in zip(runs, begins):
        out = torch.empty(pop.n, dtype=torch.float64, device="cuda")
        outs.append(out)
        segs.append(dict(prog_begin=b, n_progs=pop.n, cases=dev(x), targets=dev(y), out=out))
    gp.eval_segments(P, O, L, segs, config=gp.Config(gp.VARIANT_REGISTER, 8, 256, 0))
    for (pop, x, y), e, out, g in zip(runs, encs, outs, segs):
        Pa, Oa, La = e.to_device("cuda")
        alone = gp.eval_population(Pa, Oa, La, g["cases"], g["targets"],
                                   config=gp.Config(gp.VARIANT_REGISTER, 8, 256, 0)).cpu().numpy()
        assert np.array_equal(out.cpu().numpy().view(np.uint64), alone.view(np.uint64))


def test_bool_segments_exact():
    import torch
    problems = [("mux", 6), ("parity", 11), ("mux", 11), ("parity", 10)]
    ws = [synth.boolean_problem(kind, k, seed=500 + i, n_progs=60 + 40 * i) for i, (kind, k) in enumerate(problems)]
    encs = [gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_BOOL) for w in ws]
    P, O, L, begins = concat(encs)
    segs, outs = [], []
    for w, b in zip(ws, begins):
        out = torch.full((w.pop.n,), -1, dtype=torch.int64, device="cuda")
        outs.append(out)
        segs.append(dict(prog_begin=b, n_progs=w.pop.n, cases=dev(w.case_bits.view(np.int32)),
                         targets=dev(w.target_bits.view(np.int32)), out=out, n_cases=w.n_cases))
    for k in (1, 4, 8):
        gp.eval_segments(P, O, L, segs, kind=gp.RUN_BOOL, config=gp.Config(gp.VARIANT_REGISTER, k, 64, 0))
        for w, out in zip(ws, outs):
            exp = oracle.bool_population_hits(w.pop.words, w.pop.offsets, w.pop.lengths, w.case_bits,
                                              w.n_cases, w.target_bits)
            assert np.array_equal(out.cpu().numpy(), np.asarray(exp, np.int64)), (w.name if hasattr(w, "name") else k)


def test_segments_argument_errors():
    import torch
    runs = float_runs([(10, 100, 1), (10, 100, 1)], 600)
    encs = [gp.encode_population(p.words, p.offsets, p.lengths) for p, _, _ in runs]
    P, O, L, begins = concat(encs)
    out = torch.empty(10, dtype=torch.float64, device="cuda")
    x, y = dev(runs[0][1]), dev(runs[0][2])
    seg = lambda b, n: dict(prog_begin=b, n_progs=n, cases=x, targets=y, out=out)
    with pytest.raises(gp.GPError, match="overlap"):
        gp.eval_segments(P, O, L, [seg(0, 10), seg(5, 10)])
    with pytest.raises(gp.GPError, match="n_segments"):
        gp.eval_segments(P, O, L, [seg(0, 1)] * (gp.MAX_SEGMENTS + 1))
    with pytest.raises(gp.GPError, match="multiple of k"):
        gp.eval_segments(P, O, L, [dict(seg(0, 10), chunk=100)], config=gp.Config(gp.VARIANT_REGISTER, 8, 128, 0))
