"""Serving (gp_server_*): continuous batching of many runs' requests.

Each result must be the same alone and in the mix (bit-identical: the split
of a run's cases never depends on what is merged or overlapped with it), agree
with the CPU oracle within the stated tolerance, and host-side failures
(cancellation, timeouts, a full queue, an exhausted memory budget, a bad run,
a malformed program) must end only the request they concern.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1601_00221_gb300 as gp
from gpu_util import assert_fitness

pytestmark = pytest.mark.gpu


def float_run(seed, n_progs, n_cases, n_inputs=1):
    progs = synth.ramped_half_and_half(seed, n_progs, 2, 7, 127, n_inputs=n_inputs)
    pop = synth.pack(progs)
    x = synth.uniform_cases(seed + 1, n_inputs, n_cases)
    y = synth.quartic_target(x[0]) if n_inputs == 1 else synth.uniform_cases(seed + 2, 1, n_cases)[0]
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    return dict(kind=gp.RUN_FLOAT, pop=pop, x=x, y=y, enc=enc, n_cases=n_cases)


def bool_run(seed, kind, k, n_progs):
    w = synth.boolean_problem(kind, k, seed=seed, n_progs=n_progs)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths, gp.KIND_BOOL)
    return dict(kind=gp.RUN_BOOL, pop=w.pop, x=w.case_bits, y=w.target_bits, enc=enc,
                n_cases=w.n_cases)


def register(srv, r):
    if r["kind"] == gp.RUN_FLOAT:
        return srv.register_run(r["x"], r["y"])
    return srv.register_run(r["x"], r["y"], kind=gp.RUN_BOOL, n_cases=r["n_cases"])


def oracle_result(r, progs=None):
    pop = r["pop"]
    if r["kind"] == gp.RUN_FLOAT:
        return oracle.population_fitness(pop.words, pop.offsets, pop.lengths, r["x"], r["y"])
    return oracle.bool_population_hits(pop.words, pop.offsets, pop.lengths, r["x"], r["n_cases"],
                                       r["y"])


@pytest.fixture(scope="module")
def runs():
    return [
        float_run(101, 300, 3001),
        float_run(102, 120, 70000),            # several blocks per program
        float_run(103, 200, 4096, n_inputs=8),  # staged multi-input tile
        bool_run(104, "mux", 11, 150),
        bool_run(105, "parity", 6, 400),
        float_run(106, 50, 100),
    ]


def test_requests_match_the_oracle(runs):
    with gp.Server() as srv:
        ids = [register(srv, r) for r in runs]
        reqs = [srv.submit(i, r["enc"], kind=r["kind"]) for i, r in zip(ids, runs)]
        for q, r in zip(reqs, runs):
            out, info = srv.wait(q)
            assert info.status == 0 and info.n_progs == r["enc"].n
            assert info.t_submit_us <= info.t_admit_us <= info.t_done_us
            exp = oracle_result(r)
            if r["kind"] == gp.RUN_FLOAT:
                assert_fitness(out, exp, "served")
            else:
                assert np.array_equal(out, exp)


def test_alone_and_in_the_mix_are_bit_identical(runs):
    # alone: one request at a time, waited before the next is submitted
    alone = []
    with gp.Server(n_streams=1, max_inflight=1) as srv:
        ids = [register(srv, r) for r in runs]
        for i, r in zip(ids, runs):
            q = srv.submit(i, r["enc"], kind=r["kind"])
            alone.append(srv.wait(q)[0].copy())
    # mix: every request of every run at once, three generations each,
    # consecutive requests of a run merged into one launch, runs on 4 streams
    with gp.Server(n_streams=4, max_inflight=8) as srv:
        ids = [register(srv, r) for r in runs]
        order = []
        for gen in range(3):
            for j in range(len(runs)):
                order.append(j)
                if j % 2 == 0:
                    order.append(j)  # two consecutive requests of the same run: merged
        qs = [(j, srv.submit(ids[j], runs[j]["enc"], kind=runs[j]["kind"])) for j in order]
        for j, q in qs:
            out, info = srv.wait(q)
            if runs[j]["kind"] == gp.RUN_FLOAT:
                assert np.array_equal(out.view(np.uint64), alone[j].view(np.uint64)), j
            else:
                assert np.array_equal(out, alone[j]), j
        st = srv.stats()
        assert st["completed"] == len(qs)
        assert st["launches"] < len(qs)  # merging happened
        assert st["p99_latency_us"] >= st["p50_latency_us"] > 0
        assert st["gpop_per_s"] > 0


def test_cancel_busy_timeout(runs):
    big = float_run(110, 2048, 65536)
    with gp.Server(n_streams=1, max_inflight=1, max_queued=2, max_merge=2048) as srv:
        rb = register(srv, big)
        r0 = srv.submit(rb, big["enc"])      # admitted: runs for milliseconds
        r1 = srv.submit(rb, big["enc"])      # queued
        r2 = srv.submit(rb, big["enc"])      # queued (queue now full)
        with pytest.raises(gp.GPError) as e:
            srv.submit(rb, big["enc"])
        assert e.value.code == 7             # GP_ERR_BUSY
        assert srv.cancel(r2) == 0
        with pytest.raises(gp.GPError) as e:
            srv.wait(r2)
        assert e.value.code == 8             # cancelled
        with pytest.raises(gp.GPError) as e:
            srv.wait(r1, timeout_s=0.0)      # cannot be done yet
        assert e.value.code == 5             # GP_ERR_TIMEOUT
        out0, _ = srv.wait(r0)
        out1, _ = srv.wait(r1)
        assert np.array_equal(out0.view(np.uint64), out1.view(np.uint64))
        st = srv.stats()
        assert st["cancelled"] == 1 and st["completed"] == 2


def test_memory_budget_and_bad_run(runs):
    r = runs[0]
    with gp.Server(memory_budget=1024) as srv:
        rid = register(srv, r)
        with pytest.raises(gp.GPError) as e:
            srv.submit(rid, r["enc"])
        assert e.value.code == 4             # GP_ERR_OOM: the request alone exceeds the budget
        with pytest.raises(gp.GPError) as e:
            srv.submit(99, r["enc"])
        assert e.value.code == 1


def test_malformed_program_only_affects_its_request(runs):
    r = runs[0]
    bad = gp.EncodedPopulation(r["enc"].words.copy(), r["enc"].offsets, r["enc"].lengths,
                               r["enc"].nodes, r["enc"].kind, r["enc"].order)
    bad.words[int(bad.offsets[5]) + 4] = 0xFFFF
    with gp.Server() as srv:
        rid = register(srv, r)
        qa = srv.submit(rid, r["enc"])
        qb = srv.submit(rid, bad)            # merged with qa into one launch
        qc = srv.submit(rid, r["enc"])
        a, _ = srv.wait(qa)
        b, _ = srv.wait(qb)
        c, _ = srv.wait(qc)
    assert np.isnan(b[5])
    mask = np.arange(b.size) != 5
    assert np.array_equal(a.view(np.uint64)[mask], b.view(np.uint64)[mask])
    assert np.array_equal(a.view(np.uint64), c.view(np.uint64))


def test_extended_functions_and_fitness_measures_are_served():
    """A server configured with the extended interpreter and classification
    fitness serves Shuttle-set runs; each result equals the direct evaluation
    and the oracle's exact counts."""
    import torch
    cfg = gp.Config(gp.VARIANT_EXTENDED, 4, 128, 0, gp.FITNESS_CLASS)
    runs = [synth.shuttle_like_problem(seed=140 + i, n_progs=64 + 32 * i, n_cases=900 + 500 * i)
            for i in range(3)]
    with gp.Server(config=cfg) as srv:
        ids = [srv.register_run(w.cases, w.targets) for w in runs]
        encs = [gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths) for w in runs]
        reqs = [srv.submit(i, e) for i, e in zip(ids, encs)]
        for q, w, e in zip(reqs, runs, encs):
            out, info = srv.wait(q)
            assert info.status == 0
            exp = oracle.fset_population_fitness(w.pop.words, w.pop.offsets, w.pop.lengths, w.cases,
                                                 w.targets, oracle.FIT_CLASS)
            assert np.array_equal(out, exp)


@pytest.fixture(scope="module")
def blocker():
    """A request that keeps the GPU busy for tens of milliseconds (4096 trees
    x 2^20 cases), so that later submissions queue up behind it."""
    return float_run(120, 4096, 1 << 20)


def test_requests_of_different_runs_share_one_launch(runs, blocker):
    """While one long request occupies the only in-flight slot, requests of
    six other runs queue up; they are then admitted together -- the float
    runs' requests (one and eight inputs, different case counts) in one
    launch, the Boolean runs' in another -- and every result is bit-identical
    to the same request served alone, and equal to the oracle's within the
    tolerance (exact hits)."""
    alone = []
    with gp.Server(n_streams=1, max_inflight=1) as srv:
        ids = [register(srv, r) for r in runs]
        for i, r in zip(ids, runs):
            alone.append(srv.wait(srv.submit(i, r["enc"], kind=r["kind"]))[0].copy())
    with gp.Server(n_streams=1, max_inflight=1) as srv:
        ids = [register(srv, r) for r in runs]
        bid = register(srv, blocker)
        qb = srv.submit(bid, blocker["enc"])
        qs = [srv.submit(i, r["enc"], kind=r["kind"]) for i, r in zip(ids, runs)]
        srv.wait(qb)
        infos = []
        for q, r, a in zip(qs, runs, alone):
            out, info = srv.wait(q)
            infos.append(info)
            if r["kind"] == gp.RUN_FLOAT:
                assert np.array_equal(out.view(np.uint64), a.view(np.uint64))
                assert_fitness(out, oracle_result(r), "mixed launch")
            else:
                assert np.array_equal(out, a)
                assert np.array_equal(out, oracle_result(r))
        st = srv.stats()
    # requests admitted together carry the same admission time
    groups = {}
    for j, info in enumerate(infos):
        groups.setdefault(info.t_admit_us, []).append(j)
    biggest = max(groups.values(), key=len)
    assert len({runs[j]["kind"] for j in biggest}) == 1
    assert len(biggest) >= 3, groups
    assert st["launches"] <= 3 and st["completed"] == len(runs) + 1


def test_a_large_head_is_passed_by_requests_that_fit(runs, blocker):
    """Under a memory budget that the first queued request cannot get while
    another launch holds memory, smaller requests behind it are admitted
    first (a bounded number of times), and every result is still correct."""
    small = runs[0]
    with gp.Server(n_streams=2, max_inflight=2, memory_budget=5 << 20) as srv:  # one blocker: ~3 MB
        rb, rs = register(srv, blocker), register(srv, small)
        q0 = srv.submit(rb, blocker["enc"])   # admitted, holds most of the budget
        q1 = srv.submit(rb, blocker["enc"])   # does not fit until q0 is done
        q2 = srv.submit(rs, small["enc"])     # fits beside q0
        out2, i2 = srv.wait(q2)
        out1, i1 = srv.wait(q1)
        out0, i0 = srv.wait(q0)
    assert i2.t_admit_us < i1.t_admit_us
    assert np.array_equal(out0.view(np.uint64), out1.view(np.uint64))
    assert_fitness(out2, oracle_result(small), "passed head")
