"""Pins of the oracle's genetic operators (CPU only).

The random numbers are pinned to the published Philox4x32-10 known-answer
vectors; tournament selection to a brute-force minimum over the drawn picks;
crossover and mutation to the structure of prefix trees (every result is one
well-formed tree, the replaced subtree and the inserted one account for every
node, the size cap holds); grown subtrees to their depth bound and constant
range.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import gp_ops

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_known_answers():
    rows = 0
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        c, k, o = (list(int(v, 16) for v in part.split()) for part in line.split("|"))
        assert gp_ops.philox4x32_10(c, k) == o
        rows += 1
    assert rows == 3


def test_stream_thresholds_and_uniform():
    s = gp_ops.Stream(seed=(7 << 32) | 9, individual=3, generation=5)
    words = [s.next() for _ in range(8)]
    assert words[:4] == gp_ops.philox4x32_10((3, 5, 0, 0), (9, 7))
    assert words[4:] == gp_ops.philox4x32_10((3, 5, 1, 0), (9, 7))
    assert gp_ops.threshold(0.0) == 0 and gp_ops.threshold(1.0) == 2 ** 32 - 1
    assert gp_ops.threshold(0.5) == 2 ** 31 and gp_ops.threshold(0.25) == 2 ** 30
    s = gp_ops.Stream(1, 0, 0)
    assert all(s.uniform(1) == 0 for _ in range(100))
    counts = np.bincount([s.uniform(7) for _ in range(7000)], minlength=7)
    assert counts.min() > 850 and counts.max() < 1150


def test_uniform_is_multiply_shift():
    """uniform(n) = floor(u * n / 2^32): the top bits of u for a power of two,
    and monotone in u (a modulo would be neither)."""
    for n in (2, 8, 1024):
        s1, s2 = gp_ops.Stream(5, 1, 1), gp_ops.Stream(5, 1, 1)
        us = [s1.next() for _ in range(400)]
        vs = [s2.uniform(n) for _ in range(400)]
        shift = 32 - (n.bit_length() - 1)
        assert vs == [u >> shift for u in us]
    s1, s2 = gp_ops.Stream(6, 2, 2), gp_ops.Stream(6, 2, 2)
    pairs = sorted(zip([s1.next() for _ in range(400)], [s2.uniform(1000) for _ in range(400)]))
    assert all(a[1] <= b[1] for a, b in zip(pairs, pairs[1:]))


def test_tournament_is_the_minimum_of_its_picks():
    rng = np.random.default_rng(3)
    fit = rng.uniform(0, 10, 50)
    fit[[3, 17]] = np.nan
    fit[9] = fit[11] = 0.5
    for trial in range(200):
        s1 = gp_ops.Stream(11, trial, 2)
        s2 = gp_ops.Stream(11, trial, 2)
        w = gp_ops.tournament(s1, fit, 7)
        picks = [s2.uniform(50) for _ in range(7)]
        keys = [np.inf if np.isnan(fit[p]) else fit[p] for p in picks]
        assert w == picks[int(np.argmin(keys))]     # strictly lower wins: first minimum
        assert s1.j == s2.j and s1.buf == s2.buf    # the same draws were consumed


def _well_formed(tokens):
    return oracle.tree_nodes(np.asarray(tokens, np.uint32)) == len(gp_ops.node_starts(tokens))


def test_subtrees_are_trees():
    progs = synth.ramped_half_and_half(5, 60, 2, 6, 64, funcs=synth.KDD_FUNCS, n_inputs=3,
                                       full_fallback_to_grow=True)
    for p in progs:
        p = [int(t) for t in p]
        for st in gp_ops.node_starts(p):
            sub = p[st:gp_ops.subtree_end(p, st)]
            assert _well_formed(sub)


PARAMS = dict(tournament=7, p_crossover=0.95, p_mutation=0.2, mutation_depth=4,
              funcs=list(synth.SHUTTLE_FUNCS), n_inputs=9, p_const=0.5, const_lo=-200.0,
              const_hi=200.0, max_nodes=255)


def test_crossover_and_mutation_keep_trees_well_formed():
    progs = [[int(t) for t in p] for p in synth.ramped_half_and_half(
        8, 64, 2, 7, 255, funcs=synth.SHUTTLE_FUNCS, n_inputs=9, const_lo=-200.0, const_hi=200.0,
        full_fallback_to_grow=True)]
    fit = np.random.default_rng(9).uniform(0, 1, len(progs))
    for g in range(3):
        kids = gp_ops.generation(progs, fit, g, 1234, PARAMS)
        for k in kids:
            assert _well_formed(k)
            assert len(gp_ops.node_starts(k)) <= PARAMS["max_nodes"]
        progs = kids


def test_crossover_accounts_for_every_node():
    progs = [[int(t) for t in p] for p in synth.ramped_half_and_half(12, 40, 2, 6, 64)]
    fit = np.zeros(len(progs))
    p = dict(PARAMS, p_crossover=1.0, p_mutation=0.0, funcs=list(synth.FLOAT_FUNCS), n_inputs=1)
    for i in range(40):
        child = gp_ops.offspring(progs, fit, i, 0, 77, p)
        # replay the draws: A, B, the two nodes
        s = gp_ops.Stream(77, i, 0)
        a = gp_ops.tournament(s, fit, 7)
        s.next()
        b = gp_ops.tournament(s, fit, 7)
        A, B = progs[a], progs[b]
        sa, sb = gp_ops.node_starts(A), gp_ops.node_starts(B)
        ia, ib = sa[s.uniform(len(sa))], sb[s.uniform(len(sb))]
        ea, eb = gp_ops.subtree_end(A, ia), gp_ops.subtree_end(B, ib)
        assert child[:ia] == A[:ia] and child[ia:ia + eb - ib] == B[ib:eb]
        assert child[ia + eb - ib:] == A[ea:]
        n = len(gp_ops.node_starts(A)) - len(gp_ops.node_starts(A[ia:ea])) + \
            len(gp_ops.node_starts(B[ib:eb]))
        assert len(gp_ops.node_starts(child)) == n


def test_no_variation_copies_the_tournament_winner():
    progs = [[int(t) for t in p] for p in synth.ramped_half_and_half(13, 30, 2, 5, 40)]
    fit = np.random.default_rng(14).uniform(0, 1, 30)
    p = dict(PARAMS, p_crossover=0.0, p_mutation=0.0)
    for i in range(30):
        s = gp_ops.Stream(5, i, 1)
        assert gp_ops.offspring(progs, fit, i, 1, 5, p) == progs[gp_ops.tournament(s, fit, 7)]


def test_size_cap_holds():
    big = [[int(t) for t in p] for p in synth.ramped_half_and_half(15, 20, 7, 7, 255)]
    fit = np.zeros(len(big))
    p = dict(PARAMS, funcs=list(synth.FLOAT_FUNCS), n_inputs=1, max_nodes=80)
    for i in range(20):
        k = gp_ops.offspring(big, fit, i, 0, 99, p)
        assert len(gp_ops.node_starts(k)) <= 80 or k in big   # over the cap: a parent's copy


@pytest.mark.parametrize("depth", [1, 2, 3, 4])
def test_grow_depth_and_constants(depth):
    for i in range(200):
        s = gp_ops.Stream(21, i, depth)
        t = gp_ops.grow(s, depth, list(synth.KDD_FUNCS), 41, gp_ops.threshold(0.5), -3.0, 5.0)
        assert _well_formed(t)
        # depth of a prefix tree: walk with a stack of remaining depths
        dmax, stack, j = 0, [1], 0
        while j < len(t):
            d = stack.pop()
            dmax = max(dmax, d)
            op = t[j] & 0xFF
            if op == gp_ops.CONST:
                v = np.uint32(t[j + 1]).view(np.float32)
                assert -3.0 <= v <= 5.0
                j += 2
                continue
            if op != gp_ops.VAR:
                stack.extend([d + 1] * gp_ops.ARITY[op])
            else:
                assert (t[j] >> 8) < 41
            j += 1
        assert dmax <= depth
        if depth >= 2:
            assert (t[0] & 0xFF) not in (gp_ops.VAR, gp_ops.CONST)   # the root is a function
