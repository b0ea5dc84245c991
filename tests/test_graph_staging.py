"""Host staging of the end-to-end graph (GenerationGraph with the device
encoder), on the CPU: the caller's words are staged as they are, with the
caller's offsets, when they fit the capacity; packed back to back otherwise;
and offsets or lengths that would make the device read outside the staged
words are rejected before anything is copied."""
import numpy as np
import pytest
import torch

import synth
from paper_1601_00221_gb300.graph import GenerationGraph


def staging(n, max_tokens):
    """A GenerationGraph reduced to its staging buffers (plain CPU tensors in
    place of the pinned ones; no device work)."""
    g = object.__new__(GenerationGraph)
    g.n, g.max_tokens = n, max_tokens
    g.h_tok = torch.zeros(max(max_tokens, 1), dtype=torch.int32)
    g.h_off = torch.zeros(n, dtype=torch.int64)
    g.h_len = torch.zeros(n, dtype=torch.int32)
    return g


def staged_programs(g, n):
    tok = g.h_tok.numpy().view(np.uint32)
    off, ln = g.h_off.numpy(), g.h_len.numpy()
    return [tok[off[p]: off[p] + ln[p]].tolist() for p in range(n)]


def test_packed_population_is_staged_as_it_is():
    pop = synth.pack(synth.ramped_half_and_half(401, 50, 1, 6, 63))
    g = staging(pop.n, int(pop.lengths.sum()))
    g._stage_trees(pop.words, pop.offsets, pop.lengths)
    assert np.array_equal(g.h_off.numpy(), pop.offsets)
    assert staged_programs(g, pop.n) == [pop.program(p).tolist() for p in range(pop.n)]


def test_reversed_and_gapped_layouts_keep_their_offsets_or_are_packed():
    pop = synth.pack(synth.ramped_half_and_half(402, 40, 1, 6, 63))
    n, total = pop.n, int(pop.lengths.sum())
    want = [pop.program(p).tolist() for p in range(n)]
    # reversed: same words, offsets descending -- staged as they are
    words = np.zeros(total, np.uint32)
    off = np.zeros(n, np.int64)
    pos = 0
    for p in reversed(range(n)):
        off[p] = pos
        words[pos: pos + pop.lengths[p]] = pop.program(p)
        pos += int(pop.lengths[p])
    g = staging(n, total)
    g._stage_trees(words, off, pop.lengths)
    assert np.array_equal(g.h_off.numpy(), off)
    assert staged_programs(g, n) == want
    # gaps past the capacity: packed back to back
    gap_off = pop.offsets + 3 * np.arange(n)
    gwords = np.zeros(total + 3 * n, np.uint32)
    for p in range(n):
        gwords[gap_off[p]: gap_off[p] + pop.lengths[p]] = pop.program(p)
    g = staging(n, total)
    g._stage_trees(gwords, gap_off, pop.lengths)
    assert np.array_equal(g.h_off.numpy(), np.concatenate([[0], np.cumsum(pop.lengths)[:-1]]))
    assert staged_programs(g, n) == want


def test_bad_layouts_are_rejected():
    pop = synth.pack(synth.ramped_half_and_half(403, 8, 1, 4, 15))
    total = int(pop.lengths.sum())
    g = staging(pop.n, total)
    neg = pop.offsets.copy()
    neg[3] = -1
    with pytest.raises(ValueError, match="negative"):
        g._stage_trees(pop.words, neg, pop.lengths)
    past = pop.offsets.copy()
    past[-1] += 1  # the last tree runs one word past the array
    with pytest.raises(ValueError, match="past the end"):
        g._stage_trees(pop.words, past, pop.lengths)
    small = staging(pop.n, total - 1)  # the encoded slots need every tree's words
    with pytest.raises(ValueError, match="capacity"):
        small._stage_trees(pop.words, pop.offsets, pop.lengths)
    # trees sharing words still count every word against the capacity
    shared = np.zeros(pop.n, np.int64)
    same = np.full(pop.n, int(pop.lengths.max()), np.int32)
    words = pop.program(int(np.argmax(pop.lengths))).copy()  # one tree, read by all
    tight = staging(pop.n, int(same[0]) * (pop.n - 1))
    with pytest.raises(ValueError, match="capacity"):
        tight._stage_trees(words, shared, same)
