"""Two CPU processes (gloo) run the multi-process reporting path: each rank
evaluates its shard of a population with the CPU oracle; the union of the
shards is the whole population exactly once, and the reductions give the
maximum time and the total work.  No GPU is used."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import synth
        from paper_1601_00221_gb300 import dist as gdist
        r, w = gdist.world()
        assert (r, w) == (rank, world)
        wl = synth.regression_small(seed=7, n_progs=37, n_cases=200)
        b, e = gdist.shard(wl.pop.n, r, w)
        f = oracle.population_fitness(wl.pop.words, wl.pop.offsets, wl.pop.lengths, wl.cases,
                                      wl.targets, p_range=(b, e))[b:e]
        gathered = [None] * w
        dist.all_gather_object(gathered, (b, e, f.tolist()))
        t_max = gdist.max_over_ranks(1.0 + r)
        units = gdist.sum_over_ranks(e - b)
        out_q.put((rank, gathered, t_max, units))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    import synth
    wl = synth.regression_small(seed=7, n_progs=37, n_cases=200)
    full = oracle.population_fitness(wl.pop.words, wl.pop.offsets, wl.pop.lengths, wl.cases,
                                     wl.targets)
    for rank, gathered, t_max, units in res:
        covered = np.concatenate([np.array(f) for _, _, f in sorted(gathered)])
        assert np.array_equal(covered, full)
        assert [(b, e) for b, e, _ in sorted(gathered)] == [(0, 19), (19, 37)]
        assert t_max == 2.0 and units == 37


def test_shard_ranges_cover_exactly_once():
    from paper_1601_00221_gb300 import dist as gdist
    for n in (0, 1, 7, 100):
        for w in (1, 2, 3, 8):
            seen = []
            for r in range(w):
                b, e = gdist.shard(n, r, w)
                seen.extend(range(b, e))
            assert seen == list(range(n))
