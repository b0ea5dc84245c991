"""Helpers of the GPU parity tests: upload, compare, oracle calls."""
import numpy as np

import oracle
import paper_1601_00221_gb300 as gp

REL_TOL = 1e-5  # float fitness vs the binary64 oracle (relative)


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def upload(enc):
    return enc.to_device("cuda")


def same_bits(a, b):
    a = np.asarray(a, np.float32)
    b = np.asarray(b, np.float32)
    both_nan = np.isnan(a) & np.isnan(b)
    return (a.view(np.uint32) == b.view(np.uint32)) | both_nan


def assert_bits(got, exp, what=""):
    ok = same_bits(got, exp)
    if not np.all(ok):
        idx = np.argwhere(~ok)[:5]
        raise AssertionError(f"{what}: {int((~ok).sum())} mismatches, first at {idx.tolist()}: "
                             f"got {np.asarray(got)[tuple(idx[0])]!r} exp {np.asarray(exp)[tuple(idx[0])]!r}")


def assert_fitness(got, exp, what=""):
    got = np.asarray(got, np.float64)
    exp = np.asarray(exp, np.float64)
    for i, (g, e) in enumerate(zip(got, exp)):
        if np.isnan(e):
            assert np.isnan(g), f"{what} program {i}: got {g}, oracle NaN"
        elif np.isinf(e) or e == 0.0:
            assert g == e, f"{what} program {i}: got {g}, oracle {e}"
        else:
            rel = abs(g - e) / abs(e)
            assert rel <= REL_TOL, f"{what} program {i}: got {g!r}, oracle {e!r}, rel {rel:.3g}"


def rel_errors(got, exp):
    got = np.asarray(got, np.float64)
    exp = np.asarray(exp, np.float64)
    m = np.isfinite(exp) & (exp != 0)
    return np.abs(got[m] - exp[m]) / np.abs(exp[m])


def oracle_outputs(pop, x):
    return np.stack([oracle.tree_outputs(pop.program(p), x) for p in range(pop.n)])
