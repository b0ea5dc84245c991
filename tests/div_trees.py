"""Test inputs for divisions by constants: trees whose divisor (and numerator)
constants sit at and beyond the edges of the fast division range
[2^-50, 2^50], and fitness cases that put every kind of numerator (zeros,
subnormals, huge, infinite, NaN, ordinary) into some warps and keep others
ordinary.  Inputs only; no arithmetic of the method."""
import numpy as np

from synth import DIV, MUL, ADD, VAR, tok, const_tokens


def bitsf32(u):
    return float(np.array(u, np.uint32).view(np.float32))


# divisors at and beyond the edges of the fast range, both signs, and inside it
DIVISOR_EDGES = [2.0 ** -50, -(2.0 ** -50), 2.0 ** 50, -(2.0 ** 50), bitsf32(0x26800000 - 1),
                 bitsf32(0x58800000 + 1), 0.0, -0.0, 1e-40, float("inf"), float("nan"),
                 0.75, -1.5, 3.0, 1.0, 2.0 ** -49 * 1.25]
NUMERATORS = (0.5, 0.0, 2.0 ** 60, float("inf"))


def constant_divisor_trees(n_inputs=1):
    """x / c, (x*x) / c, c0 / c and ((x + c0) / c) / c for the edge divisors."""
    trees = []
    xv = [tok(VAR, n_inputs - 1)]
    for c in DIVISOR_EDGES:
        trees.append([tok(DIV)] + xv + const_tokens(c))
        trees.append([tok(DIV), tok(MUL)] + xv + xv + const_tokens(c))
        for c0 in NUMERATORS:
            trees.append([tok(DIV)] + const_tokens(c0) + const_tokens(c))
            trees.append([tok(DIV), tok(DIV), tok(ADD)] + xv + const_tokens(c0) + const_tokens(c)
                         + const_tokens(c))
    return [np.array(t, np.uint32) for t in trees]


def edge_cases(n_cases, seed, n_inputs=1):
    """Ordinary values U[-2, 2], with the special numerators placed in the
    first warps' cases (so those warps take the slow path) and none in the
    rest."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-2, 2, (n_inputs, n_cases)).astype(np.float32)
    special = np.array([0.0, -0.0, 1e-40, -1e-41, 2.0 ** 60, -(2.0 ** 55), float("inf"), float("-inf"),
                        float("nan"), 2.0 ** -50, 2.0 ** 50, bitsf32(0x26800000 - 1)], np.float32)
    for j, v in enumerate(special):
        x[:, (j * 37) % min(n_cases, 512)] = v
    return x
