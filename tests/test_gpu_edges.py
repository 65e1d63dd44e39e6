"""Edge cases of the solve through the C ABI, against the oracle (both sides on
the same test-made boxes): no finite terminal cost, a single cell, a single
and the largest number of inputs, the largest extent of one dimension (a long
chain: one pass per cell), and a 16.7 M-cell grid."""
import math

import numpy as np
import pytest

import oracle
import paper_2001_06231_gb300 as bf

pytestmark = pytest.mark.gpu
INF = math.inf


def same(a, b):
    return np.array_equal(np.asarray(a), np.asarray(b))


def solve_both(n, periodic, boxes, G, terminal, avoid=None, **kw):
    D = len(n)
    A = bf.abs_from_boxes(bf.make_grid(n, [0.0] * D, [float(k) for k in n], periodic), boxes)
    res = bf.bf_solve(A, G, terminal=terminal, avoid=avoid, **kw)
    ref = oracle.solve(n, periodic, boxes, G, terminal, avoid, **kw)
    assert res["status"] == ref["status"] and res["iters"] == ref["iters"]
    assert same(res["V"], ref["V"]) and same(res["mu"], ref["mu"])
    return res, ref


def shift_boxes(n, U, shifts, width=1):
    """1-D boxes [x + s, x + s + width - 1] per input shift s (blocked when off the grid)."""
    C = n
    boxes = np.zeros((C, U, 2, 1), dtype=np.int16)
    x = np.arange(C)
    for u, s in enumerate(shifts):
        lo, hi = x + s, x + s + width - 1
        ok = (lo >= 0) & (hi <= C - 1)
        boxes[:, u, 0, 0] = np.where(ok, lo, bf.BLOCKED)
        boxes[:, u, 1, 0] = np.where(ok, hi, 0)
    return boxes


def test_no_finite_terminal_cost():
    boxes = shift_boxes(50, 2, (1, -1))
    res, _ = solve_both([50], [False], boxes, np.ones((50, 2)), np.full(50, INF))
    assert res["iters"] == 0 and np.all(np.isinf(res["V"])) and np.all(res["mu"] == 0xFF)


def test_single_cell():
    boxes = np.zeros((1, 1, 2, 1), dtype=np.int16)          # its own successor
    res, _ = solve_both([1], [False], boxes, np.full((1, 1), 0.5), np.array([3.0]))
    assert res["V"][0] == 3.0 and res["status"] == bf.CONVERGED
    res, _ = solve_both([1], [False], boxes, np.full((1, 1), -0.5), np.array([3.0]))
    assert res["status"] == bf.NEG_CYCLE                       # |X| = 1 pass and still changing


@pytest.mark.parametrize("U", [1, 254])
def test_fewest_and_most_inputs(U):
    rng = np.random.default_rng(U)
    n = 300
    shifts = rng.integers(-3, 4, size=U)
    boxes = shift_boxes(n, U, shifts, width=2)
    G = rng.integers(1, 9, size=(n, U)) * 0.25
    T = np.full(n, INF)
    T[[0, n // 2, n - 1]] = 0.0
    solve_both([n], [False], boxes, G, T)


def test_longest_dimension_chain():
    """n = 16383 cells on one dim (the largest extent), a chain toward cell 0:
    one pass per cell."""
    n = 16383
    boxes = shift_boxes(n, 1, (-1,))
    T = np.full(n, INF)
    T[0] = 0.0
    res, _ = solve_both([n], [False], boxes, np.ones((n, 1)), T)
    assert res["iters"] == n - 1 and res["status"] == bf.CONVERGED
    assert res["V"][n - 1] == float(n - 1)


def test_large_grid_random_boxes():
    """8192 x 2048 = 16.7 M cells, 2 inputs, random nearby boxes."""
    n = [8192, 2048]
    C = n[0] * n[1]
    rng = np.random.default_rng(5)
    boxes = np.zeros((C, 2, 2, 2), dtype=np.int16)
    k0 = np.tile(np.arange(n[0]), n[1])
    k1 = np.repeat(np.arange(n[1]), n[0])
    for u, (s0, s1) in enumerate(((-2, 0), (0, -2))):
        lo0 = k0 + s0 + rng.integers(-1, 1, size=C)
        lo1 = k1 + s1 + rng.integers(-1, 1, size=C)
        ok = (lo0 >= 0) & (lo1 >= 0) & (lo0 + 1 <= n[0] - 1) & (lo1 + 1 <= n[1] - 1)
        boxes[:, u, 0, 0] = np.where(ok, lo0, bf.BLOCKED)
        boxes[:, u, 0, 1] = np.where(ok, lo1, 0)
        boxes[:, u, 1, 0] = np.where(ok, lo0 + 1, 0)
        boxes[:, u, 1, 1] = np.where(ok, lo1 + 1, 0)
    G = rng.integers(1, 5, size=(C, 2)).astype(np.float64)
    T = np.full(C, INF)
    T[: n[0] * 4] = 0.0                                      # the first rows are the target
    res, _ = solve_both(n, [False, False], boxes, G, T, max_iters=40)
    assert res["status"] == bf.ITER_CAP
