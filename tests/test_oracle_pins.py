"""Pins of the CPU oracle against the paper and against mathematics.

Nothing here compares the oracle with itself: every expected value is printed
in the paper (Fig. 2 and the examples around it, fixtures under
tests/golden/), follows from a closed form, or comes from an independent
method (brute force over memoryless controllers, min-max Dijkstra, matrix
exponential, scipy's adaptive integrator).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2001_06231_gb300 import workloads as wl

INF = math.inf


# --------------------------------------------------------------------------
# Fig. 2 worked example
# --------------------------------------------------------------------------

def load_fig2(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "fig2_example.json")))
    C, U = 7, 2
    boxes = np.zeros((C, U, 2, 1), dtype=np.int16)
    for ui, u in enumerate(g["inputs"]):
        for x, (lo, hi) in enumerate(g["boxes_lo_hi"][u]):
            boxes[x, ui, 0, 0] = lo
            boxes[x, ui, 1, 0] = hi
    G = np.array([[g["cost"][u][x] for u in g["inputs"]] for x in range(C)], dtype=np.float64)
    T = np.array(g["terminal"], dtype=np.float64)
    return g, boxes, G, T


def fig2_system(g):
    """Successor lists and g(x,y,u) straight from the fixture (no boxes)."""
    F = [[list(range(g["boxes_lo_hi"][u][x][0], g["boxes_lo_hi"][u][x][1] + 1))
          for u in g["inputs"]] for x in range(7)]
    cost = g["cost"]

    def gfun(x, y, u):
        assert y in F[x][u]
        return float(cost[g["inputs"][u]][x])
    T = [float(t) for t in g["terminal"]]
    return F, gfun, T


def test_fig2_final_controller_printed(golden_dir):
    g, boxes, G, T = load_fig2(golden_dir)
    r = oracle.solve([7], [False], boxes, G, T)
    assert r["status"] == oracle.CONVERGED
    code = {"U": oracle.HANDOVER, "b": 0, "g": 1}
    want = [code[g["printed"]["final_mu"][str(s)]] for s in range(1, 8)]
    assert r["mu"].tolist() == want


def test_fig2_frontiers_printed(golden_dir):
    g, boxes, G, T = load_fig2(golden_dir)
    r = oracle.solve([7], [False], boxes, G, T, max_iters=1)
    assert r["status"] == oracle.ITER_CAP and r["iters"] == 1
    assert r["f1"].tolist() == [7]                         # F1 = X after init
    f2 = sorted(int(c) + 1 for c in np.nonzero(r["f1_exit"])[0])
    assert f2 == g["printed"]["F2_after_round_1"]          # X \ {5}


def test_fig2_value_and_rounds(golden_dir):
    g, boxes, G, T = load_fig2(golden_dir)
    r = oracle.solve([7], [False], boxes, G, T)
    d = g["derived_by_hand"]
    assert r["V"].tolist() == d["V"]
    assert r["iters"] == d["iters"]
    assert r["changed"].tolist() == d["changed_per_round"]
    assert r["f1"].tolist() == d["F1_size_per_round"]


def test_fig2_cost_functional_printed(golden_dir):
    g, _, _, _ = load_fig2(golden_dir)
    F, gfun, T = fig2_system(g)
    b = 0
    x = [6, 3, 2, 2, 2, 2]          # states 7,4,3,3,...
    y = [6, 4, 0, 0, 0, 0]          # states 7,5,1,1,...
    u = [b] * 6
    v0, v1, v2 = [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]
    J = g["printed"]["J_values"]
    assert brute.cost_J(T, gfun, x, u, v0) == J["J(u,v0,x)"]
    assert brute.cost_J(T, gfun, x, u, v1) == J["J(u,v1,x)"]
    assert brute.cost_J(T, gfun, x, u, v2) == J["J(u,v2,x)"]
    assert brute.cost_J(T, gfun, y, u, v1) == J["J(u,v1,y)"]
    assert brute.cost_J(T, gfun, y, u, v2) == J["J(u,v2,y)"]
    assert brute.cost_J(T, gfun, x, u, [0, 0, 0, 0]) == INF


def test_fig2_closed_loop_performance_printed(golden_dir):
    g, _, _, _ = load_fig2(golden_dir)
    F, gfun, T = fig2_system(g)
    mu_b = [[0]] * 7
    assert brute.closed_loop_performance(F, T, gfun, 6, mu_b, horizon=10) == g["printed"]["L(7,mu=b)"]


def test_fig2_brute_force_matches(golden_dir):
    g, boxes, G, T = load_fig2(golden_dir)
    F, gfun, Tl = fig2_system(g)
    r = oracle.solve([7], [False], boxes, G, T)
    assert brute.brute_force_value(F, Tl, gfun) == r["V"].tolist()
    assert brute.performance(F, Tl, gfun, brute.controller_sets(r["mu"], 2)) == r["V"].tolist()
    # the recursion and the path enumeration agree on L(., mu = b)
    Lb = brute.performance(F, Tl, gfun, [[0]] * 7)
    for p in range(7):
        assert Lb[p] == brute.closed_loop_performance(F, Tl, gfun, p, [[0]] * 7, horizon=10)


# --------------------------------------------------------------------------
# brute force over memoryless controllers on random tiny abstractions
# --------------------------------------------------------------------------

def random_tiny(rng, nonneg=False):
    D = int(rng.integers(1, 3))
    n = [int(rng.integers(2, 4))] if D == 1 else [2, int(rng.integers(2, 4))]
    if D == 1:
        n = [int(rng.integers(3, 7))]
    periodic = [bool(rng.integers(0, 2)) for _ in range(D)]
    C = int(np.prod(n))
    U = int(rng.integers(1, 4))
    boxes = np.zeros((C, U, 2, D), dtype=np.int16)
    for x in range(C):
        for u in range(U):
            if rng.random() < 0.15:
                boxes[x, u, 0, 0] = oracle.BLOCKED
                continue
            for d in range(D):
                lo = int(rng.integers(0, n[d]))
                w = int(rng.integers(1, 3))
                hi = lo + w - 1
                if not periodic[d]:
                    hi = min(hi, n[d] - 1)
                boxes[x, u, 0, d] = lo
                boxes[x, u, 1, d] = hi
    lo_c = 0 if nonneg else -3
    G = rng.integers(lo_c, 6, size=(C, U)).astype(np.float64)
    G[rng.random((C, U)) < 0.1] = INF
    T = rng.integers(0, 6, size=C).astype(np.float64)
    T[rng.random(C) < 0.5] = INF
    return n, periodic, boxes, G, T


def test_pred_by_definition_tiny():
    """pred(y) = {x : exists u, y in F(x,u)} (Eq. (pred)) written out: every
    box of every pair enumerated cell by cell in Python (indexes wrapping on
    periodic dims, up to the whole circle; blocked pairs have no successor),
    against the oracle's CSR lists, which it also promises sorted by x."""
    import itertools
    rng = np.random.default_rng(2020)
    shapes = [([5], [False]), ([6], [True]), ([4, 3], [False, True]), ([3, 4], [True, True]),
              ([3, 4, 2], [True, False, True]), ([3, 2, 2, 3], [False, True, False, True])]
    for n, per in shapes:
        D, C, U = len(n), int(np.prod(n)), 3
        strides = np.concatenate([[1], np.cumprod(n)[:-1]]).astype(int)
        boxes = np.zeros((C, U, 2, D), dtype=np.int16)
        for x in range(C):
            for u in range(U):
                if rng.random() < 0.1:
                    boxes[x, u, 0, 0] = oracle.BLOCKED
                    continue
                for d in range(D):
                    w = int(rng.integers(1, n[d] + 1))
                    lo = int(rng.integers(0, n[d])) if per[d] else int(rng.integers(0, n[d] - w + 1))
                    boxes[x, u, 0, d], boxes[x, u, 1, d] = lo, lo + w - 1
        ptr, col = oracle.pred(n, per, boxes)
        expect = [set() for _ in range(C)]
        for x in range(C):
            for u in range(U):
                lo, hi = boxes[x, u, 0], boxes[x, u, 1]
                if lo[0] == oracle.BLOCKED:
                    continue
                axes = [[k % n[d] for k in range(lo[d], hi[d] + 1)] for d in range(D)]
                for y in itertools.product(*axes):
                    expect[int(np.dot(y, strides))].add(x)
        for y in range(C):
            got = col[ptr[y]:ptr[y + 1]].tolist()
            assert got == sorted(expect[y]), (n, per, y)


def test_brute_force_random_tiny():
    rng = np.random.default_rng(7)
    checked = 0
    for trial in range(60):
        n, periodic, boxes, G, T = random_tiny(rng, nonneg=(trial % 3 == 0))
        r = oracle.solve(n, periodic, boxes, G, T)
        if r["status"] != oracle.CONVERGED:
            continue
        F = brute.boxes_to_successors(n, periodic, boxes)
        gfun = lambda x, y, u: float(G[x, u])
        Tl = T.tolist()
        assert brute.brute_force_value(F, Tl, gfun) == r["V"].tolist(), trial
        U = boxes.shape[1]
        assert brute.performance(F, Tl, gfun, brute.controller_sets(r["mu"], U)) == r["V"].tolist(), trial
        checked += 1
    assert checked >= 30


def test_brute_force_tiny_3d_4d():
    """The brute force over static controllers on 3- and 4-D grids of 8 cells
    (dims of size 1 included, periodic or not): the oracle's cell indexing,
    box walk and predecessor lists in more than two dims."""
    rng = np.random.default_rng(34)
    shapes = [(2, 2, 2), (3, 1, 2), (2, 1, 2, 2), (1, 2, 2, 2), (2, 2, 1, 2)]
    checked = 0
    for trial in range(40):
        n = list(shapes[trial % len(shapes)])
        D, C, U = len(n), int(np.prod(n)), 2
        periodic = [bool(rng.integers(0, 2)) for _ in range(D)]
        boxes = np.zeros((C, U, 2, D), dtype=np.int16)
        for x in range(C):
            for u in range(U):
                if rng.random() < 0.1:
                    boxes[x, u, 0, 0] = oracle.BLOCKED
                    continue
                for d in range(D):
                    lo = int(rng.integers(0, n[d]))
                    hi = lo + min(int(rng.integers(0, 2)), n[d] - 1)     # at most the whole circle
                    if not periodic[d]:
                        hi = min(hi, n[d] - 1)
                    boxes[x, u, 0, d], boxes[x, u, 1, d] = lo, hi
        G = rng.integers(-1 if trial % 2 else 0, 5, size=(C, U)).astype(np.float64)
        T = rng.integers(0, 5, size=C).astype(np.float64)
        T[rng.random(C) < 0.5] = INF
        r = oracle.solve(n, periodic, boxes, G, T)
        if r["status"] != oracle.CONVERGED:
            continue
        F = brute.boxes_to_successors(n, periodic, boxes)
        gfun = lambda x, y, u: float(G[x, u])
        assert brute.brute_force_value(F, T.tolist(), gfun) == r["V"].tolist(), trial
        assert brute.performance(F, T.tolist(), gfun, brute.controller_sets(r["mu"], U)) == r["V"].tolist(), trial
        checked += 1
    assert checked >= 20


def test_successor_class_cost_brute_force():
    """Running cost that depends on the successor (Sec. VI-A, g2: a reward for
    successors in a set, another cost elsewhere), g(x,y,u) = Gc(x,u) for y in
    the class and G(x,u) else.  With non-negative costs the oracle's value is
    the brute-force value over memoryless controllers and its controller
    realizes it.  With negative costs it is a fixed point of the dynamic
    programming operator (Bellman check) no higher than that brute-force value:
    a cycle of negative cost that the adversary can leave for a dearer
    successor keeps Algorithm 1's values finite below what any memoryless
    controller attains (the adversary may also stay in the cycle, and a
    behaviour that never hands over costs +inf).  With every cell in the class
    (or none) the cost reduces to the plain Gc (or G)."""
    rng = np.random.default_rng(11)
    checked = exact = 0
    for trial in range(60):
        nonneg = trial % 3 == 0
        n, periodic, boxes, G, T = random_tiny(rng, nonneg=nonneg)
        C, U = boxes.shape[0], boxes.shape[1]
        cls = (rng.random(C) < 0.4).astype(np.uint8)
        Gc = rng.integers(0 if nonneg else -4, 3, size=(C, U)).astype(np.float64)
        r = oracle.solve(n, periodic, boxes, G, T, succ_class=cls, G_class=Gc)
        if r["status"] == oracle.CONVERGED:
            F = brute.boxes_to_successors(n, periodic, boxes)
            gfun = lambda x, y, u: float(Gc[x, u] if cls[y] else G[x, u])
            Tl = T.tolist()
            bv = brute.brute_force_value(F, Tl, gfun)
            if nonneg:
                assert bv == r["V"].tolist(), trial
                assert brute.performance(F, Tl, gfun, brute.controller_sets(r["mu"], U)) == r["V"].tolist(), trial
                exact += 1
            else:
                assert all(a <= b for a, b in zip(r["V"].tolist(), bv)), trial
            nbad, _ = oracle.bellman_check(n, periodic, boxes, G, T, None, r["V"], r["mu"],
                                           succ_class=cls, G_class=Gc)
            assert nbad == 0
            # the check sees a class-blind V as wrong when the class matters
            plain = oracle.solve(n, periodic, boxes, G, T)
            if plain["status"] == oracle.CONVERGED and not np.array_equal(plain["V"], r["V"]):
                nb2, _ = oracle.bellman_check(n, periodic, boxes, G, T, None, plain["V"], plain["mu"],
                                              succ_class=cls, G_class=Gc)
                assert nb2 > 0
            checked += 1
        for mask, cost in ((np.ones(C, np.uint8), Gc), (np.zeros(C, np.uint8), G)):
            a = oracle.solve(n, periodic, boxes, G, T, succ_class=mask, G_class=Gc)
            b = oracle.solve(n, periodic, boxes, cost, T)
            assert a["status"] == b["status"] and a["iters"] == b["iters"]
            assert np.array_equal(a["V"], b["V"]) and np.array_equal(a["mu"], b["mu"])
    assert checked >= 25 and exact >= 12


def full_sweep_rounds(n, periodic, boxes, G, T, rounds):
    """The dynamic programming operator of Eq. (dynamicprogramming) applied to
    every cell in every round (no frontier): W_{k+1}(x) = min(W_k(x), min_u
    G(x,u) + max_{y in F(x,u)} W_k(y)), blocked pairs +inf.  Returns the list
    W_0 .. W_rounds.  Written out cell by cell for tiny instances."""
    import itertools
    D, C, U = len(n), int(np.prod(n)), boxes.shape[1]
    stride = [int(np.prod(n[:d])) for d in range(D)]

    def cells(x, u):
        lo, hi = boxes[x, u, 0], boxes[x, u, 1]
        ranges = []
        for d in range(D):
            ranges.append([(int(lo[d]) + k) % n[d] if periodic[d] else int(lo[d]) + k
                           for k in range(int(hi[d]) - int(lo[d]) + 1)])
        return [sum(i * s for i, s in zip(t, stride)) for t in itertools.product(*ranges)]

    W = [np.array(T, dtype=np.float64)]
    for _ in range(rounds):
        prev = W[-1]
        nxt = prev.copy()
        for x in range(C):
            for u in range(U):
                if boxes[x, u, 0, 0] == oracle.BLOCKED:
                    continue
                d = G[x, u] + max(prev[y] for y in cells(x, u))
                if d < nxt[x]:
                    nxt[x] = d
        W.append(nxt)
    return W


def test_negative_cycle_reported_on_tiny_instances():
    """Where the oracle stops at the |X| cap (NEG_CYCLE) the plain operator,
    swept over every cell with no frontier, reaches the oracle's values after
    |X| rounds and its round |X| still lowered a value (the loop of Alg. 1
    exits with F1 non-empty).  Where it reports convergence after i rounds, the
    sweep is at a fixed point with the oracle's values from round i on.  (With
    negative costs the sweep may still settle after more than |X| rounds: the
    cap is the paper's test, not a proof of an endless descent.)"""
    rng = np.random.default_rng(11)
    seen = conv = settles = 0
    for _ in range(80):
        n, periodic, boxes, G, T = random_tiny(rng)
        C = int(np.prod(n))
        r = oracle.solve(n, periodic, boxes, G, T)
        W = full_sweep_rounds(n, periodic, boxes, G, T, 2 * C)
        if r["status"] == oracle.NEG_CYCLE:
            assert r["iters"] == C
            assert np.array_equal(W[C], r["V"])
            assert np.any(W[C] < W[C - 1])
            settles += int(np.array_equal(W[-1], W[-2]))
            # the oracle capped one round short stops with the state of round C - 1
            rc = oracle.solve(n, periodic, boxes, G, T, max_iters=C - 1)
            assert rc["status"] == oracle.ITER_CAP and rc["iters"] == C - 1
            assert np.array_equal(rc["V"], W[C - 1])
            seen += 1
        else:
            assert r["status"] == oracle.CONVERGED
            i = r["iters"]
            assert np.array_equal(W[i], r["V"]) and np.array_equal(W[-1], r["V"])
            conv += 1
    assert seen >= 3 and conv >= 20
    print("capped at |X|: %d instances, %d of them settle within 2|X| sweeps" % (seen, settles))


# --------------------------------------------------------------------------
# min-max Dijkstra (non-negative costs): bit-identical V
# --------------------------------------------------------------------------

def random_local(rng, n, U, reach=2, nonneg=True):
    D = len(n)
    C = int(np.prod(n))
    boxes = np.zeros((C, U, 2, D), dtype=np.int16)
    coords = np.stack(np.unravel_index(np.arange(C), tuple(reversed(n)))[::-1], axis=1)
    for x in range(C):
        for u in range(U):
            ok = True
            lo, hi = [], []
            for d in range(D):
                a = coords[x, d] + int(rng.integers(-reach, reach + 1))
                b = a + int(rng.integers(0, 3))
                if a < 0 or b >= n[d]:
                    ok = False
                lo.append(a)
                hi.append(b)
            if not ok:
                boxes[x, u, 0, 0] = oracle.BLOCKED
            else:
                boxes[x, u, 0, :] = lo
                boxes[x, u, 1, :] = hi
    G = rng.integers(0 if nonneg else -2, 8, size=(C, U)) * 0.125
    return boxes, G


def test_dijkstra_equals_bellman_ford_random():
    rng = np.random.default_rng(3)
    for trial in range(8):
        n = [int(rng.integers(6, 16)), int(rng.integers(6, 16))]
        U = int(rng.integers(1, 5))
        boxes, G = random_local(rng, n, U)
        C = int(np.prod(n))
        T = np.full(C, INF)
        T[rng.choice(C, size=3, replace=False)] = rng.integers(0, 4, size=3) * 0.5
        avoid = (rng.random(C) < 0.08).astype(np.uint8)
        r = oracle.solve(n, [False, False], boxes, G, T, avoid)
        assert r["status"] == oracle.CONVERGED
        Vd, _ = oracle.dijkstra(n, [False, False], boxes, G, T, avoid)
        assert np.array_equal(r["V"], Vd), trial


@pytest.mark.parametrize("n", [[9, 7, 6], [6, 5, 4, 4]])
def test_dijkstra_equals_bellman_ford_3d_4d(n):
    """Min-max Dijkstra and Algorithm 1 agree bit for bit on random 3- and
    4-D abstractions with non-negative costs."""
    rng = np.random.default_rng(len(n) * 17)
    D, C = len(n), int(np.prod(n))
    coords = np.stack(np.unravel_index(np.arange(C), tuple(reversed(n)))[::-1], axis=1)
    for trial in range(4):
        U = int(rng.integers(4, 7))
        # mostly one-cell boxes (a worst case over many cells rarely stays finite in 3-4 D)
        lo = coords[:, None, :] + rng.integers(-1, 2, size=(C, U, D))
        hi = lo + (rng.random((C, U, D)) < 0.1)
        ok = np.all((lo >= 0) & (hi < np.array(n)), axis=2)
        boxes = np.stack([lo, hi], axis=2).astype(np.int16)
        boxes[~ok, 0, 0] = oracle.BLOCKED
        G = rng.integers(0, 8, size=(C, U)) * 0.125
        T = np.full(C, INF)
        T[rng.choice(C, size=12, replace=False)] = rng.integers(0, 4, size=12) * 0.5
        avoid = (rng.random(C) < 0.05).astype(np.uint8)
        per = [False] * len(n)
        r = oracle.solve(n, per, boxes, G, T, avoid)
        assert r["status"] == oracle.CONVERGED
        Vd, _ = oracle.dijkstra(n, per, boxes, G, T, avoid)
        assert np.array_equal(r["V"], Vd), trial
        assert np.isfinite(r["V"]).sum() > C // 2              # the values spread past the targets


@pytest.mark.parametrize("tau", [0.1, 0.3])
def test_dijkstra_equals_bellman_ford_double_integrator(tau):
    w = wl.di2d(tau=tau)
    boxes = oracle.build_boxes(w.kind, w.params, w.substeps, w.grid.n, w.grid.lo, w.grid.hi,
                               w.grid.periodic, w.inputs, w.tau)
    T = w.terminal()
    r = oracle.solve(w.grid.n, w.grid.periodic, boxes, w.G, T, w.avoid)
    assert r["status"] == oracle.CONVERGED
    Vd, _ = oracle.dijkstra(w.grid.n, w.grid.periodic, boxes, w.G, T, w.avoid)
    assert np.array_equal(r["V"], Vd)
    tgt = w.target.astype(bool) & ~w.avoid.astype(bool)
    assert np.all(r["V"][tgt] == 0.0)
    if tau == 0.1:
        # In one 0.1 s step a cell moves by at most 0.5 cell widths in x1
        # unless |x2| > eta/tau, so every box off the target keeps its own
        # cell (a positive-cost self loop): V is finite on the target only and
        # Algorithm 1 stops after its first round.
        assert np.isfinite(r["V"]).sum() == tgt.sum() == 36
        assert r["iters"] == 1
    else:
        assert np.isfinite(r["V"]).sum() > 300 and r["iters"] > 10


# --------------------------------------------------------------------------
# closed forms on 1-D chains and rings
# --------------------------------------------------------------------------

def chain(nc, c, c2):
    boxes = np.zeros((nc, 2, 2, 1), dtype=np.int16)
    for k in range(nc):
        if k >= 1:
            boxes[k, 0, :, 0] = (k - 1, k - 1)         # "left by one"
        else:
            boxes[k, 0, 0, 0] = oracle.BLOCKED
        if k >= 2:
            boxes[k, 1, :, 0] = (k - 2, k - 1)         # nondeterministic: k-2 or k-1
        else:
            boxes[k, 1, 0, 0] = oracle.BLOCKED
    G = np.array([[c, c2]] * nc)
    T = np.full(nc, INF)
    T[0] = 0.0
    return boxes, G, T


def test_chain_closed_form():
    nc, c, c2 = 50, 0.375, 0.25
    boxes, G, T = chain(nc, c, c2)
    r = oracle.solve([nc], [False], boxes, G, T)
    # V(0) = 0, V(1) = c, V(k) = V(k-1) + min(c, c2) for k >= 2 (all dyadic)
    want = [0.0, c] + [c + (k - 1) * c2 for k in range(2, nc)]
    assert r["V"].tolist() == want
    assert r["mu"].tolist() == [oracle.HANDOVER, 0] + [1] * (nc - 2)
    assert r["iters"] == nc - 1
    assert r["changed"].tolist() == [1] * (nc - 1)


def test_negative_self_loop_closed_form():
    nc = 3
    boxes = np.zeros((nc, 1, 2, 1), dtype=np.int16)
    boxes[0, 0, :, 0] = (0, 0)        # self loop, cost -1
    boxes[1, 0, :, 0] = (0, 0)
    boxes[2, 0, :, 0] = (1, 1)
    G = np.array([[-1.0], [1.0], [1.0]])
    T = np.array([0.0, INF, INF])
    r = oracle.solve([nc], [False], boxes, G, T)
    assert r["status"] == oracle.NEG_CYCLE and r["iters"] == nc
    assert r["V"].tolist() == [-3.0, -1.0, 1.0]
    r = oracle.solve([nc], [False], boxes, G, T, max_iters=2)
    assert r["status"] == oracle.ITER_CAP and r["iters"] == 2
    assert r["V"].tolist() == [-2.0, 0.0, 2.0]


def test_periodic_ring_closed_form():
    nc, c = 9, 0.5
    # input 0: advance by one (wraps); input 1: {k+1, k+2} (wraps), cost 0.25
    boxes = np.zeros((nc, 2, 2, 1), dtype=np.int16)
    for k in range(nc):
        boxes[k, 0, :, 0] = ((k + 1) % nc, (k + 1) % nc)
        boxes[k, 1, :, 0] = ((k + 1) % nc, (k + 1) % nc + 1)
    G = np.array([[c, 0.25]] * nc)
    T = np.full(nc, INF)
    T[0] = 0.0
    r = oracle.solve([nc], [True], boxes, G, T)
    # distance to 0 going forward is (nc - k) steps; the wide input is only
    # safe where both successors are already finite
    V = r["V"]
    assert V[0] == 0.0 and V[nc - 1] == c
    for k in range(1, nc - 1):
        assert V[k] == V[k + 1] + min(c, 0.25) or V[k] == c + V[k + 1]
    F = brute.boxes_to_successors([nc], [True], boxes)
    assert brute.brute_force_value(F, T.tolist(), lambda x, y, u: float(G[x, u])) == V.tolist()


# --------------------------------------------------------------------------
# the Bellman checker itself must catch planted mistakes
# --------------------------------------------------------------------------

def test_bellman_check_catches_planted_errors(golden_dir):
    g, boxes, G, T = load_fig2(golden_dir)
    r = oracle.solve([7], [False], boxes, G, T)
    assert oracle.bellman_check([7], [False], boxes, G, T, None, r["V"], r["mu"]) == (0, -1)
    V = r["V"].copy()
    V[3] += 1.0
    assert oracle.bellman_check([7], [False], boxes, G, T, None, V, r["mu"])[0] >= 1
    mu = r["mu"].copy()
    mu[5] = 1                                   # the other input: not attaining
    assert oracle.bellman_check([7], [False], boxes, G, T, None, r["V"], mu) == (1, 5)
    mu = r["mu"].copy()
    mu[0] = 0                                   # hand-over cell given an input
    assert oracle.bellman_check([7], [False], boxes, G, T, None, r["V"], mu)[0] == 1


def test_avoid_cells_stay_infinite():
    nc = 6
    boxes, G, T = chain(nc, 1.0, 0.5)
    avoid = np.zeros(nc, dtype=np.uint8)
    avoid[3] = 1
    r = oracle.solve([nc], [False], boxes, G, T, avoid)
    assert r["V"][3] == INF and r["mu"][3] == oracle.HANDOVER
    assert np.all(np.isinf(r["V"][3:]))      # every path right of 3 crosses it
    assert r["V"][:3].tolist() == [0.0, 1.0, 1.5]


def test_oracle_input_rules():
    g_boxes = np.zeros((2, 1, 2, 1), dtype=np.int16)
    g_boxes[0, 0, :, 0] = (0, 0)
    g_boxes[1, 0, :, 0] = (0, 0)
    T = np.array([0.0, INF])
    with pytest.raises(ValueError):
        oracle.solve([2], [False], g_boxes, np.array([[np.nan], [1.0]]), T)
    with pytest.raises(ValueError):
        oracle.solve([2], [False], g_boxes, np.array([[-np.inf], [1.0]]), T)
    with pytest.raises(ValueError):
        oracle.solve([2], [False], g_boxes, np.array([[1e30], [1.0]]), T)
    r = oracle.solve([2], [False], g_boxes, np.array([[1.0], [-0.0]]), T)
    assert r["V"][1] == 0.0 and not math.copysign(1.0, r["V"][1]) < 0
    bad = g_boxes.copy()
    bad[1, 0, 1, 0] = 5                                   # hi outside the grid
    with pytest.raises(ValueError):
        oracle.solve([2], [False], bad, np.array([[1.0], [1.0]]), T)


# --------------------------------------------------------------------------
# abstraction builder (Sec. V-B)
# --------------------------------------------------------------------------

def _cells_of(points, lo, eta):
    return np.floor((points - lo) / eta).astype(np.int64)


def test_builder_double_integrator_sound_and_tight():
    from scipy.linalg import expm
    w = wl.di2d(n=(32, 32))
    g = w.grid
    boxes = oracle.build_boxes(w.kind, w.params, w.substeps, g.n, g.lo, g.hi, g.periodic, w.inputs, w.tau)
    # exact flow of (x0, x1, u)' = (x1, u, 0) by the matrix exponential
    A = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [0.0, 0.0, 0.0]])
    Phi = expm(A * w.tau)
    rng = np.random.default_rng(5)
    eta = np.array(g.eta)
    glo = np.array(g.lo)
    nblocked = 0
    for c in rng.choice(g.ncells, size=200, replace=False):
        k = np.array([c % g.n[0], c // g.n[0]])
        for ui, u in enumerate(w.inputs[:, 0]):
            corners = np.array([[glo[0] + (k[0] + a) * eta[0], glo[1] + (k[1] + b) * eta[1]]
                                for a in (0, 1) for b in (0, 1)])
            inner = glo + (k + rng.uniform(0.01, 0.99, size=(20, 2))) * eta
            pts = np.vstack([corners, inner])
            img = (Phi @ np.hstack([pts, np.full((len(pts), 1), u)]).T).T[:, :2]
            box = boxes[c, ui]
            cells = _cells_of(img, glo, eta)
            if box[0, 0] == oracle.BLOCKED:
                nblocked += 1
                assert (cells.min(axis=0) <= 0).any() or (cells.max(axis=0) >= np.array(g.n) - 1).any()
                continue
            # sound: every image lies in the box (1e-12 slack at cell edges)
            lo_f = glo + box[0] * eta
            hi_f = glo + (box[1] + 1) * eta
            assert np.all(img >= lo_f - 1e-12) and np.all(img <= hi_f + 1e-12)
            # tight: the extreme cells are reached by corner images
            ccell = _cells_of(img[:4], glo, eta)
            assert np.all(np.abs(ccell.min(axis=0) - box[0]) <= 1)
            assert np.all(np.abs(ccell.max(axis=0) - box[1]) <= 1)
            assert np.all(ccell.min(axis=0) >= box[0]) and np.all(ccell.max(axis=0) <= box[1])
    assert nblocked > 0


def test_builder_half_open_cells_exact_edges():
    """Quantisation on exact cell edges (half-open cells: a face on an edge
    takes the upper cell; a box past a non-periodic edge is blocked).  Unit
    cells, tau = 1: the double integrator maps cell [k0, k0+1] x [k1, k1+1]
    under u to x0 + x1 + u/2 in [k0+k1+u/2, k0+k1+2+u/2] and x1 + u in
    [k1+u, k1+1+u], every corner image an integer, so the box is
    [k0+k1+u/2, k0+k1+2+u/2] x [k1+u, k1+1+u], blocked once it leaves 0..7."""
    n = (8, 8)
    inputs = np.array([[0.0], [2.0], [-2.0]])
    boxes = oracle.build_boxes(oracle.LINEAR2D, (), 1, n, (0.0, 0.0), (8.0, 8.0), (False, False), inputs, 1.0)
    for c in range(64):
        k0, k1 = c % 8, c // 8
        for ui, u in enumerate(inputs[:, 0]):
            lo = (k0 + k1 + int(u) // 2, k1 + int(u))
            hi = (k0 + k1 + 2 + int(u) // 2, k1 + 1 + int(u))
            if min(lo) < 0 or max(hi) > 7:
                assert boxes[c, ui, 0, 0] == oracle.BLOCKED, (c, u)
            else:
                assert tuple(boxes[c, ui, 0]) == lo and tuple(boxes[c, ui, 1]) == hi, (c, u, boxes[c, ui])


@pytest.mark.parametrize("n0", [8, 3])
def test_builder_periodic_wrap_exact_edges(n0):
    """The same unit-cell double integrator with dim 0 periodic: the 3-cell
    range on dim 0 wraps (lower cell taken mod n0, upper = lower + 2, the
    indexes past n0 - 1 wrapping) and is the whole circle (0 .. n0 - 1) once
    3 >= n0; dim 1 still blocks past its edges."""
    n = (n0, 8)
    inputs = np.array([[0.0], [2.0], [-2.0]])
    boxes = oracle.build_boxes(oracle.LINEAR2D, (), 1, n, (0.0, 0.0), (float(n0), 8.0), (True, False), inputs, 1.0)
    for c in range(n0 * 8):
        k0, k1 = c % n0, c // n0
        for ui, u in enumerate(inputs[:, 0]):
            lo1, hi1 = k1 + int(u), k1 + 1 + int(u)
            if lo1 < 0 or hi1 > 7:
                assert boxes[c, ui, 0, 0] == oracle.BLOCKED, (c, u)
                continue
            if n0 <= 3:
                lo0, hi0 = 0, n0 - 1
            else:
                lo0 = (k0 + k1 + int(u) // 2) % n0
                hi0 = lo0 + 2
            assert tuple(boxes[c, ui, 0]) == (lo0, lo1) and tuple(boxes[c, ui, 1]) == (hi0, hi1), (c, u)


def test_builder_unicycle_centre_closed_form():
    rng = np.random.default_rng(9)
    for _ in range(40):
        th0 = rng.uniform(-math.pi, math.pi)
        v = rng.choice([0.5, 1.0])
        om = rng.choice([-1.0, -0.5, 0.0, 0.5, 1.0])
        tau = 0.3
        c0 = np.array([rng.uniform(0, 10), rng.uniform(0, 10), th0])
        r0 = np.array([0.025, 0.025, math.pi / 64])
        wd = 0.05
        c, r = oracle.flow(oracle.UNICYCLE3D, (wd,), 8, [v, om], tau, c0, r0)
        if om != 0.0:
            ex = c0[0] + v / om * (math.sin(th0 + om * tau) - math.sin(th0))
            ey = c0[1] - v / om * (math.cos(th0 + om * tau) - math.cos(th0))
        else:
            ex = c0[0] + v * tau * math.cos(th0)
            ey = c0[1] + v * tau * math.sin(th0)
        assert abs(c[0] - ex) < 1e-9 and abs(c[1] - ey) < 1e-9
        assert abs(c[2] - (th0 + om * tau)) < 1e-14
        # growth bound r' = L r + w, L = [[0,0,v],[0,0,v],[0,0,0]] in closed form
        rth = r0[2] + wd * tau
        rx = r0[0] + wd * tau + v * (r0[2] * tau + wd * tau * tau / 2)
        assert abs(r[2] - rth) < 1e-15
        assert abs(r[0] - rx) < 1e-15 and abs(r[1] - rx) < 1e-15


def test_builder_fire_flow_against_scipy():
    from scipy.integrate import solve_ivp
    from scipy.linalg import expm
    prm = (0.5, 9.81, 10.0, 20.0, 0.0)
    rng = np.random.default_rng(13)
    for _ in range(12):
        x0 = np.array([rng.uniform(100, 900), rng.uniform(100, 900), rng.uniform(-math.pi, math.pi),
                       rng.uniform(11.5, 18.5)])
        phi = math.radians(rng.choice([-30, -15, 0, 15, 30]))
        a = rng.choice([-1.0, 0.0, 1.0])

        def f(t, x):
            return [x[3] * math.cos(x[2]) + prm[0], x[3] * math.sin(x[2]),
                    prm[1] / x[3] * math.tan(phi), a]
        sol = solve_ivp(f, (0.0, 1.0), x0, method="DOP853", rtol=1e-13, atol=1e-12)
        r0 = np.array([5.0, 5.0, math.pi / 36, 0.625])
        c, r = oracle.flow(oracle.FIRE4D, prm, 8, [phi, a], 1.0, x0, r0)
        assert np.all(np.abs(c - sol.y[:, -1]) < 1e-6), (c, sol.y[:, -1])
        L = np.zeros((4, 4))
        L[0, 2] = L[1, 2] = prm[3]
        L[0, 3] = L[1, 3] = 1.0
        L[2, 3] = prm[1] * math.tan(abs(phi)) / prm[2] ** 2
        assert np.allclose(r, expm(L) @ r0, rtol=1e-13, atol=0)


@pytest.mark.parametrize("which", ["unicycle", "fire"])
def test_builder_sampled_soundness(which):
    from scipy.integrate import solve_ivp
    if which == "unicycle":
        w = wl.unicycle3d(n=(40, 40, 16), n_obstacles=0)
    else:
        w = wl.fire4d(n=(20, 20, 12, 4))
    g = w.grid
    boxes = oracle.build_boxes(w.kind, w.params, w.substeps, g.n, g.lo, g.hi, g.periodic, w.inputs, w.tau)
    rng = np.random.default_rng(17)
    eta = np.array(g.eta)
    glo = np.array(g.lo)
    n = np.array(g.n)
    checked = 0
    for c in rng.choice(g.ncells, size=60, replace=False):
        k = np.array(np.unravel_index(c, tuple(reversed(g.n)))[::-1])
        for ui in rng.choice(w.ninputs, size=3, replace=False):
            box = boxes[c, ui]
            if box[0, 0] == oracle.BLOCKED:
                continue
            u = w.inputs[ui]
            for _ in range(4):
                x0 = glo + (k + rng.uniform(0, 1, size=len(k))) * eta
                if which == "unicycle":
                    f = lambda t, x: [u[0] * math.cos(x[2]), u[0] * math.sin(x[2]), u[1]]
                else:
                    f = lambda t, x: [x[3] * math.cos(x[2]) + 0.5, x[3] * math.sin(x[2]),
                                      9.81 / x[3] * math.tan(u[0]), u[1]]
                sol = solve_ivp(f, (0.0, w.tau), x0, method="DOP853", rtol=1e-10, atol=1e-10)
                cell = _cells_of(sol.y[:, -1], glo, eta)
                for d in range(len(n)):
                    if g.periodic[d]:
                        off = (cell[d] - box[0, d]) % n[d]
                        assert off <= box[1, d] - box[0, d]
                    else:
                        assert box[0, d] <= cell[d] <= box[1, d]
                checked += 1
    assert checked > 100
