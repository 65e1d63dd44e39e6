"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

V, mu, the pass count and the status must be identical (bit-exact FP64,
+inf included); the per-pass count of changed cells must match the
oracle's trace.  Both sides solve the same boxes: the GPU-built boxes are
exported and handed to the oracle.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import paper_2001_06231_gb300 as bf
from paper_2001_06231_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
INF = math.inf


def same(a, b):
    return np.array_equal(np.asarray(a), np.asarray(b))


def check_parity(n, periodic, boxes, G, terminal=None, target=None, avoid=None, max_iters=0, **kw):
    D = len(n)
    grid = bf.make_grid(n, [0.0] * D, [float(k) for k in n], periodic)
    A = bf.abs_from_boxes(grid, boxes)
    if terminal is None:
        terminal = np.where(np.asarray(target).astype(bool), 0.0, INF)
        res = bf.bf_solve(A, G, target=target, avoid=avoid, max_iters=max_iters, trace_cap=4096, **kw)
    else:
        res = bf.bf_solve(A, G, terminal=terminal, avoid=avoid, max_iters=max_iters, trace_cap=4096, **kw)
    ref = oracle.solve(n, periodic, boxes, G, terminal, avoid, max_iters=max_iters)
    assert res["status"] == ref["status"]
    assert res["iters"] == ref["iters"]
    assert same(res["V"], ref["V"]), np.nonzero(res["V"] != ref["V"])[0][:10]
    assert same(res["mu"], ref["mu"])
    k = min(len(ref["changed"]), len(res["trace"]))
    assert same(res["trace"][:k, 1], ref["changed"][:k])
    # the GPU frontier is a superset of the oracle's exact F1
    assert np.all(res["trace"][:k, 0] >= ref["f1"][:k])
    return res, ref


def test_fig2_worked_example(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "fig2_example.json")))
    boxes = np.zeros((7, 2, 2, 1), dtype=np.int16)
    for ui, u in enumerate(g["inputs"]):
        for x, (lo, hi) in enumerate(g["boxes_lo_hi"][u]):
            boxes[x, ui, :, 0] = (lo, hi)
    G = np.array([[g["cost"][u][x] for u in g["inputs"]] for x in range(7)], dtype=np.float64)
    T = np.array(g["terminal"], dtype=np.float64)
    res, _ = check_parity([7], [False], boxes, G, terminal=T)
    assert res["V"].tolist() == g["derived_by_hand"]["V"]
    assert res["iters"] == 3


def random_instance(rng, n, periodic, U, reach=2, width=3, neg=True, p_blocked=0.05):
    D = len(n)
    C = int(np.prod(n))
    coords = np.stack(np.unravel_index(np.arange(C), tuple(reversed(n)))[::-1], axis=1)
    boxes = np.zeros((C, U, 2, D), dtype=np.int16)
    shift = rng.integers(-reach, reach + 1, size=(U, D))
    for u in range(U):
        lo = coords + shift[u] + rng.integers(-1, 2, size=(C, D))
        w = rng.integers(0, width, size=(C, D))
        ok = rng.random(C) >= p_blocked
        for d in range(D):
            if periodic[d]:
                lo[:, d] %= n[d]
                w[:, d] = np.minimum(w[:, d], n[d] - 1)
            else:
                ok &= (lo[:, d] >= 0) & (lo[:, d] + w[:, d] <= n[d] - 1)
        hi = lo + w
        boxes[:, u, 0, :] = np.where(ok[:, None], lo, 0)
        boxes[:, u, 1, :] = np.where(ok[:, None], hi, 0)
        boxes[~ok, u, 0, 0] = bf.BLOCKED
    G = rng.integers(-1 if neg else 0, 6, size=(C, U)) * 0.25 + 0.125
    G[rng.random((C, U)) < 0.02] = INF
    target = (rng.random(C) < 0.01).astype(np.uint8)
    avoid = (rng.random(C) < 0.05).astype(np.uint8)
    return boxes, G, target, avoid


@pytest.mark.parametrize("n,periodic,U", [
    ([37], [False], 3), ([64], [True], 2),
    ([45, 29], [False, False], 5), ([33, 20], [False, True], 4),
    ([21, 17, 12], [False, False, True], 6), ([20, 9], [True, False], 3),
    ([70, 5, 6], [True, False, True], 4), ([300], [False], 2),
    ([13, 11, 9, 6], [False, False, True, False], 7),
])
def test_random_abstractions(n, periodic, U):
    rng = np.random.default_rng(hash((tuple(n), U)) % 2**32)
    boxes, G, target, avoid = random_instance(rng, n, periodic, U)
    res, ref = check_parity(n, periodic, boxes, G, target=target, avoid=avoid)
    assert res["iters"] >= 1


@pytest.mark.parametrize("n,periodic,reach", [([400], [False], 150), ([400, 6], [False, True], 150)])
def test_far_boxes_use_the_wide_records(n, periodic, reach):
    """Boxes whose offset from the cell exceeds the 8-bit relative records are
    kept as 16-bit absolute records; results are still those of the oracle."""
    rng = np.random.default_rng(len(n) * 1000 + reach)
    boxes, G, target, avoid = random_instance(rng, n, periodic, 3, reach=reach)
    res, ref = check_parity(n, periodic, boxes, G, target=target, avoid=avoid)
    assert res["iters"] >= 1


def test_exact_frontier_count_matches_oracle():
    """Counting mode reproduces |F1| of Algorithm 1 with the exact pred."""
    rng = np.random.default_rng(21)
    n, periodic = [30, 22, 9], [False, False, True]
    boxes, G, target, avoid = random_instance(rng, n, periodic, 5)
    A = bf.abs_from_boxes(bf.make_grid(n, [0, 0, 0], [30, 22, 9], periodic), boxes)
    res = bf.bf_solve(A, G, target=target, avoid=avoid, count_exact=True, trace_cap=4096)
    T = np.where(target.astype(bool), 0.0, INF)
    ref = oracle.solve(n, periodic, boxes, G, T, avoid)
    assert res["iters"] == ref["iters"] and same(res["V"], ref["V"])
    assert same(res["trace"][:, 3], ref["f1"])
    assert res["stats"]["exact_f1_cells"] == int(ref["f1"].sum())
    assert res["stats"]["changed_cells"] == int(ref["changed"].sum())
    rt = bf.bf_solve(A, G, target=target, avoid=avoid, time_kernels=True)
    assert same(rt["V"], ref["V"]) and rt["stats"]["relax_ms"] > 0


def test_host_loop_equals_graph():
    rng = np.random.default_rng(5)
    n, periodic = [40, 30], [False, False]
    boxes, G, target, avoid = random_instance(rng, n, periodic, 4)
    A = bf.abs_from_boxes(bf.make_grid(n, [0, 0], [40, 30], periodic), boxes)
    r1 = bf.bf_solve(A, G, target=target, avoid=avoid)
    r2 = bf.bf_solve(A, G, target=target, avoid=avoid, host_loop=True)
    assert same(r1["V"], r2["V"]) and same(r1["mu"], r2["mu"]) and r1["iters"] == r2["iters"]


def test_negative_cycle_and_cap():
    nc = 50
    boxes = np.zeros((nc, 1, 2, 1), dtype=np.int16)
    boxes[0, 0, :, 0] = (0, 0)
    for k in range(1, nc):
        boxes[k, 0, :, 0] = (k - 1, k - 1)
    G = np.ones((nc, 1))
    G[0, 0] = -1.0
    T = np.full(nc, INF)
    T[0] = 0.0
    res, _ = check_parity([nc], [False], boxes, G, terminal=T)
    assert res["status"] == bf.NEG_CYCLE and res["iters"] == nc
    res, _ = check_parity([nc], [False], boxes, G, terminal=T, max_iters=7)
    assert res["status"] == bf.ITER_CAP and res["iters"] == 7


def test_invalid_costs_rejected():
    n = [10]
    boxes = np.zeros((10, 1, 2, 1), dtype=np.int16)
    A = bf.abs_from_boxes(bf.make_grid(n), boxes)
    T = np.zeros(10)
    for bad in (np.nan, -np.inf, 1e300):
        G = np.ones((10, 1))
        G[3, 0] = bad
        with pytest.raises(bf.BfError):
            bf.bf_solve(A, G, terminal=T)
    bad_boxes = boxes.copy()
    bad_boxes[2, 0, 1, 0] = 12
    with pytest.raises(bf.BfError):
        bf.abs_from_boxes(bf.make_grid(n), bad_boxes)


def builder_parity(w, mode=bf.MODE_STORED):
    A = bf.abs_build_workload(w, mode=mode)
    gb = A.export_boxes()
    ob = oracle.build_boxes(w.kind, w.params, w.substeps, w.grid.n, w.grid.lo, w.grid.hi,
                            w.grid.periodic, w.inputs, w.tau)
    mismatch = int(np.any(gb != ob, axis=(2, 3)).sum())
    return A, gb, mismatch


@pytest.mark.parametrize("which", ["di2d", "di2d_tau03", "unicycle", "fire"])
def test_builder_and_solver_parity(which):
    if which == "di2d":
        w = wl.di2d()
    elif which == "di2d_tau03":
        w = wl.di2d(tau=0.3)
    elif which == "unicycle":
        w = wl.unicycle3d(n=(60, 50, 24), n_obstacles=8)
    else:
        w = wl.fire4d(n=(30, 28, 24, 6), target=((50.0, 350.0), (50.0, 300.0), (-0.4, 0.4), (10.0, 15.0)))
    A, gb, mismatch = builder_parity(w)
    print("%s: %d of %d boxes differ from the oracle builder" % (which, mismatch, gb.shape[0] * gb.shape[1]))
    if w.kind == bf.LINEAR2D:
        assert mismatch == 0
    else:
        assert mismatch <= 0.001 * gb.shape[0] * gb.shape[1]
    res = bf.bf_solve(A, w.G, target=w.target, avoid=w.avoid, trace_cap=10000)
    ref = oracle.solve(w.grid.n, w.grid.periodic, gb, w.G, w.terminal(), w.avoid)
    assert res["status"] == ref["status"] and res["iters"] == ref["iters"]
    assert same(res["V"], ref["V"]) and same(res["mu"], ref["mu"])
    # recompute mode regenerates bit-identical boxes and results
    R = bf.abs_build_workload(w, mode=bf.MODE_RECOMPUTE)
    assert same(R.export_boxes(), gb)
    rr = bf.bf_solve(R, w.G, target=w.target, avoid=w.avoid)
    assert same(rr["V"], res["V"]) and same(rr["mu"], res["mu"]) and rr["iters"] == res["iters"]


def check_inplace(n, periodic, boxes, G, terminal, avoid, A=None):
    """In-place passes: the oracle's (Jacobi) V bit for bit, no more passes, and
    a controller that attains V (Bellman check); negative cycles still hit the cap."""
    D = len(n)
    if A is None:
        A = bf.abs_from_boxes(bf.make_grid(n, [0.0] * D, [float(k) for k in n], periodic), boxes)
    ref = oracle.solve(n, periodic, boxes, G, terminal, avoid)
    r = bf.bf_solve(A, G, terminal=terminal, avoid=avoid, schedule=bf.SCHED_INPLACE)
    if ref["status"] != bf.CONVERGED:
        assert r["status"] == ref["status"]
        return r, ref
    assert r["status"] == bf.CONVERGED
    assert same(r["V"], ref["V"]), np.nonzero(r["V"] != ref["V"])[0][:10]
    assert r["iters"] <= ref["iters"]
    nbad, first = oracle.bellman_check(n, periodic, boxes, G, terminal, avoid, r["V"], r["mu"])
    assert nbad == 0, first
    return r, ref


@pytest.mark.parametrize("n,periodic,U,neg", [
    ([45, 29], [False, False], 5, False), ([21, 17, 12], [False, False, True], 6, False),
    ([13, 11, 9, 6], [False, False, True, False], 7, False), ([300], [False], 2, False),
    ([33, 20], [False, True], 4, True), ([70, 5, 6], [True, False, True], 4, True),
])
def test_inplace_schedule_reaches_the_same_value(n, periodic, U, neg):
    rng = np.random.default_rng(hash((tuple(n), U, neg, "inplace")) % 2**32)
    boxes, G, target, avoid = random_instance(rng, n, periodic, U, neg=neg)
    terminal = np.where(target.astype(bool), 0.0, INF)
    check_inplace(n, periodic, boxes, G, terminal, avoid)


@pytest.mark.parametrize("which", ["unicycle", "fire"])
def test_inplace_schedule_builder_workloads(which):
    if which == "unicycle":
        w = wl.unicycle3d(n=(60, 50, 24), n_obstacles=8)
    else:
        w = wl.fire4d(n=(30, 28, 24, 6), target=((50.0, 350.0), (50.0, 300.0), (-0.4, 0.4), (10.0, 15.0)))
    A = bf.abs_build_workload(w)
    r, ref = check_inplace(w.grid.n, w.grid.periodic, A.export_boxes(), w.G, w.terminal(), w.avoid, A=A)
    # Jacobi again on the same handle: the graph is rebuilt for the schedule
    j = bf.bf_solve(A, w.G, target=w.target, avoid=w.avoid)
    assert j["iters"] == ref["iters"] and same(j["V"], ref["V"]) and same(j["mu"], ref["mu"])
    print("%s: %d in-place passes vs %d Jacobi passes" % (which, r["iters"], ref["iters"]))


@pytest.mark.parametrize("which", ["unicycle", "fire"])
def test_hybrid_mode_is_bit_identical(which):
    """Memory-regulated builds: the records of the first K inputs are stored, the
    rest regenerated in relax; boxes and results equal the stored mode's for
    every K, and device memory grows with K."""
    if which == "unicycle":
        w = wl.unicycle3d(n=(60, 50, 24), n_obstacles=8)
    else:
        w = wl.fire4d(n=(30, 28, 24, 6), target=((50.0, 350.0), (50.0, 300.0), (-0.4, 0.4), (10.0, 15.0)))
    S = bf.abs_build_workload(w)
    gb = S.export_boxes()
    ref = bf.bf_solve(S, w.G, target=w.target, avoid=w.avoid)
    C, U = w.ncells, w.ninputs
    rec = 4 if w.grid.ndim <= 2 else 8
    sizes = []
    for K in (0, 1, U // 2, U - 1, U):
        H = bf.abs_build_workload(w, box_budget=K * C * rec + rec * C // 2)
        assert H.stored_inputs == K
        assert H.mode == (bf.MODE_RECOMPUTE if K == 0 else bf.MODE_STORED if K == U else bf.MODE_HYBRID)
        assert same(H.export_boxes(), gb)
        r = bf.bf_solve(H, w.G, target=w.target, avoid=w.avoid)
        assert r["iters"] == ref["iters"] and r["status"] == ref["status"]
        assert same(r["V"], ref["V"]) and same(r["mu"], ref["mu"])
        sizes.append(H.device_bytes)
    assert sizes == sorted(sizes) and sizes[0] < sizes[-1]
    with pytest.raises(bf.BfError):
        bf.abs_build_workload(w, box_budget=-1)
