"""Batched solve: every instance identical to its solo solve (and to the oracle).

Instances of different dimension, size, storage mode and cost structure are
solved in one bf_solve_batch call; V, mu, the pass count and the status of
each must equal a separate bf_solve on the same inputs, which the parity tests
tie to the CPU oracle.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2001_06231_gb300 as bf
from paper_2001_06231_gb300 import workloads as wl
from parity import import_boxes, oracle_boxes

pytestmark = pytest.mark.gpu


def test_batch_equals_solo_mixed_instances():
    ws = [wl.unicycle3d(n=(40, 36, 16), n_obstacles=5, seed=1),
          wl.unicycle3d(n=(70, 64, 24), n_obstacles=12, seed=2, cost_c=0.7),
          wl.di2d(tau=0.3),
          wl.di2d(),
          wl.fire4d(n=(30, 28, 24, 6), target=((50.0, 350.0), (50.0, 300.0), (-0.4, 0.4), (10.0, 15.0))),
          wl.unicycle3d(n=(50, 44, 20), n_obstacles=6, seed=3)]
    modes = [bf.MODE_STORED, bf.MODE_RECOMPUTE, bf.MODE_STORED, bf.MODE_RECOMPUTE, bf.MODE_STORED,
             bf.MODE_HYBRID]
    As = [bf.abs_build_workload(w, mode=m) if m != bf.MODE_HYBRID
          else bf.abs_build_workload(w, box_budget=4 * w.ncells * 8)          # 4 of 10 inputs stored
          for w, m in zip(ws, modes)]
    assert As[-1].mode == bf.MODE_HYBRID and As[-1].stored_inputs == 4
    solo = [bf.bf_solve(A, w.G, target=w.target, avoid=w.avoid) for A, w in zip(As, ws)]
    res = bf.bf_solve_batch(As, [w.G for w in ws], targets=[w.target for w in ws],
                            avoids=[w.avoid for w in ws])
    for r, s in zip(res, solo):
        assert r["iters"] == s["iters"] and r["status"] == s["status"]
        assert np.array_equal(r["V"], s["V"]) and np.array_equal(r["mu"], s["mu"])
    # an instance on the oracle's own boxes, in a batch, against the oracle directly
    w = ws[1]
    ob = oracle_boxes(w)
    Ao = import_boxes(w, ob)
    rb = bf.bf_solve_batch([Ao, As[0]], [w.G, ws[0].G], targets=[w.target, ws[0].target],
                           avoids=[w.avoid, ws[0].avoid])
    ref = oracle.solve(w.grid.n, w.grid.periodic, ob, w.G, w.terminal(), w.avoid)
    assert np.array_equal(rb[0]["V"], ref["V"]) and np.array_equal(rb[0]["mu"], ref["mu"])
    assert rb[0]["iters"] == ref["iters"]


def test_batch_same_abstraction_many_costs_and_caps():
    w = wl.unicycle3d(n=(50, 44, 16), n_obstacles=6)
    A = bf.abs_build_workload(w)
    rng = np.random.default_rng(3)
    Gs, tgs, terms = [], [], []
    for i in range(6):
        G = w.G * rng.uniform(0.5, 2.0) + (i % 3) * 0.01
        Gs.append(G)
        tgs.append(w.target)
    # terminal-cost instances mixed in, with a cap
    T = np.where(w.target.astype(bool), 0.0, math.inf)
    T[:100] = 1.5
    res = bf.bf_solve_batch([A] * 7, Gs + [w.G], targets=tgs + [None], avoids=[w.avoid] * 7,
                            terminals=[None] * 6 + [T], max_iters=40)
    for i in range(6):
        s = bf.bf_solve(A, Gs[i], target=tgs[i], avoid=w.avoid, max_iters=40)
        assert res[i]["iters"] == s["iters"] and res[i]["status"] == s["status"]
        assert np.array_equal(res[i]["V"], s["V"]) and np.array_equal(res[i]["mu"], s["mu"])
    s = bf.bf_solve(A, w.G, terminal=T, avoid=w.avoid, max_iters=40)
    assert np.array_equal(res[6]["V"], s["V"]) and res[6]["iters"] == s["iters"]


def test_batch_rejects_nan_instance():
    w = wl.di2d(tau=0.3)
    A = bf.abs_build_workload(w)
    G = w.G.copy()
    G[5, 2] = np.nan
    with pytest.raises(bf.BfError):
        bf.bf_solve_batch([A, A], [w.G, G], targets=[w.target, w.target], avoids=[w.avoid, w.avoid])


def test_batch_full_size_64_uneven_unicycles():
    """The measured batch: 64 unicycle instances of uneven size (44 M cells in
    all) in one bf_solve_batch, each identical to its solo solve."""
    ws = wl.batched(count=64)
    As = [bf.abs_build_workload(w) for w in ws]
    solo = [bf.bf_solve(A, w.G, target=w.target, avoid=w.avoid) for A, w in zip(As, ws)]
    res = bf.bf_solve_batch(As, [w.G for w in ws], targets=[w.target for w in ws],
                            avoids=[w.avoid for w in ws])
    for r, s in zip(res, solo):
        assert r["iters"] == s["iters"] and r["status"] == s["status"]
        assert np.array_equal(r["V"], s["V"]) and np.array_equal(r["mu"], s["mu"])


@pytest.mark.parametrize("sched", [
    dict(fuse_mark=-1, window33=1, plane_lists=1, templates=1, pair_inputs=1),
    dict(fuse_mark=1, window33=1, plane_lists=1, templates=1, pair_inputs=0),
    dict(fuse_mark=0, window33=1, plane_lists=1, templates=0, pair_inputs=1),
    dict(fuse_mark=0, window33=0, plane_lists=0, templates=1, pair_inputs=0),
    dict(fuse_mark=1, window33=0, plane_lists=1, templates=0, pair_inputs=1),
    dict(fuse_mark=0, window33=1, plane_lists=1, templates=1, pair_inputs=1, cell_masks=2),
    dict(fuse_mark=1, window33=1, plane_lists=1, templates=1, pair_inputs=0, cell_masks=2),
    dict(fuse_mark=-1, window33=0, plane_lists=1, templates=0, pair_inputs=1, cell_masks=2),
])
def test_batch_schedules_equal_solo_and_oracle(sched):
    """The batched form's schedules (3 x 3 window table, plane lookup lists and
    their kernel, predecessor templates, two inputs per iteration, marking in
    relax or a propagate launch, the relax by cell masks with the pairs queued
    over the lanes): every instance equal to its solo solve and the instances
    on the oracle's boxes equal to the oracle."""
    ws = [wl.unicycle3d(n=(40, 36, 16), n_obstacles=5, seed=1),
          wl.fire4d(n=(30, 28, 24, 6), target=((50.0, 350.0), (50.0, 300.0), (-0.4, 0.4), (10.0, 15.0))),
          wl.unicycle3d(n=(70, 64, 24), n_obstacles=12, seed=2, cost_c=0.7),
          wl.di2d(tau=0.3)]
    obs = [oracle_boxes(w) for w in ws]
    As = [import_boxes(w, ob) for w, ob in zip(ws, obs)]
    for A in As:
        bf.bf_set_batch_schedule(A, **sched)
    res = bf.bf_solve_batch(As, [w.G for w in ws], targets=[w.target for w in ws],
                            avoids=[w.avoid for w in ws])
    for r, w, ob in zip(res, ws, obs):
        ref = oracle.solve(w.grid.n, w.grid.periodic, ob, w.G, w.terminal(), w.avoid)
        assert r["iters"] == ref["iters"] and r["status"] == ref["status"]
        assert np.array_equal(r["V"], ref["V"]) and np.array_equal(r["mu"], ref["mu"])


def test_batch_tuner_keeps_results():
    ws = [wl.unicycle3d(n=(40, 36, 16), n_obstacles=5, seed=1 + i) for i in range(4)]
    As = [bf.abs_build_workload(w) for w in ws]
    solo = [bf.bf_solve(A, w.G, target=w.target, avoid=w.avoid) for A, w in zip(As, ws)]
    t = bf.bf_tune_batch(As, [w.G for w in ws], targets=[w.target for w in ws], avoids=[w.avoid for w in ws])
    assert t["candidates"] >= 6 and t["best_ms"] <= t["default_ms"]
    assert t["fuse_mark"] in (-1, 0, 1)
    res = bf.bf_solve_batch(As, [w.G for w in ws], targets=[w.target for w in ws], avoids=[w.avoid for w in ws])
    for r, s in zip(res, solo):
        assert r["iters"] == s["iters"] and np.array_equal(r["V"], s["V"]) and np.array_equal(r["mu"], s["mu"])
