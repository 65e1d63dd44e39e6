"""GPU parity at the measured sizes, in the launch configuration the benchmark
times (one graph launch per solve, device-resident inputs, compact records).
Both sides solve the oracle's boxes (imported into the library); the library's
own builder is compared with the oracle's on every box.

* Unicycle 200 x 200 x 64 x 10 inputs: the oracle solves to the fixed point;
  V, mu, the pass count, the status and the per-pass changed counts are
  compared bit for bit, and the Bellman checker runs on every cell.
* Fire model 100 x 100 x 36 x 8 x 15 inputs, the measured case (tau 2 s, wide
  landing box): the oracle solves to the fixed point (about 80 passes, some
  minutes of CPU); V, mu, the pass count, the status, the per-pass changed
  counts and the exact |F1| of every pass (counting mode) are compared, and the
  Bellman checker runs on every cell.
* Fire model as stated with tau 1 s and the narrow landing box: a degenerate
  instance (a few passes, few finite cells), compared the same way.
* Each also with the relax forms the tuner picks at these sizes (cell masks,
  the pairs queued over the lanes, the per-input frontier; marking in its own
  launch or in relax), against the same oracle solve.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2001_06231_gb300 as bf
from paper_2001_06231_gb300 import workloads as wl
from parity import import_boxes, mismatches, oracle_boxes

pytestmark = pytest.mark.gpu
INF = math.inf
FIRE_TARGET = ((50.0, 250.0), (50.0, 150.0), (-math.radians(30), math.radians(30)), (10.0, 15.0))


def same(a, b):
    return np.array_equal(np.asarray(a), np.asarray(b))


def gpu_solve(A, w, **kw):
    dev = torch.device("cuda", 0)
    G = torch.from_numpy(w.G).to(dev)
    tg = torch.from_numpy(w.target).to(dev)
    av = torch.from_numpy(w.avoid).to(dev)
    V = torch.empty(w.ncells, dtype=torch.float64, device=dev)
    mu = torch.empty(w.ncells, dtype=torch.uint8, device=dev)
    r = bf.bf_solve(A, G, target=tg, avoid=av, V=V, mu=mu, **kw)
    torch.cuda.synchronize()
    r["V"] = V.cpu().numpy()
    r["mu"] = mu.cpu().numpy()
    return r


def test_unicycle_full_size_bit_exact():
    w = wl.unicycle3d(seed=wl.SEED_BASE + 2)
    boxes = oracle_boxes(w)
    own = bf.abs_build_workload(w)
    mis = mismatches(own.export_boxes(), boxes)
    print("unicycle 200x200x64: %d of %d boxes differ from the oracle builder" % (mis, boxes.shape[0] * 10))
    assert mis <= 0.001 * boxes.shape[0] * boxes.shape[1]
    A = import_boxes(w, boxes)
    assert A.box_record_bytes == own.box_record_bytes == 8            # the measured record format
    res = gpu_solve(A, w, trace_cap=4096)
    T = w.terminal()
    ref = oracle.solve(w.grid.n, w.grid.periodic, boxes, w.G, T, w.avoid)
    assert res["status"] == ref["status"] == bf.CONVERGED
    assert res["iters"] == ref["iters"]
    assert same(res["V"], ref["V"]), np.nonzero(res["V"] != ref["V"])[0][:10]
    assert same(res["mu"], ref["mu"])
    k = ref["iters"]
    assert same(res["trace"][:k, 1], ref["changed"][:k])
    assert np.all(res["trace"][:k, 0] >= ref["f1"][:k])
    nbad, first = oracle.bellman_check(w.grid.n, w.grid.periodic, boxes, w.G, T, w.avoid, res["V"], res["mu"])
    assert nbad == 0, first
    tuned_forms_match(A, w, ref)
    # the value is finite on the target (0) and a decent share of the state space
    assert np.all(res["V"][w.target.astype(bool)] == 0.0)
    assert np.isfinite(res["V"]).sum() > 0.5 * w.ncells


def tuned_forms_match(A, w, ref):
    """The relax forms bf_tune picks at the measured sizes (cell masks, the
    pairs queued over the lanes, the per-input frontier; marking in its own
    launch or in relax) to the fixed point: the oracle's V, mu, pass count and
    per-pass changed counts, with fewer pairs taken up than every input of the
    frontier cells."""
    k = ref["iters"]
    for fuse in (0, 1):
        bf.bf_set_schedule(A, slice_target=0, fuse_mark=fuse, window33=1, plane_lists=1, templates=1,
                           pair_inputs=1, cell_masks=2, input_frontier=1)
        q = gpu_solve(A, w, trace_cap=8192)
        assert q["status"] == ref["status"] and q["iters"] == k, fuse
        assert same(q["V"], ref["V"]) and same(q["mu"], ref["mu"]), fuse
        assert same(q["trace"][:k, 1], ref["changed"][:k]), fuse
        assert np.all(q["trace"][:k, 0] >= ref["f1"][:k]), fuse
        assert q["stats"]["executed_pairs"] < int(ref["f1"].sum()) * w.ninputs, fuse
        print("tuned form, fuse %d: %d pairs taken up of %d canonical"
              % (fuse, q["stats"]["executed_pairs"], int(ref["f1"].sum()) * w.ninputs))


def fire_parity(w):
    boxes = oracle_boxes(w)
    A = import_boxes(w, boxes)
    assert A.box_record_bytes == 8
    T = w.terminal()
    ref = oracle.solve(w.grid.n, w.grid.periodic, boxes, w.G, T, w.avoid)
    res = gpu_solve(A, w, trace_cap=8192)
    assert res["status"] == ref["status"] == bf.CONVERGED
    assert res["iters"] == ref["iters"]
    assert same(res["V"], ref["V"]), np.nonzero(res["V"] != ref["V"])[0][:10]
    assert same(res["mu"], ref["mu"])
    k = ref["iters"]
    assert same(res["trace"][:k, 1], ref["changed"][:k])
    assert np.all(res["trace"][:k, 0] >= ref["f1"][:k])
    # counting mode: the exact F1 of every pass, found on the device from the bounding-box frontier
    cnt = gpu_solve(A, w, trace_cap=8192, count_exact=True)
    assert cnt["iters"] == k and same(cnt["V"], ref["V"]) and same(cnt["mu"], ref["mu"])
    assert same(cnt["trace"][:k, 3], ref["f1"][:k])
    nbad, first = oracle.bellman_check(w.grid.n, w.grid.periodic, boxes, w.G, T, w.avoid, res["V"], res["mu"])
    assert nbad == 0, first
    tuned_forms_match(A, w, ref)
    # negative costs over the fire; avoid cells stay +inf; V <= 0 on the target
    assert (w.G < 0).any()
    assert np.all(np.isinf(res["V"][w.avoid.astype(bool)]))
    assert np.all(res["V"][w.target.astype(bool)] <= 0.0)
    return res, ref


def test_fire_full_size_bit_exact_to_the_fixed_point():
    w = wl.fire4d(seed=wl.SEED_BASE + 3, tau=2.0, target=FIRE_TARGET)
    own = bf.abs_build_workload(w)
    mis = mismatches(own.export_boxes(), oracle_boxes(w))
    print("fire 100x100x36x8 tau 2: %d boxes differ from the oracle builder" % mis)
    assert mis <= 0.001 * w.ncells * w.ninputs
    res, ref = fire_parity(w)
    print("fire tau 2: %d passes, %d finite cells" % (ref["iters"], int(np.isfinite(ref["V"]).sum())))
    assert ref["iters"] > 40
    assert np.isfinite(res["V"]).sum() > 0.5 * w.ncells


def test_fire_full_size_as_stated_tau_1():
    """The 4-D configuration with tau = 1 s and the landing box [50,250] x [50,100]
    x [-10,10] deg x [10,12.5]: a 10 m cell moves about one cell per step, so few
    cells reach the target and the solve stops after a few passes."""
    w = wl.fire4d(seed=wl.SEED_BASE + 3)
    assert w.tau == 1.0
    own = bf.abs_build_workload(w)
    mis = mismatches(own.export_boxes(), oracle_boxes(w))
    print("fire 100x100x36x8 tau 1: %d boxes differ from the oracle builder" % mis)
    assert mis <= 0.001 * w.ncells * w.ninputs
    res, ref = fire_parity(w)
    print("fire tau 1: %d passes, %d finite cells" % (ref["iters"], int(np.isfinite(ref["V"]).sum())))
