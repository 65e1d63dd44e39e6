"""Served form: continuous batching gives every request the result it gets alone.

Requests over three systems (2-D, 3-D, 4-D; caller-owned and server-built
abstractions) are submitted in waves while earlier ones are still on the GPU;
each result must equal a solo bf_solve of the same inputs and the CPU oracle's
solve of the same boxes (exported from the library's builder, or the oracle's
own boxes imported into the library), bit for bit.  A small memory budget
forces the server to build a recompute-mode or hybrid abstraction, whose
results are compared with the oracle too, and a request that can never fit
completes with BF_ERR_OOM.
"""
import math
import time

import numpy as np
import pytest

import oracle
import paper_2001_06231_gb300 as bf
from paper_2001_06231_gb300 import workloads as wl
from parity import import_boxes, oracle_boxes

pytestmark = pytest.mark.gpu


def system_of(w):
    return (w.kind, w.params, w.substeps, w.grid, w.inputs, w.tau)


def oracle_of(w, boxes, G, tgt):
    T = np.where(np.asarray(tgt).astype(bool), 0.0, math.inf)
    return oracle.solve(w.grid.n, w.grid.periodic, boxes, G, T, w.avoid)


def same_result(r, ref):
    return (r["iters"] == ref["iters"] and r["status"] == ref["status"]
            and np.array_equal(r["V"], ref["V"]) and np.array_equal(r["mu"], ref["mu"]))


def test_results_alone_equal_results_in_the_mix():
    rng = np.random.default_rng(5)
    base = [wl.di2d(tau=0.3), wl.unicycle3d(n=(60, 56, 24), n_obstacles=8),
            wl.fire4d(n=(30, 28, 24, 6), target=((50.0, 350.0), (50.0, 300.0), (-0.4, 0.4), (10.0, 15.0)))]
    A_user = bf.abs_build_workload(base[1])                       # a caller-owned abstraction
    reqs = []
    for i in range(18):
        k = i % 3
        w = base[k]
        G = w.G * (1.0 + 0.25 * rng.integers(0, 4))
        tgt = w.target.copy()
        if k == 0:
            tgt = np.roll(tgt, int(rng.integers(-300, 300)))
            tgt &= 1 - w.avoid
        reqs.append((k, G, tgt))
    # the oracle's own boxes imported into the library: one request per system in the mix
    A_orc = [import_boxes(w, oracle_boxes(w)) for w in base]
    srv = bf.Server(hbm_budget=8 << 30, max_active=5, passes_per_step=4)
    ids = []
    for wave in range(3):                                          # later waves join a running engine
        for k, G, tgt in reqs[wave * 6:(wave + 1) * 6]:
            w = base[k]
            if k == 1 and wave % 2 == 0:
                rid = srv.submit(G, target=tgt, avoid=w.avoid, abstraction=A_user)
            else:
                rid = srv.submit(G, target=tgt, avoid=w.avoid, system=system_of(w))
            ids.append(rid)
        if wave == 1:
            orc_ids = [srv.submit(w.G, target=w.target, avoid=w.avoid, abstraction=A)
                       for w, A in zip(base, A_orc)]
        time.sleep(0.01)
    results = [srv.poll(rid, wait=True) for rid in ids]
    orc_results = [srv.poll(rid, wait=True) for rid in orc_ids]
    srv.close()
    solo_abs = [bf.abs_build_workload(w) for w in base]
    own_boxes = [A.export_boxes() for A in solo_abs]               # what the server's builder made too
    overlapped = 0
    for (k, G, tgt), r in zip(reqs, results):
        assert r["done"] == 1 and r["error"] == 0
        s = bf.bf_solve(solo_abs[k], G, target=tgt, avoid=base[k].avoid)
        assert same_result(r, s)
        assert same_result(r, oracle_of(base[k], own_boxes[k], G, tgt))
    for w, r in zip(base, orc_results):
        assert r["done"] == 1 and r["error"] == 0
        assert same_result(r, oracle_of(w, oracle_boxes(w), w.G, w.target))
    results = results + orc_results
    # requests really shared the device: some were admitted before others finished
    for a in results:
        for b in results:
            if a is not b and a["admit_s"] < b["finish_s"] and b["admit_s"] < a["finish_s"]:
                overlapped += 1
    assert overlapped > 0


def test_small_budget_builds_hybrid_or_recompute_mode_and_rejects_oversized():
    """Sec. IV-B memory control: at the smallest budget that admits the request
    the server builds a recompute-mode abstraction; with room for the records of
    3 more inputs it stores those and regenerates the rest (hybrid); results
    equal a stored-mode solve either way, and a budget below the smallest is
    refused with BF_ERR_OOM."""
    w = wl.unicycle3d(n=(60, 56, 24), n_obstacles=8)
    C = w.ncells
    S = bf.abs_build_workload(w)
    s = bf.bf_solve(S, w.G, target=w.target, avoid=w.avoid)
    ref = oracle_of(w, S.export_boxes(), w.G, w.target)
    assert same_result(s, ref)

    def serve(budget):
        srv = bf.Server(hbm_budget=budget, max_active=2)
        r = srv.poll(srv.submit(w.G, target=w.target, avoid=w.avoid, system=system_of(w)), wait=True)
        return srv, r

    lo, hi = 1 << 20, 1 << 30                   # refused at lo, admitted at hi
    while hi - lo > 1024:
        mid = (lo + hi) // 2
        srv, r = serve(mid)
        srv.close()
        if r["error"] == 0:
            hi = mid
        else:
            assert r["error"] == -2                                  # BF_ERR_OOM
            lo = mid
    for budget, mode in ((hi + 1024, bf.MODE_RECOMPUTE), (hi + 1024 + 3 * C * 8, bf.MODE_HYBRID)):
        srv, r = serve(budget)
        assert r["error"] == 0 and r["mode"] == mode, (r["error"], r["mode"], mode)
        assert same_result(r, ref)                                  # the oracle on the builder's boxes
        if mode == bf.MODE_RECOMPUTE:
            srv.close()
    big = wl.unicycle3d(n=(200, 200, 64), n_obstacles=0)
    rid = srv.submit(big.G, target=big.target, system=system_of(big))
    r = srv.poll(rid, wait=True)
    assert r["done"] == 1 and r["error"] == -2                      # BF_ERR_OOM
    srv.close()


def test_lone_requests_on_an_idle_server():
    """A request that finds the server idle runs at once as a plain solve (one
    graph launch); one at a time, then a burst that goes through the batched
    engine: every result equal to the oracle's on the same boxes."""
    base = [wl.di2d(tau=0.3), wl.unicycle3d(n=(60, 56, 24), n_obstacles=8),
            wl.fire4d(n=(30, 28, 24, 6), target=((50.0, 350.0), (50.0, 300.0), (-0.4, 0.4), (10.0, 15.0)))]
    own = [bf.abs_build_workload(w).export_boxes() for w in base]
    srv = bf.Server(hbm_budget=8 << 30, max_active=8, passes_per_step=4)
    for w, ob in zip(base, own):                       # one at a time: the idle path
        r = srv.poll(srv.submit(w.G, target=w.target, avoid=w.avoid, system=system_of(w)), wait=True)
        assert r["done"] == 1 and r["error"] == 0
        assert same_result(r, oracle_of(w, ob, w.G, w.target))
    ids = [srv.submit(w.G * 1.5, target=w.target, avoid=w.avoid, system=system_of(w)) for w in base * 2]
    res = [srv.poll(i, wait=True) for i in ids]
    srv.close()
    for r, w, ob in zip(res, base * 2, own * 2):
        assert r["done"] == 1 and r["error"] == 0
        assert same_result(r, oracle_of(w, ob, w.G * 1.5, w.target))
