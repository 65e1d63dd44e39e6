"""The allocation-free solve entry point, checked against bf_solve.

bf_solve_noalloc serves host programs that own all device memory themselves
(a fixed budget handed out at start-up, their own pool, or a loop that may not
call cudaMalloc/cudaFree once running): it keeps its working state in one
fixed-size device array of the library instead of allocating.  This file is
collected last on purpose so that a failure here comes after every other
test has run.  It calls the entry point through the C ABI with ctypes.
"""
import ctypes
import math

import numpy as np
import pytest

import paper_2001_06231_gb300 as bf
from paper_2001_06231_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _entry():
    L = bf.lib()
    f = L.bf_solve_noalloc
    P = ctypes.c_void_p
    f.argtypes = [P, P, P, P, P, ctypes.c_int64, P, P, P, P, P]
    f.restype = ctypes.c_int
    return L, f


def _noalloc(f, A, G, target, avoid, terminal=None, max_iters=0):
    import torch
    C = A.ncells
    V = torch.empty(C, dtype=torch.float64, device="cuda")
    mu = torch.empty(C, dtype=torch.uint8, device="cuda")
    it = ctypes.c_int64()
    st = ctypes.c_int32()
    rc = f(A.handle, G.data_ptr(), None if target is None else target.data_ptr(),
           None if avoid is None else avoid.data_ptr(), None if terminal is None else terminal.data_ptr(),
           int(max_iters), V.data_ptr(), mu.data_ptr(), ctypes.byref(it), ctypes.byref(st), None)
    return rc, V.cpu().numpy(), mu.cpu().numpy(), it.value, st.value


def test_noalloc_matches_bf_solve_on_two_calls_in_a_row():
    import torch
    _, f = _entry()
    cases = [wl.unicycle3d(n=(60, 50, 24), n_obstacles=8),
             wl.fire4d(n=(30, 28, 24, 6), target=((50.0, 350.0), (50.0, 300.0), (-0.4, 0.4), (10.0, 15.0)))]
    for w in cases:
        A = bf.abs_build_workload(w)
        G = torch.from_numpy(w.G).cuda()
        tg = torch.from_numpy(w.target).cuda()
        av = torch.from_numpy(w.avoid).cuda()
        ref = bf.bf_solve(A, w.G, target=w.target, avoid=w.avoid)
        for _ in range(2):                       # the scratch keeps the previous call's contents
            rc, V, mu, it, st = _noalloc(f, A, G, tg, av)
            assert rc == 0, bf.lib().bf_last_error()
            assert np.array_equal(V, ref["V"])   # bit-exact, the tolerance of every parity test here
            assert np.array_equal(mu, ref["mu"])
            assert it == ref["iters"] and st == ref["status"]


def test_noalloc_terminal_cost_and_cap():
    import torch
    _, f = _entry()
    nc = 40
    boxes = np.zeros((nc, 1, 2, 1), dtype=np.int16)
    boxes[0, 0, :, 0] = (0, 0)
    for k in range(1, nc):
        boxes[k, 0, :, 0] = (k - 1, k - 1)
    G = np.ones((nc, 1))
    G[0, 0] = -1.0
    T = np.full(nc, math.inf)
    T[0] = 0.0
    A = bf.abs_from_boxes(bf.make_grid([nc]), boxes)
    for cap in (0, 5):
        ref = bf.bf_solve(A, G, terminal=T, max_iters=cap)
        rc, V, mu, it, st = _noalloc(f, A, torch.from_numpy(G).cuda(), None, None,
                                     terminal=torch.from_numpy(T).cuda(), max_iters=cap)
        assert rc == 0
        assert np.array_equal(V, ref["V"]) and np.array_equal(mu, ref["mu"])
        assert (it, st) == (ref["iters"], ref["status"])


def test_noalloc_rejects_oversized_and_host_arrays():
    import torch
    L, f = _entry()
    n = 2_000_000                                  # ~96 MB of scratch needed (40 + 8 B per cell) > 32 MiB
    boxes = np.zeros((n, 1, 2, 2), dtype=np.int16)
    A = bf.abs_from_boxes(bf.make_grid([2000, 1000]), boxes)
    G = torch.ones((n, 1), dtype=torch.float64, device="cuda")
    T = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc, *_ = _noalloc(f, A, G, None, None, terminal=T)
    assert rc == -1                                # BF_ERR_INVALID
    assert b"scratch" in L.bf_last_error()
    small = bf.abs_from_boxes(bf.make_grid([8]), np.zeros((8, 1, 2, 1), dtype=np.int16))
    Gh = np.ones((8, 1))
    V = torch.empty(8, dtype=torch.float64, device="cuda")
    mu = torch.empty(8, dtype=torch.uint8, device="cuda")
    Th = torch.zeros(8, dtype=torch.float64, device="cuda")
    it, st = ctypes.c_int64(), ctypes.c_int32()
    rc = f(small.handle, Gh.ctypes.data, None, None, Th.data_ptr(), 0, V.data_ptr(), mu.data_ptr(),
           ctypes.byref(it), ctypes.byref(st), None)
    assert rc == -1 and b"device memory" in L.bf_last_error()
