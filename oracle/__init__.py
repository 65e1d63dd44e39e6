"""CPU oracle for the generalized Bellman-Ford method (arXiv 2001.06231).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It is written from
the paper, shares no code with the CUDA library, and never imports it.

The numeric work lives in ``bf_oracle.c`` (plain single-threaded FP64 C,
compiled with ``-ffp-contract=off``); this module only compiles it, loads it
with ctypes and marshals numpy arrays.  ``brute.py`` holds pure-Python
evaluators of the paper's cost functional and closed-loop performance for
tiny systems.

Array conventions (see ``bf_oracle.c``): cell index
``c = i0 + n0*(i1 + n1*(i2 + n2*i3))``; boxes int16 ``[C][U][2][D]``
(lo then hi, ``lo[0] == -32768`` = blocked); G float64 ``[C][U]``; terminal
float64 ``[C]``; avoid uint8 ``[C]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bf_oracle.c")
SO = os.path.join(HERE, "_build", "libbf_oracle.so")

BLOCKED = -32768
HANDOVER = 0xFF
CONVERGED, NEG_CYCLE, ITER_CAP = 0, 1, 2
LINEAR2D, UNICYCLE3D, FIRE4D = 1, 2, 3

_lib = None


def build(force: bool = False) -> str:
    """Compile bf_oracle.c into _build/libbf_oracle.so (plain gcc, FP64)."""
    os.makedirs(os.path.dirname(SO), exist_ok=True)
    if force or not os.path.exists(SO) or os.path.getmtime(SO) < os.path.getmtime(SRC):
        tmp = SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, SO)
    return SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(SO)
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.orc_build_boxes.argtypes = [i32, P, i32, i32, P, P, P, P, i32, i32, P, f64, P]
        L.orc_flow.argtypes = [i32, P, i32, i32, P, f64, P, P]
        L.orc_pred_build.argtypes = [i32, P, P, i32, P, P, ctypes.POINTER(ctypes.c_void_p)]
        L.orc_free.argtypes = [P]
        L.orc_solve.argtypes = [i32, P, P, i32, P, P, P, P, P, P, i64, P, P, P, P, P, P, P, P, i64, P]
        L.orc_dijkstra.argtypes = [i32, P, P, i32, P, P, P, P, P, P]
        L.orc_bellman_check.argtypes = [i32, P, P, i32, P, P, P, P, P, P, P, P, P, i64, P, P]
        for f in (L.orc_build_boxes, L.orc_flow, L.orc_pred_build, L.orc_solve,
                  L.orc_dijkstra, L.orc_bellman_check):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _grid_arrays(n, periodic):
    n = np.ascontiguousarray(n, dtype=np.int32)
    per = np.ascontiguousarray([1 if p else 0 for p in periodic], dtype=np.uint8)
    return n, per


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed with code %d" % (what, rc))


def build_boxes(kind, params, substeps, n, glo, ghi, periodic, inputs, tau):
    """Abstraction boxes [C][U][2][D] of a sampled system (Sec. V-B)."""
    n, per = _grid_arrays(n, periodic)
    D = len(n)
    glo = np.ascontiguousarray(glo, dtype=np.float64)
    ghi = np.ascontiguousarray(ghi, dtype=np.float64)
    inputs = np.ascontiguousarray(np.atleast_2d(inputs), dtype=np.float64)
    U, udim = inputs.shape
    prm = np.zeros(8, dtype=np.float64)
    prm[:len(params)] = params
    C = int(np.prod(n))
    boxes = np.zeros((C, U, 2, D), dtype=np.int16)
    _check(lib().orc_build_boxes(kind, _p(prm), substeps, D, _p(n), _p(glo), _p(ghi), _p(per),
                                 U, udim, _p(inputs), float(tau), _p(boxes)), "build_boxes")
    return boxes


def flow(kind, params, substeps, u, tau, c, r):
    """RK4 centre and growth-bound radius after tau (for the closed-form pins)."""
    prm = np.zeros(8, dtype=np.float64)
    prm[:len(params)] = params
    u = np.ascontiguousarray(u, dtype=np.float64)
    c = np.array(c, dtype=np.float64)
    r = np.array(r, dtype=np.float64)
    _check(lib().orc_flow(kind, _p(prm), substeps, len(c), _p(u), float(tau), _p(c), _p(r)), "flow")
    return c, r


def pred(n, periodic, boxes):
    """Exact pred(y) = {x : exists u, y in F(x,u)} as CSR (row_ptr, col)."""
    n, per = _grid_arrays(n, periodic)
    D = len(n)
    C, U = boxes.shape[0], boxes.shape[1]
    boxes = np.ascontiguousarray(boxes, dtype=np.int16)
    ptr = np.zeros(C + 1, dtype=np.int64)
    colp = ctypes.c_void_p()
    _check(lib().orc_pred_build(D, _p(n), _p(per), U, _p(boxes), _p(ptr), ctypes.byref(colp)), "pred")
    nnz = int(ptr[-1])
    col = np.ctypeslib.as_array(ctypes.cast(colp, ctypes.POINTER(ctypes.c_int32)), shape=(max(nnz, 1),))[:nnz].copy()
    lib().orc_free(colp)
    return ptr, col


def solve(n, periodic, boxes, G, terminal, avoid=None, max_iters=0, pred_csr=None, trace_cap=None,
          succ_class=None, G_class=None):
    """Algorithm 1 with Jacobi rounds.  succ_class ([C] mask) and G_class
    ([C][U]) give the running cost G_class(x,u) for successors in the class.

    Returns dict(V, mu, iters, status, f1, changed, f1_exit): per-round |F1|
    and number of changed cells, and the F1 mask left when the loop ended.
    """
    n, per = _grid_arrays(n, periodic)
    D = len(n)
    C, U = boxes.shape[0], boxes.shape[1]
    boxes = np.ascontiguousarray(boxes, dtype=np.int16)
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(C, U)
    terminal = np.ascontiguousarray(terminal, dtype=np.float64).reshape(C)
    if avoid is not None:
        avoid = np.ascontiguousarray(avoid, dtype=np.uint8).reshape(C)
    cls, Gc = _class_arrays(succ_class, G_class, C, U)
    V = np.empty(C, dtype=np.float64)
    mu = np.empty(C, dtype=np.uint8)
    iters = np.zeros(1, dtype=np.int64)
    status = np.zeros(1, dtype=np.int32)
    cap = trace_cap if trace_cap is not None else min(C, max_iters if max_iters > 0 else C, 1 << 20)
    f1 = np.zeros(max(cap, 1), dtype=np.int64)
    chg = np.zeros(max(cap, 1), dtype=np.int64)
    ptr, col = (None, None) if pred_csr is None else pred_csr
    f1_exit = np.zeros(C, dtype=np.uint8)
    _check(lib().orc_solve(D, _p(n), _p(per), U, _p(boxes), _p(G), _p(terminal), _p(avoid), _p(cls), _p(Gc),
                           int(max_iters), _p(ptr), _p(col), _p(V), _p(mu), _p(iters), _p(status),
                           _p(f1), _p(chg), cap, _p(f1_exit)), "solve")
    it = int(iters[0])
    k = min(it, cap)
    return {"V": V, "mu": mu, "iters": it, "status": int(status[0]),
            "f1": f1[:k].copy(), "changed": chg[:k].copy(), "f1_exit": f1_exit}


def dijkstra(n, periodic, boxes, G, terminal, avoid=None):
    """Generalized min-max Dijkstra (requires G >= 0 and terminal >= 0)."""
    n, per = _grid_arrays(n, periodic)
    D = len(n)
    C, U = boxes.shape[0], boxes.shape[1]
    boxes = np.ascontiguousarray(boxes, dtype=np.int16)
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(C, U)
    terminal = np.ascontiguousarray(terminal, dtype=np.float64).reshape(C)
    if avoid is not None:
        avoid = np.ascontiguousarray(avoid, dtype=np.uint8).reshape(C)
    V = np.empty(C, dtype=np.float64)
    mu = np.empty(C, dtype=np.uint8)
    _check(lib().orc_dijkstra(D, _p(n), _p(per), U, _p(boxes), _p(G), _p(terminal), _p(avoid),
                              _p(V), _p(mu)), "dijkstra")
    return V, mu


def _class_arrays(succ_class, G_class, C, U):
    if succ_class is None:
        return None, None
    return (np.ascontiguousarray(succ_class, dtype=np.uint8).reshape(C),
            np.ascontiguousarray(G_class, dtype=np.float64).reshape(C, U))


def bellman_check(n, periodic, boxes, G, terminal, avoid, V, mu, cells=None, succ_class=None, G_class=None):
    """Number of cells violating P(V) = V or mu-attainment; (nbad, first_bad)."""
    n, per = _grid_arrays(n, periodic)
    D = len(n)
    C, U = boxes.shape[0], boxes.shape[1]
    boxes = np.ascontiguousarray(boxes, dtype=np.int16)
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(C, U)
    terminal = np.ascontiguousarray(terminal, dtype=np.float64).reshape(C)
    if avoid is not None:
        avoid = np.ascontiguousarray(avoid, dtype=np.uint8).reshape(C)
    V = np.ascontiguousarray(V, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.uint8)
    cl = None if cells is None else np.ascontiguousarray(cells, dtype=np.int64)
    nbad = np.zeros(1, dtype=np.int64)
    first = np.zeros(1, dtype=np.int64)
    cls, Gc = _class_arrays(succ_class, G_class, C, U)
    _check(lib().orc_bellman_check(D, _p(n), _p(per), U, _p(boxes), _p(G), _p(terminal), _p(avoid), _p(cls), _p(Gc),
                                   _p(V), _p(mu), _p(cl), 0 if cl is None else len(cl),
                                   _p(nbad), _p(first)), "bellman_check")
    return int(nbad[0]), int(first[0])
