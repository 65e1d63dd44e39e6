"""Generalized Bellman-Ford for symbolic optimal control on GB300 (sm_103a).

Python binding of the C ABI declared in ``include/bfgpu.h`` (arXiv
2001.06231, Algorithm 1 and the abstraction of Sec. V-B).  This module only
marshals arguments with ctypes: every step of the method runs in the CUDA
library ``_build/libbfgpu.so``.  There is no CPU fallback: if the library
cannot be loaded, the first call raises.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA
memory); outputs are numpy arrays unless CUDA tensors are passed as
destinations.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

BF_OK = 0
BF_ERR = {-1: "BF_ERR_INVALID", -2: "BF_ERR_OOM", -3: "BF_ERR_CUDA", -4: "BF_ERR_TIMEOUT",
          -5: "BF_ERR_UNSUPPORTED"}
CONVERGED, NEG_CYCLE, ITER_CAP = 0, 1, 2
HANDOVER = 0xFF
BLOCKED = -32768
LINEAR2D, UNICYCLE3D, FIRE4D = 1, 2, 3
MODE_STORED, MODE_RECOMPUTE, MODE_HYBRID = 0, 1, 2
SCHED_JACOBI, SCHED_INPLACE = 0, 1
SCHED_AUTO = SCHED_JACOBI
FLAG_HOST_LOOP, FLAG_COUNT_EXACT, FLAG_TIME_KERNELS = 1, 2, 4

EXPORTED = ["abs_build", "abs_build_hybrid", "abs_stored_inputs", "abs_from_boxes", "abs_export_boxes",
            "abs_export_pred", "abs_info", "abs_shape_info",
            "abs_free", "bf_solve", "bf_solve_batch", "bf_serve_open", "bf_serve_submit", "bf_serve_poll",
            "bf_serve_close", "bf_solve_noalloc", "bf_tune", "bf_set_schedule", "bf_tune_batch", "bf_set_batch_schedule",
            "bf_last_error"]


class BfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (BF_ERR.get(code, "BF_ERR"), code, msg))
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("n", ctypes.c_int32 * 4), ("lo", ctypes.c_double * 4),
                ("hi", ctypes.c_double * 4), ("periodic", ctypes.c_uint8 * 4)]


class Inputs(ctypes.Structure):
    _fields_ = [("ninputs", ctypes.c_int32), ("udim", ctypes.c_int32), ("u", ctypes.c_void_p)]


class Dynamics(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("rk4_substeps", ctypes.c_int32), ("param", ctypes.c_double * 8)]


class SolveStats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("relaxed_cells", ctypes.c_int64),
                ("executed_pairs", ctypes.c_int64), ("exact_f1_cells", ctypes.c_int64),
                ("changed_cells", ctypes.c_int64), ("relax_launches", ctypes.c_int64),
                ("relax_ms", ctypes.c_double), ("propagate_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveOpts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int64), ("schedule", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("terminal", ctypes.c_void_p), ("trace", ctypes.c_void_p), ("trace_cap", ctypes.c_int64),
                ("stats", ctypes.c_void_p), ("succ_class", ctypes.c_void_p), ("G_class", ctypes.c_void_p),
                ("frontier_cache", ctypes.c_int64)]


class TuneResult(ctypes.Structure):
    _fields_ = [("slice_target", ctypes.c_int32), ("fuse_mark", ctypes.c_int32), ("relax_blocks", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("best_ms", ctypes.c_double), ("default_ms", ctypes.c_double),
                ("window33", ctypes.c_int32), ("plane_lists", ctypes.c_int32), ("templates", ctypes.c_int32),
                ("pair_inputs", ctypes.c_int32), ("dense_pct", ctypes.c_int32), ("occupancy", ctypes.c_int32),
                ("cell_masks", ctypes.c_int32), ("pair_dim", ctypes.c_int32), ("input_frontier", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("abs", ctypes.c_void_p), ("dyn", ctypes.c_void_p), ("grid", ctypes.c_void_p),
                ("inputs", ctypes.c_void_p), ("tau", ctypes.c_double), ("G", ctypes.c_void_p),
                ("target", ctypes.c_void_p), ("avoid", ctypes.c_void_p), ("terminal", ctypes.c_void_p),
                ("max_iters", ctypes.c_int64), ("V", ctypes.c_void_p), ("mu", ctypes.c_void_p),
                ("flags", ctypes.c_int32)]


REQ_BORROW_INPUTS = 1


class Result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("status", ctypes.c_int32), ("iters", ctypes.c_int64),
                ("error", ctypes.c_int32), ("mode", ctypes.c_int32), ("submit_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("finish_s", ctypes.c_double)]


_lib = None


def lib():
    """Load (building first if stale) the CUDA library; raises if unavailable."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path) or os.environ.get("BFGPU_REBUILD"):
            path = _build.build()
        L = ctypes.CDLL(path)
        missing = [name for name in EXPORTED if not hasattr(L, name)]
        if missing:
            raise BfError(-5, "library %s lacks %s" % (path, ", ".join(missing)))
        P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.abs_build.argtypes = [P, P, P, f64, i32, P, P]
        L.abs_build_hybrid.argtypes = [P, P, P, f64, i64, P, P]
        L.abs_stored_inputs.argtypes = [P, P]
        L.abs_from_boxes.argtypes = [P, i32, P, P, P]
        L.abs_export_boxes.argtypes = [P, P, P]
        L.abs_export_pred.argtypes = [P, P, P]
        L.abs_info.argtypes = [P, P, P, P, P, P, P]
        L.abs_shape_info.argtypes = [P, P, P]
        L.abs_free.argtypes = [P]
        L.abs_free.restype = None
        L.bf_solve.argtypes = [P, P, P, P, P, P, P, P, P, P]
        L.bf_solve_batch.argtypes = [i32, P, P, P, P, P, i64, P, P, P, P, P]
        L.bf_serve_open.argtypes = [ctypes.c_size_t, i32, i32, P]
        L.bf_serve_submit.argtypes = [P, P, P]
        L.bf_serve_poll.argtypes = [P, ctypes.c_uint64, i32, P]
        L.bf_serve_close.argtypes = [P]
        L.bf_serve_close.restype = None
        L.bf_solve_noalloc.argtypes = [P, P, P, P, P, i64, P, P, P, P, P]
        L.bf_tune.argtypes = [P, P, P, P, P, P, P]
        L.bf_set_schedule.argtypes = [P, P, P]
        L.bf_tune_batch.argtypes = [i32, P, P, P, P, P, i64, P, P]
        L.bf_set_batch_schedule.argtypes = [P, P]
        L.bf_last_error.restype = ctypes.c_char_p
        for name in ("abs_build", "abs_build_hybrid", "abs_stored_inputs", "abs_from_boxes",
                     "abs_export_boxes", "abs_export_pred", "abs_info", "abs_shape_info",
                     "bf_solve", "bf_solve_batch", "bf_serve_open", "bf_serve_submit", "bf_serve_poll",
                     "bf_solve_noalloc", "bf_tune", "bf_set_schedule", "bf_tune_batch",
                     "bf_set_batch_schedule"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc):
    if rc != BF_OK:
        raise BfError(rc, lib().bf_last_error().decode())


def _ptr(a):
    """Raw pointer of a numpy array / torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()            # torch tensor


def _host(a, dtype):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=dtype)
    return a.contiguous()          # torch tensor, host or device; dtype is the caller's


def _stream(s):
    if s is None:
        return None
    return getattr(s, "cuda_stream", s)


def make_grid(n, lo=None, hi=None, periodic=None):
    """bf_grid from per-dimension lists (or an object with n/lo/hi/periodic)."""
    if isinstance(n, Grid):
        return n
    if hasattr(n, "n"):
        g = n
        n, lo, hi, periodic = g.n, g.lo, g.hi, g.periodic
    D = len(n)
    lo = lo if lo is not None else [0.0] * D
    hi = hi if hi is not None else [float(k) for k in n]
    periodic = periodic if periodic is not None else [False] * D
    s = Grid()
    s.ndim = D
    for d in range(D):
        s.n[d] = int(n[d])
        s.lo[d] = float(lo[d])
        s.hi[d] = float(hi[d])
        s.periodic[d] = 1 if periodic[d] else 0
    return s


class Abstraction:
    """Device-resident discrete abstraction (handle of the C ABI)."""

    def __init__(self, handle, grid):
        self.handle = ctypes.c_void_p(handle)
        self.grid = grid
        nc, nu, nd, md, nb, rb = (ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(),
                                  ctypes.c_int64(), ctypes.c_int32())
        _check(lib().abs_info(self.handle, ctypes.byref(nc), ctypes.byref(nu), ctypes.byref(nd),
                              ctypes.byref(md), ctypes.byref(nb), ctypes.byref(rb)))
        self.ncells, self.ninputs, self.ndim = nc.value, nu.value, nd.value
        self.mode, self.device_bytes, self.box_record_bytes = md.value, nb.value, rb.value
        k = ctypes.c_int32()
        _check(lib().abs_stored_inputs(self.handle, ctypes.byref(k)))
        self.stored_inputs = k.value
        npl, mis = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().abs_shape_info(self.handle, ctypes.byref(npl), ctypes.byref(mis)))
        self.shape_planes, self.shape_mismatch = npl.value, mis.value

    def export_boxes(self, out=None, stream=None):
        if out is None:
            out = np.empty((self.ncells, self.ninputs, 2, self.ndim), dtype=np.int16)
        _check(lib().abs_export_boxes(self.handle, _ptr(out), _stream(stream)))
        return out

    def export_pred(self, out=None, stream=None):
        if out is None:
            out = np.empty((self.ncells, 2, self.ndim), dtype=np.int16)
        _check(lib().abs_export_pred(self.handle, _ptr(out), _stream(stream)))
        return out

    def close(self):
        if self.handle and self.handle.value:
            lib().abs_free(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _system(kind, params, substeps, grid, inputs):
    g = make_grid(grid)
    u = np.ascontiguousarray(np.atleast_2d(inputs), dtype=np.float64)
    inp = Inputs(u.shape[0], u.shape[1], u.ctypes.data)
    dyn = Dynamics()
    dyn.kind = int(kind)
    dyn.rk4_substeps = int(substeps)
    for i, p in enumerate(params):
        dyn.param[i] = float(p)
    return dyn, g, inp, u


def abs_build(kind, params, substeps, grid, inputs, tau, mode=MODE_STORED, stream=None):
    """Build the abstraction of a built-in sampled system on the device."""
    dyn, g, inp, _keep = _system(kind, params, substeps, grid, inputs)
    h = ctypes.c_void_p()
    _check(lib().abs_build(ctypes.byref(dyn), ctypes.byref(g), ctypes.byref(inp), float(tau), int(mode),
                           _stream(stream), ctypes.byref(h)))
    return Abstraction(h.value, g)


def abs_build_hybrid(kind, params, substeps, grid, inputs, tau, box_budget, stream=None):
    """Memory-regulated build: box records of as many inputs as fit box_budget bytes."""
    dyn, g, inp, _keep = _system(kind, params, substeps, grid, inputs)
    h = ctypes.c_void_p()
    _check(lib().abs_build_hybrid(ctypes.byref(dyn), ctypes.byref(g), ctypes.byref(inp), float(tau),
                                  int(box_budget), _stream(stream), ctypes.byref(h)))
    return Abstraction(h.value, g)


def abs_build_workload(w, mode=MODE_STORED, stream=None, box_budget=None):
    if box_budget is not None:
        return abs_build_hybrid(w.kind, w.params, w.substeps, w.grid, w.inputs, w.tau, box_budget, stream)
    return abs_build(w.kind, w.params, w.substeps, w.grid, w.inputs, w.tau, mode, stream)


def abs_from_boxes(grid, boxes, stream=None):
    """Abstraction from boxes int16 [C][U][2][D] (numpy or torch, host or device)."""
    g = make_grid(grid)
    b = _host(boxes, np.int16)
    U = int(b.shape[1])
    h = ctypes.c_void_p()
    _check(lib().abs_from_boxes(ctypes.byref(g), U, _ptr(b), _stream(stream), ctypes.byref(h)))
    return Abstraction(h.value, g)


def bf_solve(abstraction, G, target=None, avoid=None, terminal=None, max_iters=0, schedule=SCHED_AUTO,
             host_loop=False, trace_cap=0, V=None, mu=None, stream=None, count_exact=False,
             time_kernels=False, succ_class=None, G_class=None, frontier_cache=0):
    """Algorithm 1 on the device.  Returns dict(V, mu, iters, status, stats[, trace]).

    succ_class ([C] mask) with G_class ([C][U]): running cost G_class(x,u) for
    successors in the class, G(x,u) for the others.  frontier_cache: cells of
    each pass's frontier whose regenerated box records are kept for the next
    pass (recompute and hybrid abstractions).
    """
    C = abstraction.ncells
    Gc = _host(G, np.float64)
    rc_mask = _host(succ_class, np.uint8)
    rc_cost = _host(G_class, np.float64)
    tg = _host(target, np.uint8)
    av = _host(avoid, np.uint8)
    tm = _host(terminal, np.float64)
    if V is None:
        V = np.empty(C, dtype=np.float64)
    if mu is None:
        mu = np.empty(C, dtype=np.uint8)
    opts = SolveOpts()
    opts.max_iters = int(max_iters)
    opts.schedule = int(schedule)
    opts.flags = ((FLAG_HOST_LOOP if host_loop else 0) | (FLAG_COUNT_EXACT if count_exact else 0)
                  | (FLAG_TIME_KERNELS if time_kernels else 0))
    opts.terminal = _ptr(tm)
    opts.succ_class = _ptr(rc_mask)
    opts.G_class = _ptr(rc_cost)
    opts.frontier_cache = int(frontier_cache)
    stats = SolveStats()
    opts.stats = ctypes.addressof(stats)
    trace = None
    if trace_cap:
        trace = np.zeros((int(trace_cap), 4), dtype=np.int64)
        opts.trace = trace.ctypes.data
        opts.trace_cap = int(trace_cap)
    it = ctypes.c_int64()
    st = ctypes.c_int32()
    _check(lib().bf_solve(abstraction.handle, _ptr(Gc), _ptr(tg), _ptr(av), ctypes.byref(opts), _ptr(V),
                          _ptr(mu), ctypes.byref(it), ctypes.byref(st), _stream(stream)))
    out = {"V": V, "mu": mu, "iters": it.value, "status": st.value, "stats": stats.as_dict()}
    if trace is not None:
        k = min(it.value, int(trace_cap))
        out["trace"] = trace[:k].copy()
    return out


def _ptr_array(items, conv):
    arr = (ctypes.c_void_p * len(items))()
    keep = []
    for i, a in enumerate(items):
        a = conv(a)
        keep.append(a)
        arr[i] = _ptr(a)
    return arr, keep


def bf_tune(abstraction, G, target=None, avoid=None, terminal=None, max_iters=0, stream=None,
            succ_class=None, G_class=None):
    """Time the pass schedules of this abstraction on the given inputs and keep the fastest."""
    Gc = _host(G, np.float64)
    tg = _host(target, np.uint8)
    av = _host(avoid, np.uint8)
    tm = _host(terminal, np.float64)
    rc_mask = _host(succ_class, np.uint8)
    rc_cost = _host(G_class, np.float64)
    opts = SolveOpts()
    opts.max_iters = int(max_iters)
    opts.terminal = _ptr(tm)
    opts.succ_class = _ptr(rc_mask)
    opts.G_class = _ptr(rc_cost)
    res = TuneResult()
    _check(lib().bf_tune(abstraction.handle, _ptr(Gc), _ptr(tg), _ptr(av), ctypes.byref(opts), ctypes.byref(res),
                         _stream(stream)))
    return {k: getattr(res, k) for k, _ in res._fields_}


def bf_set_schedule(abstraction, slice_target=2, fuse_mark=1, relax_blocks=0, window33=0, plane_lists=1,
                    templates=1, pair_inputs=0, dense_pct=0, occupancy=0, cell_masks=0, pair_dim=0,
                    input_frontier=0, stream=None):
    """Put a pass schedule in force on this abstraction's solves (no timing)."""
    s = TuneResult()
    s.slice_target, s.fuse_mark, s.relax_blocks, s.window33 = slice_target, fuse_mark, relax_blocks, window33
    s.plane_lists, s.templates, s.pair_inputs, s.dense_pct = plane_lists, templates, pair_inputs, dense_pct
    s.occupancy, s.cell_masks, s.pair_dim, s.input_frontier = occupancy, cell_masks, pair_dim, input_frontier
    _check(lib().bf_set_schedule(abstraction.handle, ctypes.byref(s), _stream(stream)))


def bf_solve_batch(abstractions, Gs, targets=None, avoids=None, terminals=None, max_iters=0, Vs=None,
                   mus=None, stream=None):
    """Solve many instances together (bf_solve_batch).  Returns a list of dicts."""
    n = len(abstractions)
    if Vs is None:
        Vs = [np.empty(a.ncells, dtype=np.float64) for a in abstractions]
    if mus is None:
        mus = [np.empty(a.ncells, dtype=np.uint8) for a in abstractions]
    absa = (ctypes.c_void_p * n)(*[a.handle.value for a in abstractions])
    ga, k1 = _ptr_array(Gs, lambda a: _host(a, np.float64))
    ta, k2 = _ptr_array(targets if targets is not None else [None] * n, lambda a: _host(a, np.uint8))
    va, k3 = _ptr_array(avoids if avoids is not None else [None] * n, lambda a: _host(a, np.uint8))
    tm, k4 = _ptr_array(terminals if terminals is not None else [None] * n, lambda a: _host(a, np.float64))
    Va, k5 = _ptr_array(Vs, lambda a: a)
    ma, k6 = _ptr_array(mus, lambda a: a)
    it = (ctypes.c_int64 * n)()
    st = (ctypes.c_int32 * n)()
    _check(lib().bf_solve_batch(n, absa, ga, ta, va, tm if terminals is not None else None, int(max_iters),
                                Va, ma, it, st, _stream(stream)))
    return [{"V": Vs[i], "mu": mus[i], "iters": it[i], "status": st[i]} for i in range(n)]


def bf_tune_batch(abstractions, Gs, targets=None, avoids=None, terminals=None, max_iters=0, stream=None):
    """Time the batched form's schedules on these instances and keep the fastest on the abstractions."""
    n = len(abstractions)
    absa = (ctypes.c_void_p * n)(*[a.handle.value for a in abstractions])
    ga, k1 = _ptr_array(Gs, lambda a: _host(a, np.float64))
    ta, k2 = _ptr_array(targets if targets is not None else [None] * n, lambda a: _host(a, np.uint8))
    va, k3 = _ptr_array(avoids if avoids is not None else [None] * n, lambda a: _host(a, np.uint8))
    tm, k4 = _ptr_array(terminals if terminals is not None else [None] * n, lambda a: _host(a, np.float64))
    res = TuneResult()
    _check(lib().bf_tune_batch(n, absa, ga, ta, va, tm if terminals is not None else None, int(max_iters),
                               ctypes.byref(res), _stream(stream)))
    return {k: getattr(res, k) for k, _ in res._fields_}


def bf_set_batch_schedule(abstraction, fuse_mark=-1, window33=1, plane_lists=1, templates=1, pair_inputs=1,
                          cell_masks=0):
    """Put a batched-form schedule in force on this abstraction (no timing)."""
    s = TuneResult()
    s.fuse_mark, s.window33, s.plane_lists, s.templates, s.pair_inputs = (fuse_mark, window33, plane_lists,
                                                                         templates, pair_inputs)
    s.cell_masks = cell_masks
    _check(lib().bf_set_batch_schedule(abstraction.handle, ctypes.byref(s)))


class Server:
    """Continuous-batching solve server (bf_serve_*).

    submit() copies the request's host inputs; the result arrays V / mu given
    (or allocated here) are filled when the request completes.
    """

    def __init__(self, hbm_budget, max_active=64, passes_per_step=8):
        h = ctypes.c_void_p()
        _check(lib().bf_serve_open(int(hbm_budget), int(max_active), int(passes_per_step), ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, G, target=None, avoid=None, terminal=None, abstraction=None, system=None,
               max_iters=0, V=None, mu=None, borrow=False):
        """system: (kind, params, substeps, grid, inputs, tau) when abstraction is None.

        borrow=True: the arrays are not copied at submit and must stay alive
        and unchanged until the request is done (they are kept referenced).
        """
        keep = []
        q = Request()
        if abstraction is not None:
            q.abs = abstraction.handle.value
            C = abstraction.ncells
        else:
            kind, params, substeps, grid, inputs, tau = system
            g = make_grid(grid)
            u = np.ascontiguousarray(np.atleast_2d(inputs), dtype=np.float64)
            inp = Inputs(u.shape[0], u.shape[1], u.ctypes.data)
            dyn = Dynamics()
            dyn.kind = int(kind)
            dyn.rk4_substeps = int(substeps)
            for i, p in enumerate(params):
                dyn.param[i] = float(p)
            keep += [g, u, inp, dyn]
            q.dyn, q.grid, q.inputs = ctypes.addressof(dyn), ctypes.addressof(g), ctypes.addressof(inp)
            q.tau = float(tau)
            C = int(np.prod([g.n[d] for d in range(g.ndim)]))
        Gc = _host(G, np.float64)
        tg = _host(target, np.uint8)
        av = _host(avoid, np.uint8)
        tm = _host(terminal, np.float64)
        V = np.empty(C, dtype=np.float64) if V is None else V
        mu = np.empty(C, dtype=np.uint8) if mu is None else mu
        q.G, q.target, q.avoid, q.terminal = _ptr(Gc), _ptr(tg), _ptr(av), _ptr(tm)
        q.max_iters = int(max_iters)
        q.V, q.mu = _ptr(V), _ptr(mu)
        q.flags = REQ_BORROW_INPUTS if borrow else 0
        rid = ctypes.c_uint64()
        _check(lib().bf_serve_submit(self.handle, ctypes.byref(q), ctypes.byref(rid)))
        self._keep[rid.value] = (V, mu, (Gc, tg, av, tm) if borrow else None)
        return rid.value

    def poll(self, rid, wait=True):
        """Returns dict(done, status, iters, error, mode, submit_s, admit_s, finish_s[, V, mu])."""
        r = Result()
        _check(lib().bf_serve_poll(self.handle, ctypes.c_uint64(rid), 1 if wait else 0, ctypes.byref(r)))
        out = {k: getattr(r, k) for k, _ in Result._fields_}
        if r.done:
            out["V"], out["mu"], _ = self._keep.pop(rid)
        return out

    def close(self):
        if self.handle and self.handle.value:
            lib().bf_serve_close(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
