"""Seeded synthetic workloads for the symbolic optimal-control solver.

This module only draws inputs: grids, input sets, dynamics parameters, cost
arrays and target/avoid masks.  It holds none of the method's arithmetic (no
abstraction building, no relaxation) and imports neither the CUDA library nor
the CPU oracle, so both sides can be fed the very same arrays.

Every generator is deterministic in its seed (numpy PCG64).  The recipes:

* ``di2d``       double integrator on [-5,5]^2, 64x64 cells, u in
                 {-1,-.5,0,.5,1}, tau = 0.1, target [-.5,.5]^2, obstacle
                 [1,2]x[-5,1], G = tau.  (At tau = 0.1 every box off the
                 target holds its own cell, so only the target is finite; the
                 tau = 0.3 variant is the non-degenerate parity case.)
* ``unicycle3d`` unicycle on [0,10]^2 x [-pi,pi) (theta periodic), inputs
                 v in {0.5,1} x w in {-1,-.5,0,.5,1}, tau = 0.3, RK4 with 8
                 substeps, disturbance 0.05, 40 obstacle boxes (centres
                 U[0,10]^2, sides U[0.2,1.0], redrawn if they meet the
                 target), target [8,9]^2 x all theta, G = tau (1 + 0.1 |w|).
* ``fire4d``     coordinated-turn aircraft (x, y, psi, V) on
                 [0,1000]^2 x [-pi,pi) x [10,20], bank phi in
                 {-30,-15,0,15,30} deg x acceleration a in {-1,0,1}, tau = 1,
                 wind 0.5 m/s along x; fire intensity I = max of 5 Gaussian
                 blobs (centres U[150,850]^2, sigma U[10,16] m, amplitude
                 U[0.7,1]) at the cell centre, G = tau (1 - 1.5 I); landing
                 target [50,250] x [50,100] x [-10,10] deg x [10,12.5];
                 6 no-fly boxes (sides U[50,200] m, all psi and V).
                 At tau = 1 s a 10 m cell moves about one cell per step, so
                 almost every box keeps its own cell and few cells get a
                 finite value; the measured 4-D case uses tau = 2 s and the
                 landing box [50,250] x [50,150] x [-30,30] deg x [10,15].
* ``batched``    64 unicycle instances, grid scale s ~ logU[1,4],
                 n = (round(50 s), round(50 s), round(16 s)); each with a 1x1
                 target at a random place, 10-40 obstacles and
                 G = tau (1 + c |w|), c ~ U[0,1].
* ``served``     Poisson arrivals (rate per second) over a mix of three
                 resident abstractions (di2d 64^2; unicycle 100x100x32; fire
                 60x60x24x6), each request a fresh target / fire map.

Targets are the cells contained in the closed target box; avoid cells are the
cells whose closed box meets a closed obstacle box.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 2001

LINEAR2D, UNICYCLE3D, FIRE4D = 1, 2, 3


@dataclasses.dataclass
class Grid:
    n: tuple
    lo: tuple
    hi: tuple
    periodic: tuple

    @property
    def ndim(self):
        return len(self.n)

    @property
    def ncells(self):
        return int(np.prod(self.n))

    @property
    def eta(self):
        return tuple((h - l) / k for l, h, k in zip(self.lo, self.hi, self.n))

    def cell_bounds(self, d):
        """Lower and upper edge of every cell along dim d (float64 arrays)."""
        k = np.arange(self.n[d], dtype=np.float64)
        e = (self.hi[d] - self.lo[d]) / self.n[d]
        return self.lo[d] + k * e, self.lo[d] + (k + 1.0) * e

    def centres(self, d):
        k = np.arange(self.n[d], dtype=np.float64)
        e = (self.hi[d] - self.lo[d]) / self.n[d]
        return self.lo[d] + (k + 0.5) * e


@dataclasses.dataclass
class Workload:
    name: str
    grid: Grid
    kind: int                 # dynamics kind (LINEAR2D, UNICYCLE3D, FIRE4D)
    params: tuple             # dynamics parameters (see the library header)
    substeps: int
    inputs: np.ndarray        # [U][udim] float64
    tau: float
    G: np.ndarray             # [C][U] float64
    target: np.ndarray        # [C] uint8
    avoid: np.ndarray         # [C] uint8
    seed: int
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def ncells(self):
        return self.grid.ncells

    @property
    def ninputs(self):
        return int(self.inputs.shape[0])

    def terminal(self):
        """Terminal cost: 0 on target cells, +inf elsewhere."""
        t = np.full(self.ncells, np.inf)
        t[self.target.astype(bool)] = 0.0
        return t


def _mask_from_dims(grid, per_dim):
    """Outer product of per-dimension boolean masks -> flat [C] bool."""
    m = np.ones((), dtype=bool)
    # cell index c = i0 + n0*(i1 + ...): dim 0 is the fastest, so build in
    # reverse order and flatten C-style.
    for d in reversed(range(grid.ndim)):
        m = np.multiply.outer(m, per_dim[d])
    return m.reshape(-1)


def box_contains_cells(grid, box, tol=1e-9):
    """Cells contained in the closed box (None entries = whole dimension)."""
    per = []
    for d in range(grid.ndim):
        if box[d] is None:
            per.append(np.ones(grid.n[d], dtype=bool))
            continue
        a, b = box[d]
        lo, hi = grid.cell_bounds(d)
        e = tol * (grid.hi[d] - grid.lo[d]) / grid.n[d]
        per.append((lo >= a - e) & (hi <= b + e))
    return _mask_from_dims(grid, per)


def box_meets_cells(grid, box):
    """Cells whose closed box meets the closed box (None = whole dimension)."""
    per = []
    for d in range(grid.ndim):
        if box[d] is None:
            per.append(np.ones(grid.n[d], dtype=bool))
            continue
        a, b = box[d]
        lo, hi = grid.cell_bounds(d)
        per.append((lo <= b) & (hi >= a))
    return _mask_from_dims(grid, per)


def _boxes_meet(a, b):
    return all(x0 <= y1 and y0 <= x1 for (x0, x1), (y0, y1) in zip(a, b))


# --------------------------------------------------------------------------
# configurations
# --------------------------------------------------------------------------

def di2d(n=(64, 64), seed=SEED_BASE + 1, tau=0.1):
    grid = Grid(tuple(n), (-5.0, -5.0), (5.0, 5.0), (False, False))
    inputs = np.array([[-1.0], [-0.5], [0.0], [0.5], [1.0]])
    C, U = grid.ncells, inputs.shape[0]
    G = np.full((C, U), tau)
    target = box_contains_cells(grid, [(-0.5, 0.5), (-0.5, 0.5)]).astype(np.uint8)
    avoid = box_meets_cells(grid, [(1.0, 2.0), (-5.0, 1.0)]).astype(np.uint8)
    return Workload("di2d", grid, LINEAR2D, (), 1, inputs, tau, G, target, avoid, seed,
                    {"obstacle": [(1.0, 2.0), (-5.0, 1.0)]})


def unicycle_inputs():
    return np.array([[v, w] for v in (0.5, 1.0) for w in (-1.0, -0.5, 0.0, 0.5, 1.0)])


def unicycle3d(n=(200, 200, 64), seed=SEED_BASE + 2, n_obstacles=40,
               target_xy=((8.0, 9.0), (8.0, 9.0)), cost_c=0.1, disturbance=0.05):
    rng = np.random.default_rng(seed)
    grid = Grid(tuple(n), (0.0, 0.0, -math.pi), (10.0, 10.0, math.pi), (False, False, True))
    tau = 0.3
    inputs = unicycle_inputs()
    C, U = grid.ncells, inputs.shape[0]
    g_u = tau * (1.0 + cost_c * np.abs(inputs[:, 1]))
    G = np.ascontiguousarray(np.broadcast_to(g_u, (C, U)))
    tbox = [target_xy[0], target_xy[1], None]
    target = box_contains_cells(grid, tbox)
    avoid = np.zeros(C, dtype=bool)
    obstacles = []
    while len(obstacles) < n_obstacles:
        cx, cy = rng.uniform(0.0, 10.0, size=2)
        sx, sy = rng.uniform(0.2, 1.0, size=2)
        ob = [(cx - sx / 2, cx + sx / 2), (cy - sy / 2, cy + sy / 2)]
        if _boxes_meet(ob, tbox[:2]):
            continue
        obstacles.append(ob)
        avoid |= box_meets_cells(grid, ob + [None])
    return Workload("unicycle3d", grid, UNICYCLE3D, (disturbance,), 8, inputs, tau, G,
                    target.astype(np.uint8), avoid.astype(np.uint8), seed,
                    {"obstacles": obstacles, "cost_c": cost_c})


def fire_inputs():
    phis = np.deg2rad([-30.0, -15.0, 0.0, 15.0, 30.0])
    return np.array([[p, a] for a in (-1.0, 0.0, 1.0) for p in phis])


def fire_intensity(grid, blobs):
    xc, yc = grid.centres(0), grid.centres(1)
    I = np.zeros((grid.n[1], grid.n[0]))
    for (bx, by, s, amp) in blobs:
        r2 = (xc[None, :] - bx) ** 2 + (yc[:, None] - by) ** 2
        I = np.maximum(I, amp * np.exp(-r2 / (2.0 * s * s)))
    return I   # [n1][n0]


def fire4d(n=(100, 100, 36, 8), seed=SEED_BASE + 3, n_blobs=5, n_nofly=6,
           target=((50.0, 250.0), (50.0, 100.0), (-math.radians(10), math.radians(10)), (10.0, 12.5)),
           sigma=(10.0, 16.0), tau=1.0, extent=1000.0):
    rng = np.random.default_rng(seed)
    grid = Grid(tuple(n), (0.0, 0.0, -math.pi, 10.0), (extent, extent, math.pi, 20.0),
                (False, False, True, False))
    f = extent / 1000.0
    inputs = fire_inputs()
    C, U = grid.ncells, inputs.shape[0]
    blobs = []
    for _ in range(n_blobs):
        bx, by = rng.uniform(150.0 * f, 850.0 * f, size=2)
        s = rng.uniform(*sigma)
        amp = rng.uniform(0.7, 1.0)
        blobs.append((float(bx), float(by), float(s), float(amp)))
    I2 = fire_intensity(grid, blobs)                      # [n1][n0]
    n0, n1 = grid.n[0], grid.n[1]
    rest = C // (n0 * n1)
    I = np.broadcast_to(I2.reshape(1, n1 * n0), (rest, n1 * n0)).reshape(C)
    g_cell = tau * (1.0 - 1.5 * I)
    G = np.ascontiguousarray(np.broadcast_to(g_cell[:, None], (C, U)))
    tmask = box_contains_cells(grid, list(target))
    avoid = np.zeros(C, dtype=bool)
    nofly = []
    while len(nofly) < n_nofly:
        cx, cy = rng.uniform(0.0, extent, size=2)
        sx, sy = rng.uniform(50.0 * f, 200.0 * f, size=2)
        ob = [(cx - sx / 2, cx + sx / 2), (cy - sy / 2, cy + sy / 2)]
        if _boxes_meet(ob, list(target[:2])):
            continue
        if any(_boxes_meet(ob, [(b[0] - 3 * b[2], b[0] + 3 * b[2]), (b[1] - 3 * b[2], b[1] + 3 * b[2])])
               for b in blobs):
            continue
        nofly.append(ob)
        avoid |= box_meets_cells(grid, ob + [None, None])
    params = (0.5, 9.81, 10.0, 20.0, 0.0)
    return Workload("fire4d", grid, FIRE4D, params, 8, inputs, tau, G,
                    tmask.astype(np.uint8), avoid.astype(np.uint8), seed,
                    {"blobs": blobs, "nofly": nofly, "intensity_min_cost": float(g_cell.min())})


def fire4d_fire_cells(w, threshold=0.01, speed=None):
    """Successor class of the second mission stage (A_fire x A_drop of Sec. VI-A):
    the cells whose fire intensity at the centre is at least ``threshold`` and,
    if ``speed`` = (lo, hi) is given, whose speed cell lies inside it.  uint8 [C]."""
    grid = w.grid
    I2 = fire_intensity(grid, w.meta["blobs"])
    n0, n1 = grid.n[0], grid.n[1]
    rest = grid.ncells // (n0 * n1)
    mask = np.broadcast_to((I2 >= threshold).reshape(1, n1 * n0), (rest, n1 * n0)).reshape(grid.ncells)
    if speed is not None:
        vs = grid.centres(3)
        vok = (vs >= speed[0]) & (vs <= speed[1])
        per_v = grid.ncells // grid.n[3]
        mask = mask & np.repeat(vok, per_v)
    return np.ascontiguousarray(mask, dtype=np.uint8)


def batched(count=64, seed=SEED_BASE + 4, scale=(1.0, 4.0), base=(50, 50, 16)):
    """Instances of the unicycle workload on uneven grids (config 4)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        s = math.exp(rng.uniform(math.log(scale[0]), math.log(scale[1])))
        n = (int(round(base[0] * s)), int(round(base[1] * s)), int(round(base[2] * s)))
        tx, ty = rng.uniform(1.0, 8.0, size=2)
        nob = int(rng.integers(10, 41))
        c = float(rng.uniform(0.0, 1.0))
        sub_seed = int(rng.integers(0, 2**31 - 1))
        w = unicycle3d(n=n, seed=sub_seed, n_obstacles=nob,
                       target_xy=((tx, tx + 1.0), (ty, ty + 1.0)), cost_c=c)
        w.name = "unicycle3d[%d]" % i
        w.meta["scale"] = s
        out.append(w)
    return out


def served_requests(count, rate=200.0, seed=SEED_BASE + 5, sizes=None):
    """Poisson arrival times and a request mix over three resident abstractions.

    Returns (base_workloads, requests): base_workloads[k] fixes the grid and
    dynamics of abstraction k; each request is (arrival_s, k, workload) with a
    fresh seeded target (and, for the fire model, fire map).
    """
    rng = np.random.default_rng(seed)
    sizes = sizes or {"di2d": (64, 64), "unicycle3d": (100, 100, 32), "fire4d": (60, 60, 24, 6)}
    bases = [di2d(sizes["di2d"]), unicycle3d(sizes["unicycle3d"], seed=seed + 11),
             fire4d(sizes["fire4d"], seed=seed + 12,
                    target=((50.0, 250.0), (50.0, 150.0), (-math.radians(20), math.radians(20)),
                            (10.0, 15.0)))]
    t = 0.0
    reqs = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        k = int(rng.integers(0, 3))
        rs = int(rng.integers(0, 2**31 - 1))
        if k == 0:
            r2 = np.random.default_rng(rs)
            cx, cy = r2.uniform(-3.5, 3.5, size=2)
            w = di2d(sizes["di2d"], seed=rs)
            w.target = box_contains_cells(w.grid, [(cx - 0.6, cx + 0.6), (cy - 0.6, cy + 0.6)]).astype(np.uint8)
            w.target &= (1 - w.avoid)
        elif k == 1:
            r2 = np.random.default_rng(rs)
            tx, ty = r2.uniform(1.0, 8.0, size=2)
            w = dataclasses.replace(bases[1])
            w.target = box_contains_cells(w.grid, [(tx, tx + 1.0), (ty, ty + 1.0), None]).astype(np.uint8)
            w.seed = rs
        else:
            w = fire4d(sizes["fire4d"], seed=rs,
                       target=((50.0, 250.0), (50.0, 150.0), (-math.radians(20), math.radians(20)),
                               (10.0, 15.0)))
        w.name = bases[k].name
        reqs.append((t, k, w))
    return bases, reqs
