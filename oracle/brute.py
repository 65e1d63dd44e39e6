"""Pure-Python evaluators of the paper's cost notions, for tiny systems only.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

A system is given as successor lists ``F[x][u]`` (a list of states; an empty
list is a pair whose successor is the overflow set, Sec. V-B), a running cost
``g(x, y, u)`` and a terminal cost ``T[x]`` (the paper's G).  Costs are
Python floats; ``math.inf`` is allowed.

* ``cost_J``                      -- the cost functional J(u, v, x) of Eq. (costs).
* ``closed_loop_performance``     -- L(p, mu) of Eq. (closedloopperformance):
  the sup over closed-loop behaviours of the inf over hand-over signals,
  enumerated up to a finite horizon.
* ``performance`` / ``brute_force_value`` -- L(., mu) of a static
  controller for every initial state, by the finite-horizon recursion on the
  hand-over time, and its minimum over every single-valued static
  controller: the value function of Eq. (valuefunction) among static
  controllers, by enumeration.
"""
from __future__ import annotations

import itertools
import math

def cost_J(T, g, xs, us, v):
    """J(u,v,x) = G(x(T)) + sum_{t<T} g(x(t), x(t+1), u(t)), T = first 1 of v.

    ``xs``, ``us``, ``v`` are finite prefixes long enough to contain the first
    1 of v; J is +inf when v has no 1 in the prefix (v = 0).
    """
    try:
        Ts = v.index(1)
    except ValueError:
        return math.inf
    s = 0.0
    for t in range(Ts):
        s = s + g(xs[t], xs[t + 1], us[t])
    return T[xs[Ts]] + s


def closed_loop_performance(F, T, g, p, mu, horizon):
    """L(p, mu): sup over behaviours (u, x) with u(t) in mu(x(t)) of
    inf over v of J(u, v, x), every behaviour cut at ``horizon`` steps.

    ``mu[x]`` is a collection of allowed inputs.  Pairs with an empty
    successor list lead to the overflow set: that behaviour can only stop
    before the step.  The horizon cut is exact when every cycle reachable
    under mu has non-negative cost.
    """
    best = -math.inf

    def walk(x, acc, best_stop, depth):
        nonlocal best
        stop_here = acc + T[x]
        m = min(best_stop, stop_here)
        if depth == horizon:
            best = max(best, m)
            return
        for u in mu[x]:
            succ = F[x][u]
            if not succ:                      # overflow: no further state
                best = max(best, m)
                continue
            for y in succ:
                walk(y, acc + g(x, y, u), m, depth + 1)

    walk(p, 0.0, math.inf, 0)
    return best


def performance(F, T, g, mu_sets, max_rounds=10000):
    """Closed-loop performance L(., mu) of a static controller mu (Eq.
    closedloopperformance), for every initial state at once.

    ``mu_sets[x]`` is the set of inputs mu allows at x.  With h_k the
    worst case over behaviours of the best hand-over time T <= k,
      h_0 = G (hand over at once),
      h_{k+1}(x) = min(G(x), sup_{u in mu(x), y in F(x,u)} g(x,y,u) + h_k(y)),
    and L(., mu) = lim h_k (non-increasing).  A pair whose successor is the
    overflow set contributes +inf.  Raises if h has not settled after
    ``max_rounds`` rounds (a negative cycle drives it to -inf).
    """
    n = len(F)
    h = [float(T[x]) for x in range(n)]
    for _ in range(max_rounds):
        new = []
        for x in range(n):
            worst = -math.inf
            for u in mu_sets[x]:
                succ = F[x][u]
                if not succ:
                    worst = math.inf
                    continue
                for y in succ:
                    v = g(x, y, u) + h[y]
                    if v > worst:
                        worst = v
            new.append(min(float(T[x]), worst))
        if new == h:
            return h
        h = new
    raise RuntimeError("closed-loop performance did not settle (negative cycle)")


def brute_force_value(F, T, g):
    """min over every single-valued static controller mu of L(., mu).

    Set-valued controllers only enlarge the closed-loop behaviour, so the
    minimum over single-valued ones is the value function of Eq.
    (valuefunction) among static controllers.
    """
    n = len(F)
    U = len(F[0])
    best = [math.inf] * n
    for choice in itertools.product(range(U), repeat=n):
        J = performance(F, T, g, [[u] for u in choice])
        for x in range(n):
            if J[x] < best[x]:
                best[x] = J[x]
    return best


def controller_sets(mu, U, handover=0xFF):
    """Algorithm 1's output as sets: mu(x) = U (every input) at hand-over."""
    return [list(range(U)) if int(m) == handover else [int(m)] for m in mu]


def boxes_to_successors(n, periodic, boxes):
    """Successor lists F[x][u] from int16 boxes [C][U][2][D] (blocked -> [])."""
    D = len(n)
    C, U = boxes.shape[0], boxes.shape[1]
    F = []
    for x in range(C):
        row = []
        for u in range(U):
            lo = [int(boxes[x, u, 0, d]) for d in range(D)]
            hi = [int(boxes[x, u, 1, d]) for d in range(D)]
            if lo[0] == -32768:
                row.append([])
                continue
            ranges = []
            for d in range(D):
                r = []
                for k in range(lo[d], hi[d] + 1):
                    r.append(k - n[d] if (periodic[d] and k >= n[d]) else k)
                ranges.append(r)
            cells = []
            for ks in itertools.product(*reversed(ranges)):
                ks = list(reversed(ks))
                c = 0
                for d in reversed(range(D)):
                    c = c * n[d] + ks[d]
                cells.append(c)
            row.append(cells)
        F.append(row)
    return F
