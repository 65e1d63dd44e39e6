"""Helpers shared by the GPU parity tests.

Every oracle input is built by the oracle itself: the solver parity tests hand
the oracle's boxes to both sides (imported into the library with
abs_from_boxes), and the library's own builder is compared with the oracle's
builder separately (a mismatch count; the transcendental functions of the host
and the device may differ in the last bit).
"""
import numpy as np

import oracle
import paper_2001_06231_gb300 as bf

_CACHE = {}


def oracle_boxes(w):
    """The oracle's boxes of a workload, int16 [C][U][2][D] (cached per workload)."""
    key = (w.name, w.grid.n, w.seed, w.tau, tuple(w.params))
    if key not in _CACHE:
        _CACHE[key] = oracle.build_boxes(w.kind, w.params, w.substeps, w.grid.n, w.grid.lo, w.grid.hi,
                                         w.grid.periodic, w.inputs, w.tau)
    return _CACHE[key]


def import_boxes(w, boxes):
    """A library abstraction holding exactly the given boxes on the workload's grid."""
    return bf.abs_from_boxes(w.grid, boxes)


def mismatches(a, b):
    """Number of (cell, input) pairs whose boxes differ."""
    return int(np.any(a != b, axis=(2, 3)).sum())
