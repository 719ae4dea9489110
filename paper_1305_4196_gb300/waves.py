"""Python binding of the wave-schedule host tool (include/mdgb_waves.h): argument
marshalling only, the schedule is built in the library."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import mdgb as _m

_lib = C.CDLL(_m.library_path())
_lib.md_wave_sets_1d.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]
_lib.md_wave_sets_1d.restype = C.c_int
_lib.md_waves.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
_lib.md_waves.restype = C.c_int
_lib.md_wave_schedule.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_int64]
_lib.md_wave_schedule.restype = C.c_int64


def _check(v):
    if v < 0:
        raise _m.MDError(int(v), "wave schedule: invalid arguments")
    return v


def _cells3(n):
    """The cell counts as 3 int32 values (the C calls read exactly three)."""
    n = np.ascontiguousarray(n, dtype=np.int32)
    if n.shape != (3,):
        raise ValueError("n must hold the cell counts of the 3 dimensions")
    return n


def sets_1d(D, periodic, spacing=3, start=0):
    """Set number of every cell of one dimension (0-based cells); returns (set_of_cell, n_sets)."""
    out = np.empty(int(D), dtype=np.int32)
    k = _check(_lib.md_wave_sets_1d(int(D), int(bool(periodic)), int(spacing), int(start), out.ctypes.data))
    return out, k


def waves(n, periodic, overlap=27):
    """Wave of every cell (x fastest), shape n[2] x n[1] x n[0] flattened; returns (wave_of_cell, n_waves)."""
    n = _cells3(n)
    p = np.ascontiguousarray(np.broadcast_to(np.asarray(periodic, dtype=np.int32), (3,)))
    out = np.empty(int(np.prod(n)), dtype=np.int32)
    k = _check(_lib.md_waves(n.ctypes.data, p.ctypes.data, int(overlap), out.ctypes.data))
    return out, k


def schedule(n, periodic, overlap=27, backward=False):
    """(task_cell, n_pred, succ_start, succ) of the forward or backward wave method."""
    n = _cells3(n)
    p = np.ascontiguousarray(np.broadcast_to(np.asarray(periodic, dtype=np.int32), (3,)))
    T = int(np.prod(n))
    tc = np.empty(T, dtype=np.int32)
    npred = np.empty(T, dtype=np.int32)
    start = np.empty(T + 1, dtype=np.int64)
    tot = _check(_lib.md_wave_schedule(n.ctypes.data, p.ctypes.data, int(overlap), int(bool(backward)),
                                       tc.ctypes.data, npred.ctypes.data, start.ctypes.data, None, 0))
    succ = np.empty(max(int(tot), 1), dtype=np.int32)
    _check(_lib.md_wave_schedule(n.ctypes.data, p.ctypes.data, int(overlap), int(bool(backward)), tc.ctypes.data,
                                 npred.ctypes.data, start.ctypes.data, succ.ctypes.data, int(tot)))
    return tc, npred, start, succ[:tot]


def critical_path(npred, start, succ):
    """Length (in tasks) of the longest dependency chain: the number of steps an
    unbounded number of workers needs."""
    T = npred.shape[0]
    indeg = npred.astype(np.int64).copy()
    level = np.zeros(T, dtype=np.int64)
    frontier = np.flatnonzero(indeg == 0)
    depth = 0
    while frontier.size:
        depth += 1
        nxt = []
        for t in frontier:
            for s in succ[start[t]:start[t + 1]]:
                level[s] = max(level[s], level[t] + 1)
                indeg[s] -= 1
                if indeg[s] == 0:
                    nxt.append(s)
        frontier = np.asarray(nxt, dtype=np.int64)
    return int(level.max()) + 1 if T else 0


def compare_with_colours(nc, overlap=27):
    """The paper's schedule on an nc^3 periodic cell grid beside the GPU path's 8 colour
    phases of 2x2x2-cell blocks: phases, tasks per phase, and (for the paper's dependent
    schedule) the critical path an unbounded number of workers would need."""
    n = (nc, nc, nc)
    w, k = waves(n, (1, 1, 1), overlap)
    counts = np.bincount(w, minlength=k)
    tc, npred, start, succ = schedule(n, (1, 1, 1), overlap)
    return {"cells": nc ** 3, "overlap_cells": overlap, "waves": int(k),
            "tasks_per_wave_min": int(counts.min()), "tasks_per_wave_mean": float(counts.mean()),
            "dependent_schedule_critical_path": critical_path(npred, start, succ),
            "mean_direct_predecessors": float(npred.mean()),
            "colour_phases": 8, "blocks_per_colour_phase": (nc // 2) ** 3 // 8, "cells_per_block": 8}
