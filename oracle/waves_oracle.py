"""Plain brute-force dependency graph of cell tasks run in a given order.

TEST INFRASTRUCTURE ONLY: used by the test suite to check the library's wave-schedule
tool; nothing in the product imports it.  It shares no code with the library.

Definition (Meyer 2013, arXiv:1305.4196, Sec. II.B): tasks run in the given order; a
task's direct predecessors are, for each cell it touches, the last earlier task that
touched the same cell.  This file finds them by scanning all earlier tasks, O(T^2).
"""
from __future__ import annotations

import itertools

import numpy as np


def touched(cell, n, periodic, overlap):
    """Cells touched by the task of `cell` (x fastest): the 3x3x3 block around it, or the
    3x3x2 block z..z+1 for overlap 18; outside a non-periodic grid, cells are dropped."""
    nx, ny, nz = n
    x, y, z = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    zr = (0, 1) if overlap == 18 else (-1, 0, 1)
    out = set()
    for dx, dy, dz in itertools.product((-1, 0, 1), (-1, 0, 1), zr):
        p = [x + dx, y + dy, z + dz]
        ok = True
        for d in range(3):
            if not 0 <= p[d] < n[d]:
                if not periodic[d]:
                    ok = False
                p[d] %= n[d]
        if ok:
            out.add(p[0] + nx * (p[1] + ny * p[2]))
    return out


def direct_predecessors(order, n, periodic, overlap):
    """List of sorted predecessor task indices for each task of `order` (cells in run order)."""
    acc = [touched(c, n, periodic, overlap) for c in order]
    preds = []
    for t in range(len(order)):
        ps = set()
        for c in acc[t]:
            for s in range(t - 1, -1, -1):
                if c in acc[s]:
                    ps.add(s)
                    break
        preds.append(sorted(ps))
    return preds


def overlapping(a, b, n, periodic, overlap):
    return bool(touched(a, n, periodic, overlap) & touched(b, n, periodic, overlap))
