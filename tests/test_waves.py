"""The paper's wave schedule (host tool, include/mdgb_waves.h) against the paper's own
examples and the definitions of Sec. II.B and the Appendix.

Golden values: tests/golden/waves_appendix.json (the Appendix's covers of D = 14 cells,
its statement of the fifth wave of a periodic 14 x 6 grid, and the wave counts
27/36/48/64).  Invariants: every cell in exactly one wave, no two tasks of a wave
touching a common cell, every dimension covered by three or four sets; the forward and
the backward wave method build the same graph, equal to a brute-force construction from
the definition, and any two tasks touching a common cell are ordered by it.
"""
import itertools
import json
import os

import numpy as np
import pytest

from paper_1305_4196_gb300 import build as B

B.build()
from paper_1305_4196_gb300 import waves as WV  # noqa: E402
from oracle import waves_oracle as WO  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "waves_appendix.json")))


def sets_as_lists(set_of, k):
    return [sorted((np.flatnonzero(set_of == j) + 1).tolist()) for j in range(k)]


def test_appendix_1d_covers():
    s, k = WV.sets_1d(14, False)
    assert (s + 1).tolist() == GOLD["nonperiodic_D14_coverage"]
    assert sets_as_lists(s, k) == [sorted(x) for x in GOLD["nonperiodic_D14_sets"]]
    s, k = WV.sets_1d(14, True)
    assert (s + 1).tolist() == GOLD["periodic_D14_coverage"]
    assert sets_as_lists(s, k) == [sorted(x) for x in GOLD["periodic_D14_sets"]]


def test_appendix_2d_example():
    """Periodic 14 x 6 grid (one layer in z): waves 1-4 use the y set {1, 4} with the 1-D x
    sets; wave 5 reuses the fourth x set {9, 12}, filled to {9, 12, 1, 4}, with y set {2, 5}."""
    w, k = WV.waves([14, 6, 3], [1, 1, 1])
    grid = w.reshape(3, 6, 14)[0]  # layer z = 0
    cov = GOLD["periodic_D14_coverage"]
    for x in range(14):
        for y in GOLD["periodic_14x6_waves_1_to_4_y_set"]:
            assert grid[y - 1, x] + 1 == cov[x]
    five = [(y, x) for y in range(6) for x in range(14) if grid[y, x] == 4]
    assert sorted({x + 1 for _, x in five}) == sorted(GOLD["periodic_14x6_wave_5_x_set"])
    assert sorted({y + 1 for y, _ in five}) == GOLD["periodic_14x6_wave_5_y_set"]


@pytest.mark.parametrize("n,periodic,expect", [
    ((6, 6, 6), 1, 27), ((14, 6, 6), 1, 36), ((14, 14, 6), 1, 48), ((14, 14, 14), 1, 64),
    ((14, 14, 14), 0, 27), ((12, 9, 15), 1, 27)])
def test_wave_counts(n, periodic, expect):
    assert expect in GOLD["wave_counts_3d"]
    assert WV.waves(n, [periodic] * 3)[1] == expect


@pytest.mark.parametrize("D", range(3, 61))
@pytest.mark.parametrize("periodic", [0, 1])
def test_1d_sets_from_any_start(D, periodic):
    """From every start index: an exact cover, members of a set at least three apart
    (periodic distance), and three or four sets - except a periodic dimension of 5 cells,
    where every two cells are within two of each other, so each set holds one cell."""
    for start in range(D):
        s, k = WV.sets_1d(D, periodic, 3, start)
        assert k == 5 if (periodic and D == 5) else k in (3, 4)
        for j in range(k):
            m = np.flatnonzero(s == j)
            for a, b in itertools.combinations(m, 2):
                d = abs(int(a) - int(b))
                if periodic:
                    d = min(d, D - d)
                assert d >= 3


@pytest.mark.parametrize("n,periodic,overlap", [
    ((7, 5, 6), (1, 1, 1), 27), ((8, 3, 4), (0, 1, 1), 27), ((6, 7, 5), (1, 0, 0), 27),
    ((7, 5, 6), (1, 1, 1), 18), ((6, 6, 4), (1, 1, 0), 18)])
def test_waves_cover_and_do_not_overlap(n, periodic, overlap):
    w, k = WV.waves(n, periodic, overlap)
    assert w.min() == 0 and w.max() == k - 1
    for j in range(k):
        cells = np.flatnonzero(w == j)
        for a, b in itertools.combinations(cells, 2):
            assert not WO.overlapping(int(a), int(b), n, periodic, overlap)


@pytest.mark.parametrize("n,periodic,overlap", [
    ((7, 5, 6), (1, 1, 1), 27), ((6, 4, 5), (0, 1, 1), 27), ((7, 5, 6), (1, 1, 1), 18)])
def test_schedule_forward_backward_and_definition(n, periodic, overlap):
    tc, npf, sf, suf = WV.schedule(n, periodic, overlap, backward=False)
    tb, npb, sb, sub = WV.schedule(n, periodic, overlap, backward=True)
    assert np.array_equal(tc, tb) and np.array_equal(npf, npb)
    assert np.array_equal(sf, sb) and np.array_equal(suf, sub)
    preds = WO.direct_predecessors(tc.tolist(), n, periodic, overlap)
    assert [len(p) for p in preds] == npf.tolist()
    T = len(tc)
    succ_ref = [[] for _ in range(T)]
    for t, ps in enumerate(preds):
        for p in ps:
            succ_ref[p].append(t)
    assert [sorted(x) for x in succ_ref] == [suf[sf[t]:sf[t + 1]].tolist() for t in range(T)]
    # every pair of tasks touching a common cell is ordered by the graph
    reach = np.zeros((T, T), dtype=bool)
    for t in range(T - 1, -1, -1):
        for s in suf[sf[t]:sf[t + 1]]:
            reach[t, s] = True
            reach[t] |= reach[s]
    for a, b in itertools.combinations(range(T), 2):
        if WO.overlapping(int(tc[a]), int(tc[b]), n, periodic, overlap):
            assert reach[a, b]


def test_critical_path_is_at_most_the_wave_count():
    n, periodic = (14, 14, 14), (1, 1, 1)
    _, k = WV.waves(n, periodic)
    tc, npred, start, succ = WV.schedule(n, periodic)
    assert WV.critical_path(npred, start, succ) <= k


def test_cell_counts_must_have_three_entries():
    with pytest.raises(ValueError):
        WV.waves([4, 4], True)
    with pytest.raises(ValueError):
        WV.schedule([4, 4, 4, 4], True)
