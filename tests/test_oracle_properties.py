"""Property tests of the oracle on random small inputs (hypothesis, CPU only): the
linked-cell pair set equals the O(N^2) definition for any box and atom count, and forces
are invariant under a translation of all atoms and under a permutation of their order."""
import numpy as np
import pytest

pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_1305_4196_gb300 import workloads as W  # noqa: E402


@settings(max_examples=30, deadline=None)
@given(n=st.integers(2, 400), lx=st.floats(8.5, 14.0), ly=st.floats(8.5, 14.0), lz=st.floats(8.5, 14.0),
       seed=st.integers(0, 2**31 - 1))
def test_cell_pair_set_equals_brute_force(n, lx, ly, lz, seed):
    box = np.array([lx, ly, lz])
    pos = W.random_gas(n, box, seed=seed)
    assert np.array_equal(O.neighbor_pairs(pos, box, 2.8, brute=True), O.neighbor_pairs(pos, box, 2.8, brute=False))


@settings(max_examples=12, deadline=None)
@given(n=st.integers(300, 1500), rho=st.floats(0.6, 1.0), seed=st.integers(0, 2**31 - 1),
       shift=st.tuples(st.floats(-50, 50), st.floats(-50, 50), st.floats(-50, 50)))
def test_forces_translation_and_permutation_invariant(n, rho, seed, shift):
    s = W.fcc_vacancies(n, rho, 1.0, seed=seed % 100000)
    P = O.LJParams.single()
    F0, e0, _ = O.lj_forces(s.pos, s.box, P)
    moved = W.wrap(s.pos + np.array(shift), s.box)
    F1, e1, _ = O.lj_forces(moved, s.box, P)
    scale = np.sqrt((F0 ** 2).sum(1).mean())
    assert np.abs(F1 - F0).max() <= 1e-9 * scale
    assert abs(e1 - e0) <= 1e-10 * abs(e0)
    perm = np.random.default_rng(seed).permutation(n)
    F2, e2, _ = O.lj_forces(s.pos[perm], s.box, P)
    assert np.abs(F2 - F0[perm]).max() <= 1e-9 * scale
    assert abs(e2 - e0) <= 1e-10 * abs(e0)
