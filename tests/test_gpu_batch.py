"""Ensembles of independent systems (include/mdgb_batch.h) against the FP64 oracle.

Inputs: seeded systems of uneven size from workloads.batch_ensemble (fcc sites with
vacancies at exact density, Gaussian jitter, thermal velocities), the shape of the
512-system ensemble workload, with sizes chosen so that both execution paths of the
one persistent launch (one CTA per system, and block tasks shared by all CTAs for the
larger ones) are exercised.  Bars: forces within 2e-5 (per atom, against the RMS),
potential energy within 1e-6, kinetic energy within 1e-12; bit-identical repeats; short
trajectories close to the oracle's.
"""
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_1305_4196_gb300 import build as B  # noqa: E402
from paper_1305_4196_gb300 import workloads as W  # noqa: E402

B.build()
from paper_1305_4196_gb300 import batch as BA  # noqa: E402
from paper_1305_4196_gb300 import mdgb as M  # noqa: E402

P = O.LJParams.single()


def ensemble(k=10, seed=9, n_max=12000):
    return W.batch_ensemble(n_systems=k, seed=seed, n_max=n_max)


def force_error(F, Fref):
    mag = np.sqrt((Fref ** 2).sum(1))
    frms = np.sqrt((mag ** 2).mean())
    return float((np.sqrt(((F - Fref) ** 2).sum(1)) / np.maximum(mag, frms)).max())


def split(a, systems):
    out, o = [], 0
    for s in systems:
        out.append(a[o:o + s.n])
        o += s.n
    return out


def test_both_paths_used_and_forces_match_oracle():
    systems = ensemble()
    b = BA.from_systems(systems)
    path, threads, R = b.layout()
    assert set(path.tolist()) == {0, 1}
    for s, F in zip(systems, split(b.forces(), systems)):
        Fref, _, _ = O.lj_forces(s.pos, s.box, P)
        assert force_error(F, Fref) <= 2e-5


def test_energies_match_oracle():
    systems = ensemble(seed=10)
    b = BA.from_systems(systems)
    pe, ke = b.energies()
    for k, s in enumerate(systems):
        _, pe_ref, _ = O.lj_forces(s.pos, s.box, P)
        ke_ref = O.kinetic(s.vel, P)
        assert abs(pe[k] - pe_ref) <= 1e-6 * abs(pe_ref)
        assert abs(ke[k] - ke_ref) <= 1e-12 * ke_ref


def test_steps_are_deterministic_and_follow_the_oracle():
    """20 steps: two ensembles from the same input agree bit for bit; every system stays
    within 1e-5 sigma of the FP64 oracle's trajectory (mixed-precision forces)."""
    systems = ensemble(k=8, seed=11, n_max=6000)
    a = BA.from_systems(systems)
    b = BA.from_systems(systems)
    a.step(20)
    b.step(13)
    b.step(7)
    pa, va, ia = a.get_state()
    pb, vb, ib = b.get_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb) and np.array_equal(ia, ib)
    for s, p, im in zip(systems, split(pa, systems), split(ia, systems)):
        r = O.run_nve(s.pos, s.vel, s.box, P, 0.005, 0.3, 20)
        un = p + im * s.box
        ref = r["pos"] + r["image"] * s.box
        assert np.abs(un - ref).max() <= 1e-5


def test_energy_after_100_steps_matches_oracle():
    """The potential is unshifted, so the total energy jumps by u(r_cut) whenever a pair
    crosses the cutoff and drifts while an fcc start melts; the reference for the energy
    after 100 steps is therefore the FP64 oracle's own trajectory (per atom, within 1e-4)."""
    systems = [W.fcc_vacancies(n, 0.8, 0.9, seed=5 + n) for n in (300, 900, 6000)]
    b = BA.from_systems(systems)
    assert b.layout()[0].tolist() == [0, 0, 1]  # the 6,000-atom system runs as block tasks
    b.step(100)
    pe, ke = b.energies()
    for k, s in enumerate(systems):
        ref = O.run_nve(s.pos, s.vel, s.box, P, 0.005, 0.3, 100, history=True)
        e_ref = ref["pe"][-1] + ref["ke"][-1]
        assert abs(pe[k] + ke[k] - e_ref) / s.n < 1e-4


def test_autotune_writes_and_reads_its_cache():
    systems = ensemble(k=6, seed=12, n_max=8000)
    b = BA.from_systems(systems)
    path = os.path.join(tempfile.mkdtemp(), "tune.json")
    before = b.get_state()
    b.autotune(path)
    after = b.get_state()
    assert all(np.array_equal(x, y) for x, y in zip(before, after))  # the state is restored
    text = open(path).read()
    assert '"gpu":' in text and '"shape": [' in text
    lay = b.layout()
    c = BA.from_systems(systems)
    c.autotune(path)
    lay2 = c.layout()
    assert all(np.array_equal(x, y) for x, y in zip(lay, lay2))
    for s, F in zip(systems, split(c.forces(), systems)):
        assert force_error(F, O.lj_forces(s.pos, s.box, P)[0]) <= 2e-5


def test_cutoff_decided_by_the_definition():
    """Pairs at r_cut (1 -/+ 1e-7) in small boxes on the one-CTA path: the cutoff is decided in
    FP64 as the definition, so the forces match the oracle."""
    systems = []
    for k in range(3):
        box = np.array([14.0, 14.0, 14.0])
        pos = W.threshold_pairs(27, box, 2.5, 1e-7, seed=20 + k)
        systems.append(W.System(pos, np.zeros_like(pos), np.zeros(len(pos), dtype=np.int32), box))
    b = BA.from_systems(systems)
    assert np.all(b.layout()[0] == 0)
    for s, F in zip(systems, split(b.forces(), systems)):
        Fref, _, _ = O.lj_forces(s.pos, s.box, P)
        assert np.abs(Fref).max() > 0.03
        assert np.abs(F - Fref).max() <= 2e-5 * np.abs(Fref).max()


def test_full_ensemble_sampled_systems():
    """The benchmark's ensemble itself: 512 systems, 3.6 million atoms, autotuned, 10 steps.
    Forces of sampled systems on both paths (one CTA per system and block tasks), at the
    state the GPU reached, match the oracle's."""
    systems = W.batch_ensemble(512, seed=4)
    b = BA.from_systems(systems)
    b.autotune(os.path.join(tempfile.mkdtemp(), "tune.json"))
    b.step(10)
    pos, _, _ = b.get_state()
    F = b.forces()
    path, _, _ = b.layout()
    offs = np.concatenate([[0], np.cumsum([s.n for s in systems])])
    picks = [k for k in range(512) if path[k] == 0][::60] + [k for k in range(512) if path[k] == 1][::40]
    assert len(picks) >= 8
    for k in picks:
        sl = slice(offs[k], offs[k + 1])
        Fref, _, _ = O.lj_forces(pos[sl], systems[k].box, P)
        assert force_error(F[sl], Fref) <= 2e-5, k


def test_cutoff_decided_by_the_definition_in_block_tasks():
    """Pairs at r_cut (1 -/+ 1e-7), 5 sigma apart, in a 2,200-atom system, which runs as
    block tasks."""
    box = np.array([55.0, 55.0, 55.0])
    pos = W.threshold_pairs(1100, box, 2.5, 1e-7, seed=31)
    s = W.System(pos, np.zeros_like(pos), np.zeros(len(pos), dtype=np.int32), box)
    b = BA.from_systems([s])
    assert b.layout()[0].tolist() == [1]
    Fref, _, _ = O.lj_forces(s.pos, s.box, P)
    F = b.forces()
    assert np.abs(Fref).max() > 0.03
    assert np.abs(F - Fref).max() <= 2e-5 * np.abs(Fref).max()


def test_close_pairs_in_block_tasks_exact():
    """Pairs at 0.6 sigma (force terms beyond the 32-bit split) in a block-task system are
    finished by the exact pass: forces match the oracle."""
    s = W.fcc_vacancies(6000, 0.8, 0.9, seed=41)
    pos = s.pos.copy()
    for i in range(0, 40, 4):
        pos[i + 1] = W.wrap(pos[i] + np.array([0.6, 0.0, 0.0]), s.box)
    s2 = W.System(pos, s.vel, s.species, s.box)
    b = BA.from_systems([s2])
    assert b.layout()[0].tolist() == [1]
    Fref, _, _ = O.lj_forces(pos, s.box, P)
    assert np.abs(b.forces() - Fref).max() <= 2e-5 * np.abs(Fref).max()


def test_wait_timeout_is_reported_without_a_fault():
    """A held system never becomes ready, so the CTAs run out of work and out of their wait
    budget: the call returns MD_ERR_TIMEOUT, the context stays usable, and after a new state
    the ensemble steps exactly like a fresh one."""
    systems = ensemble(k=6, seed=13, n_max=6000)
    b = BA.from_systems(systems)
    b.set_wait_budget(2_000_000, held_system=int(np.argmax([s.n for s in systems])))
    with pytest.raises(M.MDError) as e:
        b.step(5)
    assert e.value.code == M.MD_ERR_TIMEOUT
    b.set_wait_budget(0, -1)
    b.set_state(np.ascontiguousarray(np.concatenate([s.pos for s in systems])),
                np.ascontiguousarray(np.concatenate([s.vel for s in systems])))
    b.step(5)
    c = BA.from_systems(systems)
    c.step(5)
    assert all(np.array_equal(x, y) for x, y in zip(b.get_state(), c.get_state()))


def test_empty_system_in_the_ensemble():
    """A system of no atoms beside a one-CTA and a block system: it has no work and zero
    energies, and the others match the oracle."""
    a = W.fcc_vacancies(300, 0.8, 0.9, seed=51)
    c = W.fcc_vacancies(7000, 0.8, 0.9, seed=52)
    empty = W.System(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, dtype=np.int32), np.array([10.0, 10.0, 10.0]))
    systems = [a, empty, c]
    b = BA.from_systems(systems)
    assert b.layout()[0].tolist() == [0, 0, 1]
    F = b.forces()
    for s, Fs in zip(systems, split(F, systems)):
        if s.n:
            assert force_error(Fs, O.lj_forces(s.pos, s.box, P)[0]) <= 2e-5
    pe, ke = b.energies()
    assert pe[1] == 0.0 and ke[1] == 0.0
    b.step(5)
    pos, _, _ = b.get_state()
    assert pos.shape == (a.n + c.n, 3) and np.isfinite(pos).all()
