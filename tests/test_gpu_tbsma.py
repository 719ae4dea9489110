"""The many-body (TB-SMA, Cleri-Rosato copper) path against the FP64 oracle.

Inputs: fcc copper at its lattice constant 3.615 A with Gaussian displacements of
0.08 A (about the thermal amplitude at room temperature) and thermal velocities at
kT = 0.02585 eV (eV, Angstrom, amu; the time unit is 10.18 fs); isolated pairs at
r_cut (1 -/+ 1e-7).  Bars as for the pair potential in mixed precision: forces per atom
within 2e-5 of max(|F_i|, F_rms), energy and virial within 1e-6 relative, bit-identical
forces for any input order; a 20-step trajectory within 1e-6 A of the oracle's many-body
velocity-Verlet run.
"""
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
from paper_1305_4196_gb300 import mdgb as M  # noqa: E402

CU = O.TBSMAParams.copper()
MASS = 63.546
SKIN = 0.4
KT = 0.02585


def crystal(n_cells=16, jitter=0.08, seed=3, T=KT):
    pos, box = W.fcc_lattice(n_cells, n_cells, n_cells, 3.615)
    pos = W.gaussian_jitter(pos, box, jitter, seed, stream=2)
    vel = W.thermal_velocities(np.full(len(pos), MASS), T, seed, stream=1)
    return pos, vel, box


def make(pos, vel, box, dt=0.2, P=CU, **kw):
    s = M.System(len(pos), box, r_cut=P.rc, skin=SKIN, mass=MASS, dt=dt, precision=M.MD_MIXED, **kw)
    s.set_tbsma(P.A, P.xi, P.p, P.q, P.r0, P.rc)
    s.set_state(np.ascontiguousarray(pos), np.ascontiguousarray(vel), np.zeros(len(pos), dtype=np.int32))
    return s


def force_error(F, Fref):
    mag = np.sqrt((Fref ** 2).sum(1))
    frms = np.sqrt((mag ** 2).mean())
    return float((np.sqrt(((F - Fref) ** 2).sum(1)) / np.maximum(mag, frms)).max())


def test_forces_energy_virial_match_oracle():
    pos, vel, box = crystal()
    s = make(pos, vel, box)
    F = s.forces()
    Fref, E_ref, vir_ref = O.tbsma_forces(pos, box, CU)
    assert force_error(F, Fref) <= 2e-5
    pe, _, vir = s.energy_virial()
    assert abs(pe - E_ref) <= 1e-6 * abs(E_ref)
    assert np.abs(vir - vir_ref).max() <= 1e-6 * np.abs(E_ref)
    assert s.info()["n_builds"] >= 1


def test_forces_bit_identical_for_any_input_order():
    pos, vel, box = crystal(seed=5)
    F = make(pos, vel, box).forces()
    perm = np.random.default_rng(2).permutation(len(pos))
    Fp = make(pos[perm], vel[perm], box).forces()
    assert np.array_equal(Fp, F[perm])
    assert np.array_equal(make(pos, vel, box).forces(), F)


def test_cutoff_decided_by_the_definition():
    """Isolated pairs at r_cut (1 -/+ 1e-7): the densities and forces of both passes decide
    the cutoff by the FP64 definition."""
    box = np.array([80.0, 80.0, 80.0])
    pos = W.threshold_pairs(216, box, CU.rc, 1e-7, seed=15)
    s = make(pos, np.zeros_like(pos), box)
    F = s.forces()
    Fref, E_ref, _ = O.tbsma_forces(pos, box, CU)
    assert np.abs(Fref).max() > 1e-3  # half the pairs interact
    assert np.abs(F - Fref).max() <= 2e-5 * np.abs(Fref).max()
    pe, _, _ = s.energy_virial()
    assert abs(pe - E_ref) <= 1e-6 * abs(E_ref)


def test_trajectory_follows_oracle_velocity_verlet():
    pos, vel, box = crystal(n_cells=8, seed=7)
    dt, steps = 0.2, 20
    s = make(pos, vel, box, dt=dt)
    s.step(steps)
    p_gpu, v_gpu, img = s.get_state()
    ref = O.run_nve_tbsma(pos, vel, box, CU, MASS, dt, SKIN, steps)
    x = ref["pos"] + ref["image"] * box
    assert np.abs(p_gpu + img * box - x).max() <= 1e-6
    assert np.abs(v_gpu - ref["vel"]).max() <= 1e-6 * np.abs(ref["vel"]).max()


def test_energy_drift_small_over_1000_steps():
    """NVE at room temperature, 1 fs steps for 10 ps: total energy drift per atom stays
    far below kT (the potential is cut without a shift, so crossings move E slightly)."""
    pos, vel, box = crystal(n_cells=10, seed=8)
    s = make(pos, vel, box, dt=0.0982)
    pe0, ke0, _ = s.energy_virial()
    s.step(1000)
    pe1, ke1, _ = s.energy_virial()
    n = len(pos)
    assert abs((pe1 + ke1) - (pe0 + ke0)) / n < 2e-3 * KT
    assert 0.3 * KT < 2 * ke1 / (3 * n) < 1.5 * KT  # equipartition with the potential: about half of KT


def test_switch_back_to_pair_potential_and_argument_errors():
    pos, vel, box = crystal(n_cells=8, seed=9)
    s = make(pos, vel, box)
    s.forces()
    P = O.LJParams.single(eps=0.4, sig=2.3, rc=CU.rc, mass=MASS)
    s.set_params(P.eps, P.sig)
    Fref, _, _ = O.lj_forces(pos, box, P)
    assert force_error(s.forces(), Fref) <= 2e-5
    with pytest.raises(M.MDError):
        s.set_tbsma(CU.A, CU.xi, CU.p, CU.q, CU.r0, CU.rc + 1.0)  # beyond the lists' radius
    f64 = M.System(len(pos), box, r_cut=CU.rc, skin=SKIN, mass=MASS, precision=M.MD_FP64)
    with pytest.raises(M.MDError):
        f64.set_tbsma(CU.A, CU.xi, CU.p, CU.q, CU.r0, CU.rc)
    half = M.System(len(pos), box, r_cut=CU.rc, skin=SKIN, mass=MASS, list_kind=M.MD_LIST_HALF_COLOUR8)
    with pytest.raises(M.MDError):
        half.set_tbsma(CU.A, CU.xi, CU.p, CU.q, CU.r0, CU.rc)
    with pytest.raises(M.MDError):
        s.set_tbsma(CU.A, CU.xi, CU.p, 40.0, CU.r0, CU.rc)  # xi^2 exp(2q) beyond the density range
    s.set_tbsma(CU.A, CU.xi, CU.p, CU.q, CU.r0, CU.rc)
    with pytest.raises(M.MDError):
        s.forces_backward(np.zeros_like(pos))  # derivatives are for the pair potential


def test_full_size_bulk_copper():
    """The benchmark's many-body workload, the paper's bulk copper size: 1,000,188 atoms
    (63^3 fcc cells) at room-temperature displacements, all forces and the energy against
    the oracle, after 20 steps in the benchmark's launch configuration."""
    pos, vel, box = crystal(n_cells=63, seed=11)
    s = make(pos, vel, box, dt=0.0982)
    s.step(20)
    p, _, _ = s.get_state()
    F = s.forces()
    Fref, E_ref, _ = O.tbsma_forces(p, box, CU)
    assert force_error(F, Fref) <= 2e-5
    pe, _, _ = s.energy_virial()
    assert abs(pe - E_ref) <= 1e-6 * abs(E_ref)


def test_on_a_coarser_linear_grid():
    """The two TB-SMA passes on the coarser, linearly numbered grid a pair-potential system
    takes at its first build: a 296,352-atom LJ-unit liquid (42^3 fcc cells at rho* = 0.8442,
    22 instead of 24 cells per side), switched to a TB-SMA parameter set in the same units
    (A = 0.1, xi = 1, p = 10, q = 2.5, r0 = 1.12, r_cut = 2.5).  Forces, energy and virial
    against the oracle at the mixed bars."""
    sysm = W.lj_fcc(42, seed=6, jitter=0.05)
    s = M.System(sysm.n, sysm.box, r_cut=2.5, skin=0.3, precision=M.MD_MIXED)
    s.set_state(sysm.pos, sysm.vel, sysm.species)
    s.forces()
    assert s.info()["ncell"] == [22, 22, 22]
    P = O.TBSMAParams(0.1, 1.0, 10.0, 2.5, 1.12, 2.5)
    s.set_tbsma(P.A, P.xi, P.p, P.q, P.r0, P.rc)
    F = s.forces()
    Fref, E_ref, vir_ref = O.tbsma_forces(sysm.pos, sysm.box, P)
    assert force_error(F, Fref) <= 2e-5
    pe, _, vir = s.energy_virial()
    assert abs(pe - E_ref) <= 1e-6 * abs(E_ref)
    assert np.abs(vir - vir_ref).max() <= 1e-6 * np.abs(vir_ref[:3]).max()

