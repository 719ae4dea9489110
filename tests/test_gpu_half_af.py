"""The atom-free Newton-3 half list (MD_LIST_HALF_ATOMIC_FREE) against the FP64 oracle.

Each pair is evaluated once, in 8 colour launches of 2x2x2-cell blocks, 14 barrier-separated
half-shell phases inside a block and conflict-free steps inside a cell's warp, with no atomic
operation on any force.  Bars as for the other mixed paths: neighbour pairs bit-exact, forces
per atom within 2e-5 of max(|F_i|, F_rms), energy and virial within 1e-6; and, because every
reaction is the exact negative of its action, a fixed-point total force of exactly zero and
bit-identical forces for any input order.
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

RC, SKIN, DT = 2.5, 0.3, 0.005
AF = M.MD_LIST_HALF_ATOMIC_FREE


def force_error(F, Fref):
    mag = np.sqrt((Fref ** 2).sum(1))
    frms = np.sqrt((mag ** 2).mean())
    return float((np.sqrt(((F - Fref) ** 2).sum(1)) / np.maximum(mag, frms)).max())


def make(sysm, lst=AF, params=None, **kw):
    params = params or O.LJParams.single()
    s = M.System(sysm.n, sysm.box, r_cut=float(params.rc.max()), skin=SKIN, eps=params.eps, sigma=params.sig,
                 mass=params.mass, dt=DT, precision=M.MD_MIXED, list_kind=lst,
                 rcut=params.rc if params.nsp > 1 else None, **kw)
    s.set_state(np.ascontiguousarray(sysm.pos), np.ascontiguousarray(sysm.vel), np.ascontiguousarray(sysm.species))
    return s


def liquid(n_cells=14, seed=21):
    return W.lj_fcc(n_cells, seed=seed, jitter=0.05)


def gas():
    box = np.array([22.5, 25.0, 31.0])
    pos = W.random_gas(3000, box, seed=5)
    return W.System(pos, np.zeros_like(pos), np.zeros(3000, dtype=np.int32), box, "gas")


def threshold():
    box = np.array([30.0, 30.0, 30.0])
    pos = W.threshold_pairs(343, box, RC + SKIN, 1e-12, seed=9)
    return W.System(pos, np.zeros_like(pos), np.zeros(len(pos), dtype=np.int32), box, "threshold")


def slab():
    return W.slab_nanoparticles(L=40.0, n_particles=4, r_min=3.0, r_max=5.0, seed=3)


KINDS = {"liquid": liquid, "gas": gas, "threshold": threshold, "slab": slab}


@pytest.mark.parametrize("kind", sorted(KINDS))
def test_pair_set_bit_exact(kind):
    sysm = KINDS[kind]()
    s = make(sysm)
    assert np.array_equal(s.neighbors(), O.neighbor_pairs(sysm.pos, sysm.box, RC + SKIN))


@pytest.mark.parametrize("kind", ["liquid", "slab"])
def test_forces_energy_virial_vs_oracle(kind):
    sysm = KINDS[kind]()
    s = make(sysm)
    Fref, pe_ref, vir_ref = O.lj_forces(sysm.pos, sysm.box, O.LJParams.single())
    assert force_error(s.forces(), Fref) <= 2e-5
    pe, _, vir = s.energy_virial()
    assert abs(pe - pe_ref) <= 1e-6 * abs(pe_ref)
    assert np.abs(vir - vir_ref).max() <= 1e-6 * np.abs(vir_ref[:3]).max()


def test_total_force_exactly_zero_and_order_independent():
    """Every reaction is the exact negative of its action: the Q31.32 total is zero in
    integers, and the forces do not depend on run or input order."""
    sysm = liquid()
    F = make(sysm).forces()
    q = np.rint(F * 2.0 ** 32).astype(np.int64)
    assert np.array_equal(q.astype(np.float64) * 2.0 ** -32, F)
    assert np.all(q.sum(axis=0) == 0)
    assert np.array_equal(make(sysm).forces(), F)
    perm = np.argsort(W.splitmix64(3, 3, sysm.n))
    sp = W.System(sysm.pos[perm], sysm.vel[perm], sysm.species[perm], sysm.box)
    assert np.array_equal(make(sp).forces(), F[perm])


def test_agrees_with_the_atomic_half_list_and_the_full_list():
    sysm = liquid(14, seed=4)
    a = make(sysm).forces()
    b = make(sysm, lst=M.MD_LIST_HALF_COLOUR8).forces()
    c = make(sysm, lst=M.MD_LIST_FULL).forces()
    assert force_error(a, b) <= 2e-5 and force_error(a, c) <= 2e-5


def test_multispecies_per_pair_cutoff():
    a = W.lattice_constant(1.2)
    pos, box = W.fcc_lattice(16, 16, 16, a)
    pos = W.gaussian_jitter(pos, box, 0.03, seed=4)
    sp = W.species_shuffle(len(pos), 0.2, seed=4)
    sysm = W.System(pos, np.zeros_like(pos), sp, box)
    sig = np.array([[1.0, 0.8], [0.8, 0.88]])
    P = O.LJParams([[1.0, 1.5], [1.5, 0.5]], sig, 2.5 * sig, [1.0, 1.0])
    Fref, pe_ref, _ = O.lj_forces(pos, box, P, species=sp)
    s = make(sysm, params=P)
    assert force_error(s.forces(), Fref) <= 2e-5
    assert abs(s.energy_virial()[0] - pe_ref) <= 1e-6 * abs(pe_ref)


def test_cells_of_more_than_32_atoms_take_a_second_pass():
    """rho* = 1.3 in a 26.2 sigma box (8 cells of 3.27 sigma per side): about 45 atoms per
    cell, so every warp runs a second pass per phase for the atoms past the 32nd."""
    sysm = W.lj_fcc(18, rho=1.3, seed=7, jitter=0.03)
    s = make(sysm)
    Fref, _, _ = O.lj_forces(sysm.pos, sysm.box, O.LJParams.single())
    F = s.forces()
    assert force_error(F, Fref) <= 2e-5
    q = np.rint(F * 2.0 ** 32).astype(np.int64)
    assert np.all(q.sum(axis=0) == 0)
    assert np.array_equal(s.neighbors(), O.neighbor_pairs(sysm.pos, sysm.box, RC + SKIN))


def test_dense_cell_is_reported():
    """A cell of more than 63 atoms is refused with MD_ERR_CELL_OVERFLOW (the per-tile sums
    stay exact only up to 504 terms), not evaluated wrongly."""
    sysm = W.lj_fcc(12, rho=2.0, seed=7, jitter=0.01)  # 4 cells of 3.78 sigma: ~108 atoms each
    s = M.System(sysm.n, sysm.box, r_cut=RC, skin=SKIN, precision=M.MD_MIXED, list_kind=AF)
    with pytest.raises(M.MDError) as e:
        s.set_state(sysm.pos, sysm.vel, sysm.species)
        s.forces()
    assert e.value.code == M.MD_ERR_CELL_OVERFLOW


def test_close_pairs_exact_or_reported():
    """Pairs at 0.45 sigma (terms beyond the split, through the warps' 64-bit queues) are
    exact; a pair at 0.40 sigma is reported."""
    sysm = liquid()
    rng = np.random.default_rng(21)
    pos = sysm.pos.copy()
    picks = rng.choice(sysm.n // 2, 16, replace=False)
    for c in range(4):
        i, js = picks[4 * c], picks[4 * c + 1:4 * c + 4]
        for k, j in enumerate(js):
            ang = (k - 1) * np.pi / 3
            pos[j] = W.wrap(pos[i] + 0.45 * np.array([np.cos(ang), np.sin(ang), 0.0]), sysm.box)
    F = make(W.System(pos, sysm.vel, sysm.species, sysm.box)).forces()
    Fref, _, _ = O.lj_forces(pos, sysm.box, O.LJParams.single())
    assert np.abs(F - Fref).max() <= 2e-5 * np.abs(Fref).max()
    # (no integer total here: forces above 2^21 eps/sigma exceed the 53-bit mantissa of the
    # FP64 values they are returned as, so rint(F * 2^32) no longer recovers the Q31.32 sums)
    pos2 = sysm.pos.copy()
    pos2[picks[1]] = W.wrap(pos2[picks[0]] + np.array([0.40, 0.0, 0.0]), sysm.box)
    with pytest.raises(M.MDError) as e:
        make(W.System(pos2, sysm.vel, sysm.species, sysm.box)).forces()
    assert e.value.code == M.MD_ERR_NONFINITE


def test_cutoff_decided_by_the_definition():
    box = np.array([30.0, 30.0, 30.0])
    pos = W.threshold_pairs(216, box, RC, 1e-7, seed=13)
    sysm = W.System(pos, np.zeros_like(pos), np.zeros(len(pos), dtype=np.int32), box)
    F = make(sysm).forces()
    Fref, _, _ = O.lj_forces(pos, box, O.LJParams.single())
    assert np.abs(F - Fref).max() <= 2e-5 * np.abs(Fref).max()


def test_trajectory_and_energy():
    sysm = W.lj_fcc(14, seed=1)  # 10,976 atoms, 8 cells per side
    s = make(sysm)
    pe0, ke0, _ = s.energy_virial()
    s.step(20)
    pos, vel, img = s.get_state()
    ref = O.run_nve(sysm.pos, sysm.vel, sysm.box, O.LJParams.single(), DT, SKIN, 20)
    assert np.abs(pos + img * sysm.box - (ref["pos"] + ref["image"] * sysm.box)).max() < 1e-6
    s.step(80)
    pe1, ke1, _ = s.energy_virial()
    ref = O.run_nve(sysm.pos, sysm.vel, sysm.box, O.LJParams.single(), DT, SKIN, 100, history=True)
    assert abs((pe1 + ke1) - (ref["pe"][-1] + ref["ke"][-1])) / sysm.n < 1e-4


def test_fp64_is_refused():
    with pytest.raises(M.MDError) as e:
        M.System(1000, np.array([20.0, 20.0, 20.0]), precision=M.MD_FP64, list_kind=AF)
    assert e.value.code == M.MD_ERR_ARG
