"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: neighbour sets bit-exact; forces per atom e_i = |F_i - F_i^ref| /
max(|F_i^ref|, F_rms) <= 1e-12 (FP64 path) and <= 2e-5 (mixed path); energy
and virial relative error <= 1e-12 (FP64) and <= 1e-6 (mixed); FP64
trajectories within 1e-10 sigma over 100 steps; fixed-point forces bit-equal
across list kinds, runs and input orderings, with an exactly zero sum.
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
PRECISIONS = {"fp64": M.MD_FP64, "mixed": M.MD_MIXED}
LISTS = {"full": M.MD_LIST_FULL, "half": M.MD_LIST_HALF_COLOUR8}
TOL = {"fp64": 1e-12, "mixed": 2e-5}


def force_error(F, Fref):
    mag = np.sqrt((Fref ** 2).sum(1))
    frms = np.sqrt((mag ** 2).mean())
    e = np.sqrt(((F - Fref) ** 2).sum(1)) / np.maximum(mag, frms)
    return float(e.max())


def make(sysm, precision="mixed", lst="full", params=None, **kw):
    if params is None:
        params = O.LJParams.single()
    s = M.System(sysm.n, sysm.box, r_cut=float(params.rc.max()), skin=SKIN, eps=params.eps, sigma=params.sig,
                 mass=params.mass, dt=DT, precision=PRECISIONS[precision], list_kind=LISTS[lst],
                 rcut=params.rc if params.nsp > 1 else None, **kw)
    s.set_state(np.ascontiguousarray(sysm.pos), np.ascontiguousarray(sysm.vel),
                np.ascontiguousarray(sysm.species))
    return s


def liquid(n_cells=14, seed=21):
    return W.lj_fcc(n_cells, seed=seed, jitter=0.05)


def gas(n=3000, box=(22.5, 25.0, 31.0), seed=5):
    box = np.array(box)
    pos = W.random_gas(n, box, seed=seed)
    return W.System(pos, np.zeros_like(pos), np.zeros(n, dtype=np.int32), box, "gas")


def threshold():
    box = np.array([30.0, 30.0, 30.0])
    pos = W.threshold_pairs(343, box, RC + SKIN, 1e-12, seed=9)
    return W.System(pos, np.zeros_like(pos), np.zeros(len(pos), dtype=np.int32), box, "threshold")


def slab():
    s = W.slab_nanoparticles(L=40.0, n_particles=4, r_min=3.0, r_max=5.0, seed=3)
    return s


# ---------------------------------------------------------------- binning
def test_binning_puts_every_atom_in_its_cell():
    sysm = liquid()
    s = make(sysm)
    s.bin_cells()
    cells = s.cells()
    pos, _, img = s.get_state()
    info = s.info()
    nc = np.array(info["ncell"])
    w = np.array(info["cell_width"])
    c3 = np.stack([cells % nc[0], (cells // nc[0]) % nc[1], cells // (nc[0] * nc[1])], axis=1)
    assert np.all(pos >= 0.0) and np.all(pos < sysm.box)
    assert np.all(c3 * w <= pos + 1e-12) and np.all(pos < (c3 + 1) * w + 1e-12)
    # wrapping is the only change: unwrapped positions are the inputs
    assert np.array_equal(pos + img * sysm.box, sysm.pos) or np.allclose(pos + img * sysm.box, sysm.pos, atol=1e-13)
    assert np.bincount(cells, minlength=int(nc.prod())).sum() == sysm.n


# ---------------------------------------------------------------- neighbour sets
@pytest.mark.parametrize("kind", ["liquid", "gas", "threshold", "slab"])
@pytest.mark.parametrize("lst", ["full", "half"])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_neighbour_set_bit_exact(kind, lst, precision):
    sysm = {"liquid": liquid, "gas": gas, "threshold": threshold, "slab": slab}[kind]()
    s = make(sysm, precision, lst)
    s.build_neighbors()
    got = s.neighbors()
    ref = O.neighbor_pairs(sysm.pos, sysm.box, RC + SKIN)
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)


def test_fcc_list_lengths():
    """Perfect fcc at rho*=0.8442: every atom has exactly 78 neighbours inside 2.8."""
    sysm = W.lj_fcc(14, seed=1)
    s = make(sysm, "mixed", "full")
    s.build_neighbors()
    info = s.info()
    assert info["list_entries"] == 78 * sysm.n and info["max_list"] == 78
    s2 = make(sysm, "mixed", "half")
    s2.build_neighbors()
    assert s2.info()["list_entries"] == 39 * sysm.n


# ---------------------------------------------------------------- forces
@pytest.mark.parametrize("lst", ["full", "half"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["liquid", "slab"])
def test_forces_vs_oracle(kind, lst, precision):
    sysm = liquid() if kind == "liquid" else slab()
    s = make(sysm, precision, lst)
    F = s.forces()
    Fref, _, _ = O.lj_forces(sysm.pos, sysm.box, O.LJParams.single())
    assert force_error(F, Fref) <= TOL[precision]


@pytest.mark.parametrize("lst", ["full", "half"])
def test_mixed_forces_bitwise_reproducible_and_order_independent(lst):
    """Fixed-point sums do not depend on summation order: repeated runs and any input
    ordering give bit-identical forces."""
    sysm = liquid()
    a = make(sysm, "mixed", lst).forces()
    b = make(sysm, "mixed", lst).forces()
    assert np.array_equal(a, b)
    perm = np.argsort(W.splitmix64(3, 3, sysm.n))
    sp = W.System(sysm.pos[perm], sysm.vel[perm], sysm.species[perm], sysm.box)
    d = make(sp, "mixed", lst).forces()
    assert np.array_equal(d, a[perm])


def test_mixed_full_and_half_lists_agree():
    sysm = liquid()
    a = make(sysm, "mixed", "full").forces()
    c = make(sysm, "mixed", "half").forces()
    assert force_error(c, a) <= 2 * TOL["mixed"]


def test_mixed_force_sum():
    """Half lists evaluate each pair once, so f_ji = -f_ij bit for bit and the fixed-point
    total is exactly zero.  Full lists evaluate a pair from both sides, in each block's own
    FP32 frame: the total is zero to FP32 rounding."""
    sysm = liquid()
    F = make(sysm, "mixed", "half").forces()
    q = np.rint(F * 2.0 ** 32).astype(np.int64)
    assert np.array_equal(q.astype(np.float64) * 2.0 ** -32, F)
    assert np.all(q.sum(axis=0) == 0)
    F = make(sysm, "mixed", "full").forces()
    frms = np.sqrt((F ** 2).sum(1).mean())
    assert np.abs(F.sum(axis=0)).max() <= 1e-5 * frms * np.sqrt(sysm.n)


def test_forces_translation_invariance_mixed():
    sysm = liquid()
    F = make(sysm, "mixed").forces()
    t = np.array([3.3, -7.1, 0.37])
    sh = W.System(W.wrap(sysm.pos + t, sysm.box), sysm.vel, sysm.species, sysm.box)
    F2 = make(sh, "mixed").forces()
    assert force_error(F2, F) <= 2 * TOL["mixed"]


def test_multispecies_per_pair_cutoff():
    """Kob-Andersen-type binary mixture: per-pair eps, sigma and r_cut = 2.5 sigma_ab."""
    a = W.lattice_constant(1.2)
    pos, box = W.fcc_lattice(16, 16, 16, a)
    pos = W.gaussian_jitter(pos, box, 0.03, seed=4)
    sp = W.species_shuffle(len(pos), 0.2, seed=4)
    sysm = W.System(pos, np.zeros_like(pos), sp, box)
    sig = np.array([[1.0, 0.8], [0.8, 0.88]])
    P = O.LJParams([[1.0, 1.5], [1.5, 0.5]], sig, 2.5 * sig, [1.0, 1.0])
    Fref, pe_ref, vir_ref = O.lj_forces(pos, box, P, species=sp)
    for precision in ("fp64", "mixed"):
        for lst in ("full", "half"):
            s = make(sysm, precision, lst, params=P)
            F = s.forces()
            assert force_error(F, Fref) <= TOL[precision], (precision, lst)
            pe, _, vir = s.energy_virial()
            tol = 1e-12 if precision == "fp64" else 1e-6
            assert abs(pe - pe_ref) <= tol * abs(pe_ref)
            assert np.abs(vir - vir_ref).max() <= tol * np.abs(vir_ref[:3]).max()


def test_dense_blocks_cooperative_tail():
    """At rho* = 1.5 a 2x2x2-cell block holds several hundred atoms, more than a force CTA
    has threads: the atoms past the first pass are shared out over the whole CTA.  Forces
    match the oracle, and a permuted input (which moves different atoms into that tail
    pass) gives bit-identical forces; energy and virial launches match too."""
    sysm = W.lj_fcc(12, rho=1.5, seed=4, jitter=0.03)
    s = make(sysm, "mixed", "full")
    F = s.forces()
    Fref, pe_ref, vir_ref = O.lj_forces(sysm.pos, sysm.box, O.LJParams.single())
    assert force_error(F, Fref) <= TOL["mixed"]
    perm = np.argsort(W.splitmix64(5, 3, sysm.n))
    sp = W.System(sysm.pos[perm], sysm.vel[perm], sysm.species[perm], sysm.box)
    assert np.array_equal(make(sp, "mixed", "full").forces(), F[perm])
    pe, _, vir = s.energy_virial()
    assert abs(pe - pe_ref) <= 1e-6 * abs(pe_ref)
    assert np.abs(vir - vir_ref).max() <= 1e-6 * np.abs(vir_ref[:3]).max()


def test_long_lists_match_oracle():
    """r_cut = 5 sigma: lists of ~530 entries (67 chunks) and a tile of the whole box (4
    cells per side); mixed forces and energy match the oracle."""
    sysm = W.lj_fcc(13, seed=6, jitter=0.05)
    P = O.LJParams.single(rc=5.0)
    s = make(sysm, "mixed", "full", params=P)
    Fref, pe_ref, _ = O.lj_forces(sysm.pos, sysm.box, P)
    assert force_error(s.forces(), Fref) <= TOL["mixed"]
    pe, _, _ = s.energy_virial()
    assert abs(pe - pe_ref) <= 1e-6 * abs(pe_ref)
    assert s.info()["max_list"] > 500


@pytest.mark.parametrize("lst", ["full", "half"])
def test_close_pairs_take_the_exact_wide_path(lst):
    """Pairs at 0.6 sigma carry forces far above 2048 eps/sigma, beyond the two-part
    fixed-point split: those atoms go through the exact FP64 path and still match the
    oracle, bit-identically for any input order."""
    sysm = liquid()
    pos = sysm.pos.copy()
    rng = np.random.default_rng(11)
    for i in rng.choice(sysm.n // 2, 12, replace=False):
        j = sysm.n - 1 - i
        u = rng.normal(size=3)
        pos[j] = W.wrap(pos[i] + 0.6 * u / np.linalg.norm(u), sysm.box)
    dense = W.System(pos, sysm.vel, sysm.species, sysm.box)
    F = make(dense, "mixed", lst).forces()
    Fref, _, _ = O.lj_forces(pos, sysm.box, O.LJParams.single())
    assert np.abs(F).max() > 1e4
    assert force_error(F, Fref) <= TOL["mixed"]
    perm = np.argsort(W.splitmix64(6, 3, sysm.n))
    sp = W.System(pos[perm], sysm.vel[perm], sysm.species[perm], sysm.box)
    assert np.array_equal(make(sp, "mixed", lst).forces(), F[perm])

@pytest.mark.parametrize("lst", ["full", "half"])
def test_very_close_pairs_exact_or_reported(lst):
    """Pair forces of 1.5e6 eps/sigma (atoms 0.45 sigma apart), three of them adding up to
    3.1e6 on one atom: beyond 2^20 eps/sigma, the range of 32-bit high-part sums, so the
    exact 64-bit path must carry them and match the oracle.  Atoms 0.40 sigma apart (7.1e6
    eps/sigma, beyond the 2^22 the 64-bit sums accept per term) are reported as
    MD_ERR_NONFINITE instead of a wrapped force."""
    sysm = liquid()
    rng = np.random.default_rng(21)
    pos = sysm.pos.copy()
    picks = rng.choice(sysm.n // 2, 16, replace=False)
    for c in range(4):  # each: an atom and three partners at 0.45 sigma, 60 degrees apart
        i, js = picks[4 * c], picks[4 * c + 1:4 * c + 4]
        for k, j in enumerate(js):
            a = (k - 1) * np.pi / 3
            pos[j] = W.wrap(pos[i] + 0.45 * np.array([np.cos(a), np.sin(a), 0.0]), sysm.box)
    dense = W.System(pos, sysm.vel, sysm.species, sysm.box)
    F = make(dense, "mixed", lst).forces()
    Fref, _, _ = O.lj_forces(pos, sysm.box, O.LJParams.single())
    assert np.abs(Fref).max() > 3.0e6
    assert force_error(F, Fref) <= TOL["mixed"]
    assert np.abs(F - Fref).max() <= 2e-5 * np.abs(Fref).max()
    pos2 = sysm.pos.copy()
    pos2[picks[1]] = W.wrap(pos2[picks[0]] + np.array([0.40, 0.0, 0.0]), sysm.box)
    s = make(W.System(pos2, sysm.vel, sysm.species, sysm.box), "mixed", lst)
    with pytest.raises(M.MDError) as e:
        s.forces()
    assert e.value.code == M.MD_ERR_NONFINITE


@pytest.mark.parametrize("lst", ["full", "half"])
def test_cutoff_decided_by_the_definition(lst):
    """Isolated pairs at r_cut (1 -/+ 1e-7): inside and outside by the FP64 definition, but
    closer to r_cut than FP32 distances resolve.  The unshifted force jumps by |f(r_cut)| there,
    so the mixed path must take the FP64 decision for them (and the energy with it)."""
    box = np.array([30.0, 30.0, 30.0])
    pos = W.threshold_pairs(216, box, RC, 1e-7, seed=13)
    sysm = W.System(pos, np.zeros_like(pos), np.zeros(len(pos), dtype=np.int32), box)
    P = O.LJParams.single()
    s = make(sysm, "mixed", lst)
    F = s.forces()
    Fref, pe_ref, _ = O.lj_forces(pos, box, P)
    assert np.abs(Fref).max() > 0.03  # half the pairs interact
    assert np.abs(F - Fref).max() <= 2e-5 * np.abs(Fref).max()
    pe, _, _ = s.energy_virial()
    assert abs(pe - pe_ref) <= 1e-6 * abs(pe_ref)

# ---------------------------------------------------------------- energies
@pytest.mark.parametrize("lst", ["full", "half"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_energy_virial_vs_oracle(lst, precision):
    sysm = liquid()
    s = make(sysm, precision, lst)
    pe, ke, vir = s.energy_virial()
    P = O.LJParams.single()
    _, pe_ref, vir_ref = O.lj_forces(sysm.pos, sysm.box, P)
    ke_ref = O.kinetic(sysm.vel, P)
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert abs(pe - pe_ref) <= tol * abs(pe_ref)
    assert abs(ke - ke_ref) <= 1e-12 * ke_ref
    assert np.abs(vir - vir_ref).max() <= tol * np.abs(vir_ref[:3]).max()


def test_fcc_lattice_energy_on_gpu():
    """Perfect fcc crystal: energy and virial per atom equal the oracle's (compensated, and
    pinned to the exact lattice sum); forces vanish by symmetry."""
    sysm = W.lj_fcc(14, seed=1)
    _, pe_ref, vir_ref = O.lj_forces(sysm.pos, sysm.box, O.LJParams.single())
    for precision in ("fp64", "mixed"):
        for lst in ("full", "half"):
            s = make(sysm, precision, lst)
            pe, _, vir = s.energy_virial()
            tol = 1e-12 if precision == "fp64" else 1e-6
            assert pe == pytest.approx(pe_ref, rel=tol)
            assert vir[:3].sum() == pytest.approx(vir_ref[:3].sum(), rel=tol)
            assert np.abs(s.forces()).max() < (1e-11 if precision == "fp64" else 1e-4)


# ---------------------------------------------------------------- trajectories
@pytest.mark.parametrize("lst", ["full", "half"])
def test_fp64_trajectory_config1(lst):
    """4,000-atom fcc at T*=0.72, 100 velocity-Verlet steps, skin/2 rebuilds: FP64 GPU vs oracle."""
    sysm = W.lj_fcc(10, seed=1)
    s = make(sysm, "fp64", lst)
    s.step(100)
    pos, vel, img = s.get_state()
    ref = O.run_nve(sysm.pos, sysm.vel, sysm.box, O.LJParams.single(), DT, SKIN, 100)
    assert np.abs(pos + img * sysm.box - (ref["pos"] + ref["image"] * sysm.box)).max() < 1e-10
    assert np.abs(vel - ref["vel"]).max() < 1e-9
    info = s.info()
    assert info["n_builds"] - 1 == ref["rebuilds"], info
    assert info["n_redos"] == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_and_direct_launch_give_identical_steps(precision, monkeypatch):
    """md_step through CUDA graphs with the rebuild decided on the device, and the same
    kernels launched from the host (MDGB_NO_GRAPHS=1), give bit-identical trajectories."""
    sysm = W.lj_fcc(10, seed=3)
    a = make(sysm, precision, "full")
    a.step(60)
    monkeypatch.setenv("MDGB_NO_GRAPHS", "1")
    b = make(sysm, precision, "full")
    b.step(60)
    pa, va, ia = a.get_state()
    pb, vb, ib = b.get_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb) and np.array_equal(ia, ib)
    assert a.info()["n_builds"] == b.info()["n_builds"]


@pytest.mark.parametrize("graphs", [True, False])
def test_fused_steps_equal_separate_kernels(graphs, monkeypatch):
    """On the full-list mixed path the force kernel also performs the velocity-Verlet
    updates (double-buffered FP32 coordinates).  Over several md_step calls of uneven
    length, with rebuilds, that gives bit-identical positions, velocities and forces to
    separate force and integration kernels (MDGB_NO_FUSE=1), in graph and direct mode."""
    if not graphs:
        monkeypatch.setenv("MDGB_NO_GRAPHS", "1")
    sysm = W.lj_fcc(12, seed=8)
    a = make(sysm, "mixed", "full")
    monkeypatch.setenv("MDGB_NO_FUSE", "1")
    b = make(sysm, "mixed", "full")
    for n in (1, 37, 2, 120):
        a.step(n)
        b.step(n)
    pa, va, ia = a.get_state()
    pb, vb, ib = b.get_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb) and np.array_equal(ia, ib)
    assert np.array_equal(a.forces(), b.forces())
    assert a.info()["n_builds"] == b.info()["n_builds"] > 2
    ea, eb = a.energy_virial(), b.energy_virial()
    assert ea[0] == eb[0] and ea[1] == eb[1] and np.array_equal(ea[2], eb[2])

def test_mixed_trajectory_short():
    sysm = W.lj_fcc(10, seed=1)
    s = make(sysm, "mixed", "full")
    s.step(20)
    pos, vel, img = s.get_state()
    ref = O.run_nve(sysm.pos, sysm.vel, sysm.box, O.LJParams.single(), DT, SKIN, 20)
    assert np.abs(pos + img * sysm.box - (ref["pos"] + ref["image"] * sysm.box)).max() < 1e-6


def test_rebuild_every_k_policy_matches_oracle():
    sysm = W.lj_fcc(10, seed=2)
    s = make(sysm, "fp64", "full", rebuild=M.MD_REBUILD_EVERY_K, rebuild_k=5)
    s.step(30)
    pos, vel, img = s.get_state()
    ref = O.run_nve(sysm.pos, sysm.vel, sysm.box, O.LJParams.single(), DT, SKIN, 30, policy=1, every_k=5)
    assert s.info()["n_builds"] - 1 == ref["rebuilds"] == 6
    assert np.abs(pos + img * sysm.box - (ref["pos"] + ref["image"] * sysm.box)).max() < 1e-10


def test_energy_conservation_mixed():
    sysm = W.lj_fcc(10, seed=1)
    s = make(sysm, "mixed")
    pe0, ke0, _ = s.energy_virial()
    s.step(100)
    pe1, ke1, _ = s.energy_virial()
    ref = O.run_nve(sysm.pos, sysm.vel, sysm.box, O.LJParams.single(), DT, SKIN, 100, history=True)
    e_ref = (ref["pe"][-1] + ref["ke"][-1]) / sysm.n
    assert abs((pe1 + ke1) / sysm.n - e_ref) < 1e-4


# ---------------------------------------------------------------- device pointers and edge cases
def test_device_pointer_path_matches_host_path():
    sysm = liquid(10)
    dev = torch.device("cuda")
    s = M.System(sysm.n, sysm.box, stream=torch.cuda.current_stream().cuda_stream)
    s.set_state(torch.from_numpy(sysm.pos).to(dev), torch.from_numpy(sysm.vel).to(dev),
                torch.from_numpy(sysm.species).to(dev))
    Fd = torch.empty((sysm.n, 3), dtype=torch.float64, device=dev)
    s.forces(Fd)
    torch.cuda.synchronize()
    Fh = make(sysm, "mixed").forces()
    assert np.array_equal(Fd.cpu().numpy(), Fh)


def test_edge_cases():
    box = np.array([12.0, 12.0, 12.0])
    # one atom: no neighbours, zero force
    s = M.System(1, box)
    s.set_state(np.array([[1.0, 2.0, 3.0]]), np.zeros((1, 3)))
    assert np.all(s.forces() == 0.0)
    assert len(s.neighbors()) == 0
    s.step(3)
    # two atoms beyond the list radius
    s2 = M.System(2, box, precision=M.MD_FP64)
    s2.set_state(np.array([[1.0, 1.0, 1.0], [7.0, 7.0, 7.0]]), np.zeros((2, 3)))
    assert np.all(s2.forces() == 0.0)
    # empty system
    s0 = M.System(0, box)
    s0.set_state(np.zeros((0, 3)), np.zeros((0, 3)))
    s0.step(2)
    assert s0.energy_virial()[0] == 0.0
    # errors surface as codes
    s3 = M.System(4, box)
    with pytest.raises(M.MDError) as e:
        s3.forces()
    assert e.value.code == M.MD_ERR_STATE
    with pytest.raises(M.MDError) as e:
        s3.set_state(np.ones((4, 3)), np.zeros((4, 3)), np.array([0, 1, 0, 0], dtype=np.int32))
    assert e.value.code == M.MD_ERR_ARG
    # a dense clump in a mostly empty box overflows the capacities sized from the mean
    # density; the library regrows them and still matches the oracle
    clump, _ = W.fcc_lattice(5, 5, 4, 0.5)
    clump = W.gaussian_jitter(clump + 4.0, box, 0.01, seed=7)
    s4 = M.System(len(clump), box, sigma=0.3, r_cut=0.75, skin=0.3)
    s4.set_state(np.ascontiguousarray(clump), np.zeros_like(clump))
    P = O.LJParams.single(sig=0.3, rc=0.75)
    assert force_error(s4.forces(), O.lj_forces(clump, box, P)[0]) <= 2e-5
    assert s4.info()["max_list"] > 24


# ---------------------------------------------------------------- full size (2,048,000 atoms)
@pytest.mark.parametrize("lst", ["full", "half"])
def test_full_size_config2_sampled(lst):
    """80^3 fcc cells at rho*=0.8442 with liquid-like jitter, the benchmark's launch
    configuration: pair count equals the oracle's, sampled forces match.  The r_list fit
    gives 44 cells per side; the homogeneous full-list system takes 42 at its first build
    (blocks of ~221 atoms for the 256-thread CTAs), the half list keeps the 44 its colour
    classes need."""
    sysm = W.lj_fcc(80, seed=2, jitter=0.05)
    s = make(sysm, "mixed", lst)
    F = s.forces()
    info = s.info()
    assert info["ncell"] == ([42, 42, 42] if lst == "full" else [44, 44, 44])
    n_pairs_ref = O._load().orc_neighbor_pairs(sysm.n, np.ascontiguousarray(sysm.pos).ravel(), sysm.box,
                                               RC + SKIN, 0, 0, None)
    expect = n_pairs_ref if lst == "half" else 2 * n_pairs_ref
    assert info["list_entries"] == expect
    idx = np.sort(W.splitmix64(11, 0, 256) % np.uint64(sysm.n)).astype(np.int64)
    Fs, _, _ = O.lj_forces_subset(sysm.pos, sysm.box, O.LJParams.single(), idx)
    mag = np.sqrt((Fs ** 2).sum(1))
    frms = np.sqrt((F ** 2).sum(1).mean())
    e = np.sqrt(((F[idx] - Fs) ** 2).sum(1)) / np.maximum(mag, frms)
    assert e.max() <= TOL["mixed"]
    if lst == "half":
        q = np.rint(F * 2.0 ** 32).astype(np.int64)
        assert np.all(q.sum(axis=0) == 0)


def test_full_size_fused_steps_sampled():
    """The benchmark's launch configuration itself: 100 graph-launched fused steps of the
    2,048,000-atom liquid from the fcc start (lists rebuilt inside the graphs).  At the end,
    sampled forces at the GPU's positions match the oracle's, and the total momentum per atom
    stays below 1e-6 (full lists evaluate each pair twice in different FP32 frames, so
    momentum is conserved only to FP32 rounding; thermal momentum per atom is ~0.85).  The
    energy is not a check here: the potential is unshifted and the lattice melts, so pairs
    crossing r_cut move it."""
    sysm = W.lj_fcc(80, seed=2)
    s = make(sysm, "mixed", "full")
    s.step(100)
    assert s.info()["n_builds"] >= 3
    pos, vel, _ = s.get_state()
    n = sysm.n
    assert np.abs(vel.sum(0)).max() / n < 1e-6
    F = s.forces()
    idx = np.sort(W.splitmix64(12, 0, 256) % np.uint64(n)).astype(np.int64)
    Fs, _, _ = O.lj_forces_subset(pos, sysm.box, O.LJParams.single(), idx)
    mag = np.sqrt((Fs ** 2).sum(1))
    frms = np.sqrt((F ** 2).sum(1).mean())
    assert (np.sqrt(((F[idx] - Fs) ** 2).sum(1)) / np.maximum(mag, frms)).max() <= TOL["mixed"]


# ---------------------------------------------------------------- race detection, faults, checkpoints
@pytest.mark.parametrize("n_cells", [10, 20])
def test_colour_schedule_race_detector(n_cells):
    """On the GPU, with the kernels' own block and tile mapping: no atom is claimed by two
    blocks of one colour phase (the non-overlap rule of Sec. II.A for each of the 8 waves),
    while one phase holding every block shows the overlaps the colours avoid."""
    sysm = liquid(n_cells)
    s = make(sysm, "mixed", "half")
    s.forces()
    assert s.colour_conflicts(8) == 0
    assert s.colour_conflicts(1) > 0
    with pytest.raises(M.MDError):
        s.colour_conflicts(3)


def test_nonfinite_state_is_refused():
    sysm = liquid(8)
    s = make(sysm)
    bad = sysm.pos.copy()
    bad[17, 1] = np.nan
    with pytest.raises(M.MDError) as ei:
        s.set_state(bad, sysm.vel, sysm.species)
    assert ei.value.code == M.MD_ERR_NONFINITE
    vel = sysm.vel.copy()
    vel[3, 0] = np.inf
    with pytest.raises(M.MDError):
        s.set_state(sysm.pos, vel, sysm.species)
    s.set_state(sysm.pos, sysm.vel, sysm.species)  # a valid state loads again
    assert force_error(s.forces(), O.lj_forces(sysm.pos, sysm.box, O.LJParams.single())[0]) <= TOL["mixed"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_resume_is_bitwise(precision):
    """Save the state after 50 steps (md_get_state), restore it into a new system
    (md_set_state) and run 50 more: bit-identical to the run that continued, when that run
    rebuilds its lists at the save point as the restored one does."""
    sysm = liquid(10)
    a = make(sysm, precision)
    a.step(50)
    pos, vel, img = a.get_state()
    a.build_neighbors()
    a.step(50)
    b = make(W.System(pos, vel, sysm.species, sysm.box), precision)
    b.step(50)
    pa, va, ia = a.get_state()
    pb, vb, ib = b.get_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    assert np.array_equal(ia, ib + img)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("lst", ["full", "half"])
def test_nonfinite_force_is_reported(precision, lst):
    """Two atoms on one spot (a pair at r = 0, an infinite force): the force kernels raise
    the sticky non-finite flag, so md_forces and md_step return MD_ERR_NONFINITE."""
    sysm = liquid(8)
    pos = sysm.pos.copy()
    pos[5] = pos[4]
    bad = W.System(pos, sysm.vel, sysm.species, sysm.box)
    s = make(bad, precision, lst)
    with pytest.raises(M.MDError) as ei:
        s.forces()
    assert ei.value.code == M.MD_ERR_NONFINITE
    s2 = make(bad, precision, lst)
    with pytest.raises(M.MDError) as ei:
        s2.step(2)
    assert ei.value.code == M.MD_ERR_NONFINITE


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_skin_violation_is_reported(precision):
    """Fixed-interval rebuilds (the paper's every-k protocol) with an interval far too long:
    once an atom has moved more than skin/2 since the last build, md_step reports
    MD_ERR_SKIN_VIOLATION instead of running on with incomplete lists."""
    sysm = W.lj_fcc(10, seed=2)
    s = make(sysm, precision, "full", rebuild=M.MD_REBUILD_EVERY_K, rebuild_k=100000)
    with pytest.raises(M.MDError) as ei:
        s.step(300)
    assert ei.value.code == M.MD_ERR_SKIN_VIOLATION


def test_redo_after_tile_growth_in_a_long_chunk(monkeypatch):
    """The strongly inhomogeneous workload (fcc slab plus 40 particles in vacuum, 1,192,114
    atoms, T* = 0.3) in one 500-step call on the r_list fit grid (MDGB_FIT_GRID=1; the
    coarser grid its first build would pick starts with tiles large enough that this run
    needs no redo): the cold slab contracts, so a rebuild inside a chunk of graph-launched
    steps outgrows the captured tile capacity and the chunk is redone from its snapshot
    with grown capacities.  The redo must converge (the grown capacity is kept through the
    rebuild of the restored state), and sampled forces at the end match the oracle."""
    sysm = W.slab_nanoparticles(152.0, rho=0.8442, T=0.3, seed=3)
    monkeypatch.setenv("MDGB_FIT_GRID", "1")
    s = make(sysm)
    s.step(100)
    s.step(500)
    assert s.info()["n_redos"] >= 1
    pos, _, _ = s.get_state()
    F = s.forces()
    idx = np.sort(W.splitmix64(13, 0, 256) % np.uint64(sysm.n)).astype(np.int64)
    Fs, _, _ = O.lj_forces_subset(pos, sysm.box, O.LJParams.single(), idx)
    mag = np.sqrt((Fs ** 2).sum(1))
    frms = np.sqrt((F ** 2).sum(1).mean())
    assert (np.sqrt(((F[idx] - Fs) ** 2).sum(1)) / np.maximum(mag, frms)).max() <= TOL["mixed"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_time_reversibility(precision):
    """Velocity Verlet is time-reversible: 50 steps forward, velocities negated, 50 steps back
    return the atoms to their start.  On the FP64 path only the rounding of the updates is
    left (bound 1e-8 sigma).  On the mixed path a force also carries the FP32 rounding of the
    frame of the atoms' cells at the last rebuild, and the way back rebuilds at other steps,
    so the bound is set by the mixed force error (about 1e-6 of F) over 100 steps: 1e-5 sigma."""
    sysm = liquid(10)
    s = make(sysm, precision)
    x0, s_vel0, i0 = s.get_state()
    s.step(50)
    pos, vel, img = s.get_state()
    s.set_state(pos, -vel, sysm.species)
    s.step(50)
    x1, v1, i1 = s.get_state()
    # set_state starts the image counters again from zero
    d = np.abs((x1 + (i1 + img) * sysm.box) - (x0 + i0 * sysm.box)).max()
    tol = 1e-8 if precision == "fp64" else 1e-5
    assert d < tol, d
    assert np.abs(v1 + s_vel0).max() < (1e-8 if precision == "fp64" else 1e-3)


@pytest.mark.parametrize("seed", range(6))
def test_randomised_small_systems(seed):
    """Seeded random shapes: a gas of 2..800 atoms in a box with sides drawn from 11.3..17
    sigma (neighbour set bit for bit against the oracle, both list kinds), and a jittered fcc
    crystal of 1,500..4,000 atoms at a density drawn from 0.7..0.95 with random vacancies,
    whose ragged cells the forces must handle (both precisions and list kinds).  Boxes this
    small have 4 cells per side, so every tile holds the whole system; 4,000 atoms keep the
    FP64 half-list tile (52 B per atom) within shared memory."""
    rng = np.random.default_rng(1000 + seed)
    box = rng.uniform(11.3, 17.0, 3)
    n = int(rng.integers(2, 800))
    pos = W.random_gas(n, box, seed=200 + seed)
    for lst in (M.MD_LIST_FULL, M.MD_LIST_HALF_COLOUR8):
        s = M.System(n, box, list_kind=lst)
        s.set_state(pos, np.zeros_like(pos))
        assert np.array_equal(s.neighbors(), O.neighbor_pairs(pos, box, RC + SKIN))
        s.close()
    sysm = W.fcc_vacancies(int(rng.integers(1500, 4000)), float(rng.uniform(0.7, 0.95)), 1.0, seed=300 + seed)
    Fref = O.lj_forces(sysm.pos, sysm.box, O.LJParams.single())[0]
    for precision in ("fp64", "mixed"):
        for lst in ("full", "half"):
            s = make(sysm, precision, lst)
            assert force_error(s.forces(), Fref) <= TOL[precision], (precision, lst)
            s.close()


def test_compact_grids_bit_identical():
    """A mostly empty system (a slab and nanoparticles in vacuum) runs the force kernel and
    the list builder over its occupied blocks only: forces and a 30-step trajectory are
    bit-identical to one CTA per block (integer force sums), and match the oracle."""
    import os
    sysm = slab()
    os.environ["MDGB_NO_COMPACT"] = "1"
    try:
        a = make(sysm)
    finally:
        del os.environ["MDGB_NO_COMPACT"]
    b = make(sysm)
    assert np.array_equal(a.forces(), b.forces())
    a.step(30)
    b.step(30)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    Fref, _, _ = O.lj_forces(*b.get_state()[:1], sysm.box, O.LJParams.single())
    assert force_error(b.forces(), Fref) <= TOL["mixed"]


def test_homogeneous_system_takes_coarser_cells(monkeypatch):
    """A homogeneous liquid on the mixed full-list path takes cells coarser than the r_list
    fit at its first build: 42^3 fcc cells (296,352 atoms, box 70.5 sigma) fit 24 cells per
    side and take 22, so a block holds ~220 atoms.  Pair set bit-exact, forces against the
    oracle, and a 20-step trajectory within 2e-5 sigma of the fit grid's (MDGB_FIT_GRID=1),
    which differs only in the FP32 frames of its cells; FP64 and half lists keep the fit
    grid."""
    sysm = W.lj_fcc(42, seed=6, jitter=0.05)
    s = make(sysm)
    F = s.forces()
    assert s.info()["ncell"] == [22, 22, 22]
    assert np.array_equal(s.neighbors(), O.neighbor_pairs(sysm.pos, sysm.box, RC + SKIN))
    Fref = O.lj_forces(sysm.pos, sysm.box, O.LJParams.single())[0]
    assert force_error(F, Fref) <= TOL["mixed"]
    monkeypatch.setenv("MDGB_FIT_GRID", "1")
    f = make(sysm)
    monkeypatch.delenv("MDGB_FIT_GRID")
    f.forces()
    assert f.info()["ncell"] == [24, 24, 24]
    s.step(20)
    f.step(20)
    (pa, va, ia), (pb, vb, ib) = s.get_state(), f.get_state()
    # the two runs differ only in the FP32 frames of their cells: forces by ~1e-6 of F per
    # step, which 20 steps of the jittered lattice carry to a few 1e-6 sigma over 296,352 atoms
    assert np.abs(pa + ia * sysm.box - (pb + ib * sysm.box)).max() < 2e-5
    for precision, lst in (("fp64", "full"), ("mixed", "half")):
        t = make(sysm, precision, lst)
        t.forces()
        assert t.info()["ncell"] == [24, 24, 24], (precision, lst)


def test_inhomogeneous_system_takes_coarser_cells(monkeypatch):
    """An fcc slab with 10 nanoparticles in vacuum (190,154 atoms, box 90.7 sigma, most
    blocks empty) on the mixed full-list path: the fit grid has 32 cells per side, and the
    first build takes 30 from the density its atoms see (200 atoms per block), running the
    compact kernels over the occupied blocks of a linearly numbered grid.  Pair set
    bit-exact, forces against the oracle, and a 20-step trajectory within 2e-5 sigma of the
    fit grid's (MDGB_FIT_GRID=1)."""
    sysm = W.slab_nanoparticles(L=91.0, n_particles=10, r_min=3.0, r_max=6.0, seed=5)
    s = make(sysm)
    F = s.forces()
    assert s.info()["ncell"] == [30, 30, 30]
    assert np.array_equal(s.neighbors(), O.neighbor_pairs(sysm.pos, sysm.box, RC + SKIN))
    Fref = O.lj_forces(sysm.pos, sysm.box, O.LJParams.single())[0]
    assert force_error(F, Fref) <= TOL["mixed"]
    monkeypatch.setenv("MDGB_FIT_GRID", "1")
    f = make(sysm)
    monkeypatch.delenv("MDGB_FIT_GRID")
    f.forces()
    assert f.info()["ncell"] == [32, 32, 32]
    s.step(20)
    f.step(20)
    (pa, _, ia), (pb, _, ib) = s.get_state(), f.get_state()
    assert np.abs(pa + ia * sysm.box - (pb + ib * sysm.box)).max() < 2e-5


def test_coarser_cells_per_side_in_a_non_cubic_mixture():
    """Sec. II.A, cells at least r_list wide, on a non-cubic box: a binary mixture with
    per-pair cutoffs (r_c = 2.5 sigma_ab) on 41 x 34 x 24 fcc cells at rho* = 0.8442
    (133,824 atoms, box 68.9 x 57.1 x 40.3 sigma).  The r_list fit gives 24 x 20 x 12 cells;
    the homogeneous rule's width (224 / (8 rho))^(1/3) = 3.213 sigma asks for 22 x 18 x 14,
    capped at the fit: 22 x 18 x 12, two sides that are not multiples of 4 (linear block
    numbering).  Pair set bit-exact, forces, energy and virial against the oracle, a
    20-step trajectory against the oracle's velocity Verlet; a second md_set_state keeps
    the grid and its forces match the oracle again."""
    a = W.lattice_constant(0.8442)
    lat, box = W.fcc_lattice(41, 34, 24, a)
    sig = np.array([[1.0, 0.8], [0.8, 0.88]])
    P = O.LJParams([[1.0, 1.5], [1.5, 0.5]], sig, 2.5 * sig, [1.0, 1.0])

    def config(seed):
        pos = W.gaussian_jitter(lat, box, 0.05, seed=seed)
        sp = W.species_shuffle(len(pos), 0.2, seed=seed)
        vel = W.thermal_velocities(np.ones(len(pos)), 0.72, seed)
        return W.System(pos, vel, sp, box)

    sysm = config(12)
    s = make(sysm, params=P)
    F = s.forces()
    assert s.info()["ncell"] == [22, 18, 12]
    assert np.array_equal(s.neighbors(), O.neighbor_pairs(sysm.pos, box, RC + SKIN))
    Fref, pe_ref, vir_ref = O.lj_forces(sysm.pos, box, P, species=sysm.species)
    assert force_error(F, Fref) <= TOL["mixed"]
    pe, _, vir = s.energy_virial()
    assert abs(pe - pe_ref) <= 1e-6 * abs(pe_ref)
    assert np.abs(vir - vir_ref).max() <= 1e-6 * np.abs(vir_ref[:3]).max()
    s.step(20)
    pos, _, img = s.get_state()
    ref = O.run_nve(sysm.pos, sysm.vel, box, P, DT, SKIN, 20, species=sysm.species)
    d = np.abs(pos + img * box - (ref["pos"] + ref["image"] * box)).max(axis=1)
    # FP32 pair forces keep nearly every atom within 1e-6 sigma of the FP64 run.  The
    # potential is cut unshifted at r_c (Sec. I: no interaction beyond r_c), so its force
    # steps there, by up to 24 * 1.5 / 2.0 * |2 * 0.4^12 - 0.4^6| = 0.073 eps/sigma (the AB
    # pair).  A pair within the runs' ~1e-8 sigma difference of r_c (about two such
    # crossings in 20 steps of 133,824 atoms) is cut in one run a step before the other:
    # its atoms' velocities then differ by 0.073 dt and their positions by at most
    # 0.073 dt * 20 dt = 3.7e-5 sigma at the end, and their neighbours by less.  Two runs of
    # the oracle itself from positions 1e-9 sigma apart show the same: 2.7e-5 sigma at two
    # atoms, 3.7e-9 sigma at the 99.9th percentile.
    assert np.quantile(d, 0.999) < 1e-6
    assert d.max() < 2 * 0.0732 * DT * 20 * DT
    other = config(13)
    s.set_state(other.pos, other.vel, other.species)
    F = s.forces()
    assert s.info()["ncell"] == [22, 18, 12]
    assert force_error(F, O.lj_forces(other.pos, box, P, species=other.species)[0]) <= TOL["mixed"]


def test_timing_brackets_one_force_launch_per_step_graph():
    """md_set_timing on the fused path: in the 8-step graphs only the first step's force
    kernel is bracketed by events, every singly launched step is too, and
    timed_force_evals counts exactly the bracketed launches (100 steps: 12 graphs of 8 and
    4 single steps, 16 timed), so force_ms / timed_force_evals is a mean launch time."""
    sysm = liquid(14)
    s = make(sysm)
    s.forces()
    s.set_timing(True)
    i0 = s.info()
    s.step(100)
    i1 = s.info()
    s.set_timing(False)
    assert i1["force_evals"] - i0["force_evals"] == 100
    timed = i1["timed_force_evals"] - i0["timed_force_evals"]
    assert 0 < timed < 100
    assert i1["force_ms"] > 0.0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_small_box_full_list_even_cell_count(precision):
    """Sec. II.A: full lists need no colour classes and take 6 cells per side where 6 fit and
    a multiple of 4 would leave 4.  A 9,400-atom liquid at rho* = 0.8442 (box 22.28 sigma, 7.96 r_list) gets 6 cells and 3
    linearly numbered blocks per side, so each tile is 4 of the 6 cells per side rather than
    the whole box (a whole-box FP64 tile of 9,400 atoms would not fit on chip).  Pair set,
    forces, energy, virial and a 20-step trajectory against the oracle."""
    sysm = W.fcc_vacancies(9400, 0.8442, 0.72, seed=8)
    s = make(sysm, precision, "full")
    F = s.forces()
    assert s.info()["ncell"] == [6, 6, 6]
    assert np.array_equal(s.neighbors(), O.neighbor_pairs(sysm.pos, sysm.box, RC + SKIN))
    P = O.LJParams.single()
    Fref, pe_ref, vir_ref = O.lj_forces(sysm.pos, sysm.box, P)
    assert force_error(F, Fref) <= TOL[precision]
    pe, _, vir = s.energy_virial()
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert abs(pe - pe_ref) <= tol * abs(pe_ref)
    assert np.abs(vir - vir_ref).max() <= tol * np.abs(vir_ref[:3]).max()
    s.step(20)
    pos, _, img = s.get_state()
    ref = O.run_nve(sysm.pos, sysm.vel, sysm.box, P, DT, SKIN, 20)
    dx = np.abs(pos + img * sysm.box - (ref["pos"] + ref["image"] * sysm.box)).max()
    assert dx < (1e-10 if precision == "fp64" else 1e-6)
    # 3 blocks per side cannot be split into the 8 parity classes of Sec. II.A: the race
    # detector refuses 8 phases on this grid, while one phase of all 27 blocks still shows
    # the overlap of neighbouring tiles.
    with pytest.raises(M.MDError) as ei:
        s.colour_conflicts(8)
    assert ei.value.code == M.MD_ERR_ARG
    assert s.colour_conflicts(1) > 0


def test_whole_system_tile_limit_is_reported():
    """With 4 cells per side every tile is the whole system.  A system whose tile does not
    fit the kernel's shared memory (here the FP64 half-list kernel, 52 B per atom, at 6,000
    atoms) is refused with MD_ERR_CELL_OVERFLOW, while the full-list kernels take it."""
    sysm = W.fcc_vacancies(6000, 0.8, 1.0, seed=5)
    s = make(sysm, "fp64", "half")
    with pytest.raises(M.MDError) as ei:
        s.forces()
    assert ei.value.code == M.MD_ERR_CELL_OVERFLOW
    Fref = O.lj_forces(sysm.pos, sysm.box, O.LJParams.single())[0]
    for precision in ("fp64", "mixed"):
        assert force_error(make(sysm, precision, "full").forces(), Fref) <= TOL[precision]
