"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test pins one part of what the hot path computes (Sec. I cutoff problem,
Sec. II.A linked cells and neighbour lists, Sec. II.D.3 each pair once) or
of the textbook physics around it (Lennard-Jones pair, virial, velocity
Verlet), chosen so that a plausible slip in the oracle - a dropped term, a
wrong sign, factor or index, a '<=' for '<', a missing periodic image -
fails at least one of them:

  * LJ dimer: the minimum sits at 2^(1/6) sigma with depth -eps (a property
    of the potential, checked by locating the minimum numerically);
  * force = -grad(E) by central finite differences of the oracle's energy;
  * virial W_ab = -dE/d(strain_ab) by finite differences (all 6 components);
  * perfect fcc crystal: exact neighbour counts 54 / 78 from the lattice's
    shell structure, zero force by symmetry, lattice sums from an independent
    enumeration of lattice vectors;
  * neighbour sets: brute force == linked cells bit for bit, pairs placed at
    r_list (1 -/+ 1e-12) fall on the right side, a pair at exactly r_list is
    excluded (strict '<');
  * sum of forces = 0, translation and permutation invariance;
  * velocity Verlet is second order and time reversible; the skin/2 rebuild
    rule fires at the step the kinematics dictate;
  * the direct per-atom summation agrees with the cell-list whole-system path;
  * force-matching gradients: central finite differences of the oracle's forces
    with respect to every species-pair parameter and to positions, a dimer's
    closed-form derivatives, and exact scaling identities (L is linear in eps;
    forces are homogeneous of degree -1 in all lengths; sigma dE/dsigma summed
    is the virial trace).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1305_4196_gb300 import workloads as W


def _dimer(r, eps=0.7, sig=1.3, rc=4.0, direction=(0.3, -0.5, 0.81)):
    u = np.asarray(direction, dtype=np.float64)
    u /= np.linalg.norm(u)
    box = np.array([40.0, 40.0, 40.0])
    c = box / 2
    pos = np.stack([c - 0.5 * r * u, c + 0.5 * r * u])
    P = O.LJParams.single(eps=eps, sig=sig, rc=rc)
    return pos, box, P, u


def test_dimer_minimum_location_and_depth():
    """Minimum of the pair energy at 2^(1/6) sigma, depth -eps, zero force there."""
    eps, sig = 0.7, 1.3
    rs = np.linspace(1.0, 2.2, 2401)
    es = np.array([O.lj_forces(*_dimer(r, eps, sig)[:3])[1] for r in rs])
    k = int(np.argmin(es))
    # refine by golden-section search on the oracle energy
    lo, hi = rs[max(k - 1, 0)], rs[min(k + 1, len(rs) - 1)]
    g = (math.sqrt(5) - 1) / 2
    for _ in range(80):
        a = hi - g * (hi - lo)
        b = lo + g * (hi - lo)
        if O.lj_forces(*_dimer(a, eps, sig)[:3])[1] < O.lj_forces(*_dimer(b, eps, sig)[:3])[1]:
            hi = b
        else:
            lo = a
    rmin = 0.5 * (lo + hi)
    assert rmin == pytest.approx(2.0 ** (1.0 / 6.0) * sig, rel=1e-7)
    pos, box, P, _ = _dimer(2.0 ** (1.0 / 6.0) * sig, eps, sig)
    f, pe, _ = O.lj_forces(pos, box, P)
    assert pe == pytest.approx(-eps, rel=1e-13)
    assert np.abs(f).max() < 1e-12


def test_dimer_force_is_repulsive_inside_attractive_outside():
    eps, sig = 1.0, 1.0
    for r, sign in [(1.0, +1), (1.5, -1)]:
        pos, box, P, u = _dimer(r, eps, sig)
        f, _, _ = O.lj_forces(pos, box, P)
        # atom 1 sits at +u from atom 0: repulsion pushes it further along +u
        assert np.sign(np.dot(f[1], u)) == sign
        assert np.allclose(f[0], -f[1], rtol=0, atol=1e-14)


def test_cutoff_is_strict_and_unshifted():
    """No interaction at r >= r_cut; just inside, the full unshifted energy."""
    rc = 2.5
    pos, box, P, _ = _dimer(rc, 1.0, 1.0, rc=rc, direction=(1.0, 0.0, 0.0))
    f, pe, _ = O.lj_forces(pos, box, P)
    assert pe == 0.0 and np.all(f == 0.0)
    pos, box, P, _ = _dimer(rc * (1 - 1e-12), 1.0, 1.0, rc=rc, direction=(1.0, 0.0, 0.0))
    _, pe_in, _ = O.lj_forces(pos, box, P)
    # continuity of the (unshifted) pair energy: just inside r_c equals the limit from a
    # fine sampling of the oracle's own energy curve, which is smooth below r_c
    e = [O.lj_forces(*_dimer(rc * (1 - k * 1e-3), 1.0, 1.0, rc=rc, direction=(1.0, 0.0, 0.0))[:3])[1]
         for k in (1, 2, 3)]
    extrap = 3.0 * e[0] - 3.0 * e[1] + e[2]  # quadratic extrapolation to r_c
    assert pe_in < 0.0
    assert pe_in == pytest.approx(extrap, rel=1e-6)


def _small_liquid(n_cells=4, seed=11, jitter=0.05):
    return W.lj_fcc(n_cells, seed=seed, jitter=jitter)


def _safe_from_cutoff(pos, box, rc, margin):
    """True if no pair distance lies within margin of rc (so finite differences are smooth)."""
    pr = O.neighbor_pairs(pos, box, rc + margin)
    d = pos[pr[:, 0]] - pos[pr[:, 1]]
    d -= box * np.rint(d / box)
    r = np.sqrt((d * d).sum(1))
    return not np.any(np.abs(r - rc) < margin)


def test_force_is_minus_gradient_of_energy():
    P = O.LJParams.single(eps=1.2, sig=0.95, rc=2.5)
    for seed in range(11, 40):
        s = _small_liquid(seed=seed)
        if _safe_from_cutoff(s.pos, s.box, 2.5, 1e-4):
            break
    else:
        pytest.skip("no seed without a pair near the cutoff")
    f, _, _ = O.lj_forces(s.pos, s.box, P)
    h = 1e-6
    rng_atoms = [0, 5, 17, 101, 200]
    for i in rng_atoms:
        for k in range(3):
            xp = s.pos.copy()
            xm = s.pos.copy()
            xp[i, k] += h
            xm[i, k] -= h
            ep = O.lj_forces(xp, s.box, P)[1]
            em = O.lj_forces(xm, s.box, P)[1]
            fd = -(ep - em) / (2 * h)
            assert fd == pytest.approx(f[i, k], rel=2e-6, abs=2e-6 * (1 + abs(f[i, k])))


def test_virial_is_minus_strain_derivative_of_energy_cluster():
    """All six W_ab on an isolated cluster (no periodic images involved)."""
    rng_pos = W.fcc_lattice(2, 2, 2, 1.55)[0]
    box = np.array([1000.0, 1000.0, 1000.0])
    # near the origin (small coordinates keep the strained positions exact to ~1e-16)
    pos = rng_pos + 1.0 + 0.05 * W.normal(5, 2, rng_pos.size).reshape(rng_pos.shape)
    P = O.LJParams.single(eps=1.0, sig=1.0, rc=50.0)  # every pair interacts; smooth
    _, _, vir = O.lj_forces(pos, box, P)
    c = pos.mean(axis=0)
    comps = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    h = 1e-6
    for k, (a, b) in enumerate(comps):
        def energy(eta):
            e = np.eye(3)
            e[a, b] += eta
            return O.lj_forces(c + (pos - c) @ e.T, box, P)[1]
        dE = (energy(h) - energy(-h)) / (2 * h)
        assert -dE == pytest.approx(vir[k], rel=1e-6, abs=1e-6)


def test_virial_diagonal_is_minus_box_strain_derivative_periodic():
    P = O.LJParams.single()
    for seed in range(11, 40):
        s = _small_liquid(seed=seed)
        if _safe_from_cutoff(s.pos, s.box, 2.5, 1e-4):
            break
    _, _, vir = O.lj_forces(s.pos, s.box, P)
    h = 1e-7
    for a in range(3):
        def energy(eta):
            sc = np.ones(3)
            sc[a] += eta
            return O.lj_forces(s.pos * sc, s.box * sc, P)[1]
        dE = (energy(h) - energy(-h)) / (2 * h)
        assert -dE == pytest.approx(vir[a], rel=1e-6)


def _fcc_shell_sums(a, rmax):
    """Per-atom neighbour count, energy and virial trace of a perfect fcc crystal,
    by enumerating lattice vectors (integer combinations of the primitive
    vectors a/2 (0,1,1), (1,0,1), (1,1,0)) - independent of the oracle's
    cell list and minimum image."""
    m = int(math.ceil(2 * rmax / a)) + 2
    r = np.arange(-m, m + 1)
    n1, n2, n3 = np.meshgrid(r, r, r, indexing="ij")
    prim = 0.5 * a * np.array([[0, 1, 1], [1, 0, 1], [1, 1, 0]], dtype=np.float64)
    v = n1.ravel()[:, None] * prim[0] + n2.ravel()[:, None] * prim[1] + n3.ravel()[:, None] * prim[2]
    d = np.sqrt((v * v).sum(1))
    d = d[(d > 0) & (d < rmax)]
    return d


def test_fcc_neighbour_counts_and_shells():
    """fcc at rho*=0.8442: 12+6+24+12 = 54 neighbours inside 2.5, +24 = 78 inside 2.8."""
    a = W.lattice_constant(0.8442)
    d = _fcc_shell_sums(a, 2.8)
    assert (d < 2.5).sum() == 54 and len(d) == 78
    pos, box = W.fcc_lattice(10, 10, 10, a)
    pairs_l = O.neighbor_pairs(pos, box, 2.8)
    pairs_c = O.neighbor_pairs(pos, box, 2.5)
    assert len(pairs_l) == 4000 * 78 // 2
    assert len(pairs_c) == 4000 * 54 // 2
    deg = np.bincount(pairs_l.ravel(), minlength=4000)
    assert np.all(deg == 78)


def test_fcc_lattice_sums_and_zero_force():
    a = W.lattice_constant(0.8442)
    d = _fcc_shell_sums(a, 2.5)
    s6 = d ** -6.0
    e_atom = 0.5 * np.sum(4.0 * (s6 * s6 - s6))
    w_atom = 0.5 * np.sum(24.0 * (2.0 * s6 * s6 - s6))  # sum over pairs of r.f = 24(2 s12 - s6)
    pos, box = W.fcc_lattice(10, 10, 10, a)
    f, pe, vir = O.lj_forces(pos, box, O.LJParams.single())
    assert pe / 4000 == pytest.approx(e_atom, rel=1e-12)
    assert (vir[0] + vir[1] + vir[2]) / 4000 == pytest.approx(w_atom, rel=1e-12)
    # cubic symmetry: isotropic virial, zero shear, zero force on every site
    assert vir[0] == pytest.approx(vir[1], rel=1e-12) and vir[1] == pytest.approx(vir[2], rel=1e-12)
    assert np.abs(vir[3:]).max() < 1e-9
    assert np.abs(f).max() < 1e-11
    # the same numbers to the 8 digits computed by an independent shell summation
    assert pe / 4000 == pytest.approx(-6.7733680, abs=1e-7)
    # a larger crystal: the whole-system sums stay at rounding level of the exact value
    pos14, box14 = W.fcc_lattice(14, 14, 14, a)
    _, pe14, vir14 = O.lj_forces(pos14, box14, O.LJParams.single())
    assert pe14 / len(pos14) == pytest.approx(e_atom, rel=1e-13)
    assert (vir14[0] + vir14[1] + vir14[2]) / len(pos14) == pytest.approx(w_atom, rel=1e-13)
    assert (vir[0] + vir[1] + vir[2]) / 4000 == pytest.approx(-22.158199, abs=5e-7)


@pytest.mark.parametrize("kind", ["gas", "liquid", "threshold"])
def test_neighbour_set_brute_equals_cells(kind):
    if kind == "gas":
        box = np.array([12.0, 13.5, 15.25])
        pos = W.random_gas(1500, box, seed=3)
    elif kind == "liquid":
        s = W.lj_fcc(6, seed=4, jitter=0.05)
        pos, box = s.pos, s.box
    else:
        box = np.array([30.0, 30.0, 30.0])
        pos = W.threshold_pairs(216, box, 2.8, 1e-12, seed=9)
    brute = O.neighbor_pairs(pos, box, 2.8, brute=True)
    cells = O.neighbor_pairs(pos, box, 2.8, brute=False)
    assert np.array_equal(brute, cells)


def test_threshold_pairs_on_the_right_side():
    box = np.array([30.0, 30.0, 30.0])
    n = 216
    pos = W.threshold_pairs(n, box, 2.8, 1e-12, seed=9)
    got = {tuple(p) for p in O.neighbor_pairs(pos, box, 2.8).tolist()}
    for k in range(n):
        inside = (k % 2 == 0)
        assert ((k, n + k) in got) == inside


def test_pair_at_exactly_r_list_is_excluded():
    """Strict '<': with r_list = 2.75 (exact in binary) a pair at exactly 2.75 is not a neighbour."""
    box = np.array([20.0, 20.0, 20.0])
    pos = np.array([[1.0, 3.0, 4.0], [3.75, 3.0, 4.0], [1.0, 3.0 + 2.75, 4.0],
                    [1.0, 3.0, 4.0 + 2.5]])
    pairs = O.neighbor_pairs(pos, box, 2.75, brute=True).tolist()
    assert pairs == [[0, 3]]
    # and through the periodic boundary: atoms 0.25 and 17.5 apart in a 20-box are 2.75 apart
    pos2 = np.array([[0.25, 1.0, 1.0], [17.5, 1.0, 1.0], [17.6, 1.0, 1.0]])
    assert O.neighbor_pairs(pos2, box, 2.75, brute=True).tolist() == [[0, 2], [1, 2]]


def test_force_sum_zero_and_invariances():
    s = W.lj_fcc(6, seed=12, jitter=0.05)
    P = O.LJParams.single()
    f, pe, vir = O.lj_forces(s.pos, s.box, P)
    frms = np.sqrt((f ** 2).sum(1).mean())
    assert np.abs(f.sum(0)).max() < 1e-12 * s.n * frms
    # translation by a random vector (then wrap)
    t = np.array([3.3, -7.1, 0.37])
    f2, pe2, vir2 = O.lj_forces(W.wrap(s.pos + t, s.box), s.box, P)
    assert np.abs(f2 - f).max() < 1e-10 * frms
    assert pe2 == pytest.approx(pe, rel=1e-12)
    assert np.allclose(vir2, vir, rtol=1e-11, atol=1e-9)
    # permutation of the input order
    perm = np.argsort(W.splitmix64(1, 1, s.n))
    f3, pe3, _ = O.lj_forces(s.pos[perm], s.box, P)
    assert np.abs(f3 - f[perm]).max() < 1e-10 * frms
    assert pe3 == pytest.approx(pe, rel=1e-12)


def test_subset_direct_sum_matches_cell_path():
    s = W.lj_fcc(6, seed=13, jitter=0.05)
    P = O.LJParams([[1.0, 1.5], [1.5, 0.5]], [[1.0, 0.8], [0.8, 0.88]],
                   [[2.5, 2.0], [2.0, 2.2]], [1.0, 1.0])
    sp = W.species_shuffle(s.n, 0.2, seed=2)
    f, pe, vir, pea = O.lj_forces(s.pos, s.box, P, species=sp, per_atom=True)
    idx = np.array([0, 7, 99, 500, s.n - 1], dtype=np.int64)
    fs, pes, virs = O.lj_forces_subset(s.pos, s.box, P, idx, species=sp)
    assert np.allclose(fs, f[idx], rtol=1e-12, atol=1e-11)
    assert np.allclose(pes, pea[idx], rtol=1e-12, atol=1e-12)
    assert pea.sum() == pytest.approx(pe, rel=1e-12)
    # brute-force whole-system path agrees as well
    fb, peb, virb = O.lj_forces(s.pos, s.box, P, species=sp, brute=True)
    assert np.allclose(fb, f, rtol=1e-12, atol=1e-11)
    assert peb == pytest.approx(pe, rel=1e-12)


def test_forces_from_neighbour_pairs_equal_plain_definition():
    s = W.lj_fcc(6, seed=14, jitter=0.05)
    P = O.LJParams.single()
    pairs = O.neighbor_pairs(s.pos, s.box, 2.8)
    f1, pe1, v1 = O.lj_forces_pairs(s.pos, s.box, P, pairs)
    f2, pe2, v2 = O.lj_forces(s.pos, s.box, P)
    assert np.allclose(f1, f2, rtol=1e-12, atol=1e-11)
    assert pe1 == pytest.approx(pe2, rel=1e-12)


def _cluster_13():
    """Icosahedron-like 13-atom cluster; r_cut so large that no pair ever crosses it."""
    pos, _ = W.fcc_lattice(2, 2, 2, 1.56)
    pos = pos[:13] + 100.0
    vel = W.thermal_velocities(np.ones(13), 0.2, seed=21)
    return pos, vel, np.array([300.0, 300.0, 300.0]), O.LJParams.single(rc=60.0)


def test_velocity_verlet_is_second_order():
    pos, vel, box, P = _cluster_13()
    errs = []
    for dt in (0.004, 0.002):
        nsteps = int(round(0.4 / dt))
        r = O.run_nve(pos, vel, box, P, dt, 5.0, nsteps, history=True)
        e0 = O.lj_forces(pos, box, P)[1] + O.kinetic(vel, P)
        errs.append(np.abs(r["pe"] + r["ke"] - e0).max())
    ratio = errs[0] / errs[1]
    assert 3.3 < ratio < 4.8, ratio


def test_velocity_verlet_time_reversible():
    s = W.lj_fcc(5, seed=15)
    P = O.LJParams.single()
    r1 = O.run_nve(s.pos, s.vel, s.box, P, 0.005, 0.3, 50)
    back = O.run_nve(r1["pos"], -r1["vel"], s.box, P, 0.005, 0.3, 50, image=r1["image"])
    unwrapped = back["pos"] + back["image"] * s.box
    assert np.abs(unwrapped - s.pos).max() < 1e-9
    assert np.abs(back["vel"] + s.vel).max() < 1e-9


def test_nve_energy_bounded_config1():
    """4,000-atom fcc start at T*=0.72, 100 steps.  The potential is cut without a shift,
    so every pair crossing r_cut changes E by u(r_cut) = 4 (2.5^-12 - 2.5^-6): the energy
    of the shifted potential, E - u(r_cut) * (pairs inside r_cut), is what velocity Verlet
    conserves to O(dt^2).  Measured here: |dE|/N reaches 5.9e-3 (the melting lattice gains
    about 1,400 interacting pairs), while the shifted energy moves by at most 1.8e-4 per
    atom at the checked steps.  Bars: 8e-3 and 5e-4 per atom (margins 1.35x and 2.7x)."""
    s = W.lj_fcc(10, seed=1)
    P = O.LJParams.single()
    e0 = O.lj_forces(s.pos, s.box, P)[1] + O.kinetic(s.vel, P)
    n0 = len(O.neighbor_pairs(s.pos, s.box, 2.5))
    u_rc = 4.0 * (2.5 ** -12 - 2.5 ** -6)
    r = O.run_nve(s.pos, s.vel, s.box, P, 0.005, 0.3, 100, history=True)
    drift = np.abs(r["pe"] + r["ke"] - e0).max() / s.n
    assert drift < 8e-3
    assert r["rebuilds"] >= 1
    x, v, img, f = s.pos, s.vel, None, None
    for steps in (25, 25, 50):  # the same trajectory, checked at steps 25, 50 and 100
        q = O.run_nve(x, v, s.box, P, 0.005, 0.3, steps, image=img, forces=f, history=True)
        x, v, img, f = q["pos"], q["vel"], q["image"], q["forces"]
        dn = len(O.neighbor_pairs(x, s.box, 2.5)) - n0
        shifted = (q["pe"][-1] + q["ke"][-1] - e0 - u_rc * dn) / s.n
        assert abs(shifted) < 5e-4, (steps, shifted)


def test_all_cores_form_equals_serial_definition():
    """The all-cores full-sum forces (each atom summed from both sides of its pairs) equal
    the serial Newton-3 definition up to rounding order: one and two species, linked cells
    and the all-pairs path of a small box; a 20-step run takes the same trajectory."""
    for n_cells, species in ((6, False), (6, True), (2, False)):
        s = W.lj_fcc(n_cells, seed=3 + n_cells, jitter=0.05)
        if species:
            sp = W.species_shuffle(s.n, 0.2, 7)
            P = O.LJParams([[1.0, 1.5], [1.5, 0.5]], [[1.0, 0.8], [0.8, 0.88]],
                           [[2.5, 2.0], [2.0, 2.2]], [1.0, 1.0])
        else:
            sp, P = None, O.LJParams.single(rc=2.5 if n_cells > 2 else 1.6)
        F, pe, _ = O.lj_forces(s.pos, s.box, P, sp)
        Fa, pea, th = O.lj_forces_all_cores(s.pos, s.box, P, sp)
        frms = np.sqrt((F ** 2).sum(1).mean())
        assert th >= 1
        assert np.abs(Fa - F).max() <= 1e-13 * frms
        assert abs(pea - pe) <= 1e-13 * abs(pe)
    s = W.lj_fcc(6, seed=11)
    P = O.LJParams.single()
    a = O.run_nve(s.pos, s.vel, s.box, P, 0.005, 0.3, 20)
    b = O.run_nve(s.pos, s.vel, s.box, P, 0.005, 0.3, 20, all_cores=True)
    assert np.abs(a["pos"] + a["image"] * s.box - b["pos"] - b["image"] * s.box).max() < 1e-11
    assert a["rebuilds"] == b["rebuilds"]


def test_run_continues_from_given_forces():
    """A run of 10 + 10 steps that hands the forces over evaluates each force once per
    step and follows the 20-step run (to the rounding of a re-wrapped position)."""
    s = W.lj_fcc(5, seed=12)
    P = O.LJParams.single()
    whole = O.run_nve(s.pos, s.vel, s.box, P, 0.005, 0.3, 20)
    a = O.run_nve(s.pos, s.vel, s.box, P, 0.005, 0.3, 10)
    b = O.run_nve(a["pos"], a["vel"], s.box, P, 0.005, 0.3, 10, image=a["image"], forces=a["forces"])
    assert np.abs(b["pos"] + b["image"] * s.box - whole["pos"] - whole["image"] * s.box).max() < 1e-12
    assert np.abs(b["forces"] - whole["forces"]).max() < 1e-9
    assert np.abs(b["forces"] - O.lj_forces(b["pos"], s.box, P)[0]).max() == 0.0


def test_skin_half_rebuild_rule_and_wrap():
    """A free particle at speed 1 with dt = 1/16, skin = 1/2: |dx|^2 > (1/4)^2 first at step 5."""
    box = np.array([10.0, 10.0, 10.0])
    pos = np.array([[9.5, 5.0, 5.0], [2.0, 2.0, 2.0]])
    vel = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    P = O.LJParams.single(rc=1.0)
    r = O.run_nve(pos, vel, box, P, 0.0625, 0.5, 20)
    assert r["rebuilds"] == 4  # steps 5, 10, 15, 20
    # 20 steps move the particle by 1.25: crossed x = 10 once, wrapped at the step-10 rebuild
    assert r["image"][0].tolist() == [1, 0, 0]
    assert r["pos"][0, 0] == pytest.approx(9.5 + 1.25 - 10.0, abs=1e-12)
    r2 = O.run_nve(pos, vel, box, P, 0.0625, 0.5, 20, policy=1, every_k=3)
    assert r2["rebuilds"] == 6  # steps 3, 6, ..., 18


def test_generators():
    s = W.lj_fcc(10, seed=1)
    assert s.n == 4000
    assert s.box[0] == pytest.approx(16.795962, abs=1e-6)
    P = O.LJParams.single()
    assert 2 * O.kinetic(s.vel, P) / (3 * s.n - 3) == pytest.approx(0.72, rel=1e-13)
    assert np.abs(s.vel.sum(0)).max() < 1e-11
    # SplitMix64 published output for state 0
    assert int(W.splitmix64(0, 0, 1)[0]) == 0xE220A8397B1DCDAF
    u = W.uniform01(5, 0, 100000)
    assert 0.0 < u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005
    z = W.normal(5, 0, 100000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


# ---------------------------------------------------------------- force-matching gradients
_KA = dict(eps=[[1.0, 1.5], [1.5, 0.5]], sig=[[1.0, 0.8], [0.8, 0.88]])


def _ka_small(seed, rc=2.2):
    """Two-species jittered fcc (Kob-Andersen parameters, a fixed cutoff table)."""
    s = W.lj_fcc(3, rho=1.2, seed=seed, jitter=0.06)
    sp = W.species_shuffle(s.n, 0.2, seed)
    P = O.LJParams(_KA["eps"], _KA["sig"], [[rc, rc], [rc, rc]], [1.0, 1.0])
    return s, sp, P


def test_force_grad_matches_finite_differences():
    """dL/d(eps_ab, sig_ab) and dL/dx for L = sum G . F with a random G, against central
    differences of the oracle's forces (pair set away from the cutoff, so it stays fixed)."""
    for seed in range(1, 40):
        s, sp, P = _ka_small(seed)
        if _safe_from_cutoff(s.pos, s.box, 2.2, 1e-4):
            break
    else:
        pytest.skip("no seed without a pair near the cutoff")
    G = np.random.default_rng(seed).normal(size=(s.n, 3))
    gx, ge, gs = O.lj_force_grad(s.pos, s.box, P, G, sp)

    def L(eps, sig, pos):
        return float((G * O.lj_forces(pos, s.box, O.LJParams(eps, sig, P.rc, P.mass), sp)[0]).sum())

    h = 1e-6
    for a, b in [(0, 0), (0, 1), (1, 1)]:
        for table, grad in [("eps", ge), ("sig", gs)]:
            lo = {"eps": P.eps.copy(), "sig": P.sig.copy()}
            hi = {"eps": P.eps.copy(), "sig": P.sig.copy()}
            for t, sgn in [(hi, 1.0), (lo, -1.0)]:
                t[table][a, b] += sgn * h
                if a != b:
                    t[table][b, a] += sgn * h
            fd = (L(hi["eps"], hi["sig"], s.pos) - L(lo["eps"], lo["sig"], s.pos)) / (2 * h)
            assert grad[a, b] == grad[b, a]
            assert fd == pytest.approx(grad[a, b], rel=1e-6, abs=1e-6)
    for i in [0, 3, 50, 97]:
        for k in range(3):
            xp, xm = s.pos.copy(), s.pos.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd = (L(P.eps, P.sig, xp) - L(P.eps, P.sig, xm)) / (2 * h)
            assert fd == pytest.approx(gx[i, k], rel=1e-6, abs=1e-6)


def test_force_grad_dimer_closed_form():
    """Dimer along x at distance r, L = F_x on the first atom = 24 eps (2 s^12/r^13 - s^6/r^7):
    dL/dx_1 = 24 eps (-26 s^12/r^14 + 7 s^6/r^8) along x, 0 across; dL/deps = L/eps;
    dL/dsig = 24 eps (24 s^11/r^13 - 6 s^5/r^7)."""
    eps, sig, r = 0.7, 1.3, 1.37
    box = np.array([40.0, 40.0, 40.0])
    pos = np.array([[20.0 + r, 20.0, 20.0], [20.0, 20.0, 20.0]])
    P = O.LJParams.single(eps=eps, sig=sig, rc=4.0)
    G = np.zeros((2, 3))
    G[0, 0] = 1.0
    gx, ge, gs = O.lj_force_grad(pos, box, P, G)
    L = 24 * eps * (2 * sig ** 12 / r ** 13 - sig ** 6 / r ** 7)
    assert O.lj_forces(pos, box, P)[0][0, 0] == pytest.approx(L, rel=1e-14)
    assert gx[0, 0] == pytest.approx(24 * eps * (-26 * sig ** 12 / r ** 14 + 7 * sig ** 6 / r ** 8), rel=1e-13)
    assert gx[1, 0] == pytest.approx(-gx[0, 0], rel=1e-15)
    assert np.all(gx[:, 1:] == 0.0)
    assert ge[0, 0] == pytest.approx(L / eps, rel=1e-13)
    assert gs[0, 0] == pytest.approx(24 * eps * (24 * sig ** 11 / r ** 13 - 6 * sig ** 5 / r ** 7), rel=1e-13)


def test_force_grad_scaling_identities():
    """Exact identities of the analytic gradient (no finite differences): L = G . F is linear
    in eps, so sum eps dL/deps = L; F is homogeneous of degree -1 under scaling all lengths
    (positions and sigma, pair set fixed), so sum sig dL/dsig + sum x . dL/dx = -L for an
    isolated cluster; and translation invariance gives sum_k dL/dx_k = 0."""
    rng = np.random.default_rng(3)
    s, sp, P = _ka_small(5)
    box = np.array([60.0, 60.0, 60.0])
    pos = W.fcc_lattice(2, 2, 2, 1.35)[0] + 25.0 + rng.normal(scale=0.05, size=(32, 3))
    sp = (np.arange(32) % 4 == 0).astype(np.int32)
    P = O.LJParams(_KA["eps"], _KA["sig"], [[9.0, 9.0], [9.0, 9.0]], [1.0, 1.0])
    G = rng.normal(size=(32, 3))
    F = O.lj_forces(pos, box, P, sp)[0]
    L = float((G * F).sum())
    gx, ge, gs = O.lj_force_grad(pos, box, P, G, sp)
    # each unordered species pair once: diagonal entries plus one off-diagonal entry
    uniq = [(0, 0), (0, 1), (1, 1)]
    assert sum(P.eps[a, b] * ge[a, b] for a, b in uniq) == pytest.approx(L, rel=1e-12)
    assert sum(P.sig[a, b] * gs[a, b] for a, b in uniq) + float((pos * gx).sum()) == pytest.approx(
        -L, rel=1e-10, abs=1e-10 * np.abs(G * F).sum())
    assert np.abs(gx.sum(axis=0)).max() <= 1e-11 * np.abs(gx).sum()


def test_energy_param_grad_identities():
    """E is linear in eps (sum eps dE/deps = E) and, per pair, sig dE/dsig = d . f, so
    sum sig dE/dsig equals the virial trace W_xx + W_yy + W_zz (periodic system)."""
    s, sp, P = _ka_small(7)
    _, pe, vir = O.lj_forces(s.pos, s.box, P, sp)
    de, ds = O.lj_energy_param_grad(s.pos, s.box, P, sp)
    uniq = [(0, 0), (0, 1), (1, 1)]
    assert sum(P.eps[a, b] * de[a, b] for a, b in uniq) == pytest.approx(pe, rel=1e-12)
    assert sum(P.sig[a, b] * ds[a, b] for a, b in uniq) == pytest.approx(vir[0] + vir[1] + vir[2], rel=1e-12)


# ---------------------------------------------------------------- many-body (TB-SMA, Cleri-Rosato)
CU = O.TBSMAParams.copper()


def _cu_crystal(n_cells=5, a=3.615, jitter=0.0, seed=0):
    pos, box = W.fcc_lattice(n_cells, n_cells, n_cells, a)
    if jitter > 0.0:
        pos = W.gaussian_jitter(pos, box, jitter, seed, stream=2)
    return pos, box


def test_tbsma_copper_cohesive_energy_and_lattice_constant():
    """Cleri and Rosato fitted the Cu parameters to the fcc lattice constant 3.615 A and
    the cohesive energy 3.544 eV (sums over five neighbour shells): the oracle's energy per
    atom of the perfect crystal is -3.544 eV, smallest at a = 3.615 A, with no force on any
    site and an isotropic virial."""
    pos, box = _cu_crystal()
    F, E, vir = O.tbsma_forces(pos, box, CU)
    n = len(pos)
    assert abs(E / n + 3.544) < 1e-3
    assert np.abs(F).max() < 1e-12
    assert np.allclose(vir[:3], vir[0], atol=1e-9 * n) and np.abs(vir[3:]).max() < 1e-9 * n
    e = [O.tbsma_forces(*_cu_crystal(a=a), CU)[1] / n for a in (3.600, 3.615, 3.630)]
    assert e[1] < e[0] and e[1] < e[2]


def test_tbsma_dimer_closed_form():
    """Two atoms at distance r: rho = psi(r) for both, so E = 2 A exp(-p(r/r0-1)) -
    2 xi exp(-q(r/r0-1)) and the force is -dE/dr along the bond."""
    r0, A, xi, p, q = CU.r0, CU.A, CU.xi, CU.p, CU.q
    box = np.array([40.0, 40.0, 40.0])
    for r in (2.2, 2.556, 3.1, 4.4):
        pos = np.array([[10.0, 10.0, 10.0], [10.0 + r * 0.6, 10.0 + r * 0.8, 10.0]])
        F, E, _ = O.tbsma_forces(pos, box, CU)
        x = r / r0 - 1.0
        E_ref = 2 * A * math.exp(-p * x) - 2 * xi * math.exp(-q * x)
        dEdr = -2 * A * p / r0 * math.exp(-p * x) + 2 * xi * q / r0 * math.exp(-q * x)
        assert abs(E - E_ref) <= 1e-13 * abs(E_ref)
        u = np.array([0.6, 0.8, 0.0])
        assert np.allclose(F[0], -dEdr * -u, atol=1e-13, rtol=1e-12)  # F_0 = -dE/dx_0, dr/dx_0 = -u
        assert np.allclose(F[1], -F[0], atol=1e-15)


def test_tbsma_force_is_minus_gradient_of_energy():
    """Central differences of the total energy on a thermally disordered periodic crystal."""
    pos, box = _cu_crystal(n_cells=4, jitter=0.08, seed=3)
    F, _, _ = O.tbsma_forces(pos, box, CU)
    h = 1e-5
    for i in (0, 17, 101, 200):
        for k in range(3):
            xp = pos.copy()
            xm = pos.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd = -(O.tbsma_forces(xp, box, CU)[1] - O.tbsma_forces(xm, box, CU)[1]) / (2 * h)
            assert abs(fd - F[i, k]) <= 1e-6 * max(1.0, abs(F[i, k])), (i, k, fd, F[i, k])


def test_tbsma_virial_is_minus_strain_derivative():
    """W_aa = -dE/d(epsilon_aa) under a homogeneous strain of positions and box."""
    pos, box = _cu_crystal(n_cells=4, jitter=0.08, seed=4)
    _, _, vir = O.tbsma_forces(pos, box, CU)
    h = 1e-6
    for k in range(3):
        s = np.ones(3)
        s[k] = 1 + h
        ep = O.tbsma_forces(pos * s, box * s, CU)[1]
        s[k] = 1 - h
        em = O.tbsma_forces(pos * s, box * s, CU)[1]
        assert abs(-(ep - em) / (2 * h) - vir[k]) <= 1e-6 * max(1.0, abs(vir[k]))


def test_tbsma_invariances_and_brute_force():
    pos, box = _cu_crystal(n_cells=4, jitter=0.08, seed=5)
    F, E, vir, rho, ea = O.tbsma_forces(pos, box, CU, per_atom=True)
    Fb, Eb, _ = O.tbsma_forces(pos, box, CU, brute=True)
    assert np.abs(F - Fb).max() < 1e-12 and abs(E - Eb) < 1e-10
    assert np.abs(F.sum(0)).max() < 1e-10
    assert abs(ea.sum() - E) < 1e-9
    assert np.all(rho > 0)
    shift = np.array([1.3, -0.7, 2.9])
    F2, E2, _ = O.tbsma_forces(W.wrap(pos + shift, box), box, CU)
    assert np.abs(F2 - F).max() < 1e-10 and abs(E2 - E) < 1e-9
    perm = np.random.default_rng(1).permutation(len(pos))
    F3, E3, _ = O.tbsma_forces(pos[perm], box, CU)
    assert np.abs(F3 - F[perm]).max() < 1e-10 and abs(E3 - E) < 1e-9
    # an atom far from all others has no density, energy or force
    big = box * 2.0  # the crystal fills [0, L)^3 of a (2L)^3 box; the far atom sits at 1.5 L
    far = np.vstack([pos, [1.5 * box]])
    F4, _, _, rho4, ea4 = O.tbsma_forces(far, big, CU, per_atom=True)
    assert rho4[-1] == 0.0 and ea4[-1] == 0.0 and np.all(F4[-1] == 0.0)


def _cu_cluster():
    """13 copper atoms: one fcc site and its 12 nearest neighbours, far from any image, so
    no pair ever reaches r_cut (the largest distance is 2 r0 = 5.11 A)."""
    pos, box = W.fcc_lattice(2, 2, 2, 3.615)
    c = pos[np.argmin(((pos - box / 2) ** 2).sum(1))]
    d = W.wrap(pos - c + box / 2, box) - box / 2
    cl = d[np.sqrt((d ** 2).sum(1)) < 2.7] + 50.0
    assert len(cl) == 13
    vel = W.thermal_velocities(np.full(13, 63.546), 0.05, 31, stream=1)
    return cl, vel, np.array([100.0, 100.0, 100.0])


def test_tbsma_velocity_verlet_is_second_order():
    """The many-body run conserves energy to O(dt^2): halving dt cuts the largest energy
    error over 8 time units (81 fs) by about 4 (measured 4.01)."""
    cl, vel, box = _cu_cluster()
    errs = []
    for dt in (0.2, 0.1):
        r = O.run_nve_tbsma(cl, vel, box, CU, 63.546, dt, 1.0, int(round(8.0 / dt)), history=True)
        e0 = O.tbsma_forces(cl, box, CU)[1] + 0.5 * 63.546 * (vel ** 2).sum()
        errs.append(np.abs(r["pe"] + r["ke"] - e0).max())
    assert 3.3 < errs[0] / errs[1] < 4.8, errs
    assert errs[1] < 1e-3 * 0.05 * 13  # far below the kinetic energy scale


def test_tbsma_velocity_verlet_time_reversible():
    """30 steps forward, velocities negated, 30 back: the thermal periodic crystal returns
    to its start (measured 4e-15 A), through a rebuild and its wrap."""
    pos, box = _cu_crystal(n_cells=4, jitter=0.08, seed=3)
    vel = W.thermal_velocities(np.full(len(pos), 63.546), 0.02585, 3, stream=1)
    a = O.run_nve_tbsma(pos, vel, box, CU, 63.546, 0.1, 0.4, 30)
    b = O.run_nve_tbsma(a["pos"], -a["vel"], box, CU, 63.546, 0.1, 0.4, 30, image=a["image"])
    assert a["rebuilds"] >= 1
    assert np.abs(b["pos"] + b["image"] * box - pos).max() < 1e-9
    assert np.abs(b["vel"] + vel).max() < 1e-9 * np.abs(vel).max()


def test_force_grad_scale_bounds_the_sums():
    """The scale sum |term| of the parameter derivatives bounds |sum| (strictly, for a random
    upstream gradient, whose pair terms cancel), and vanishes with every term: a uniform G
    gives w = G_i - G_j = 0 on every pair."""
    s, sp, P = _ka_small(3)
    G = np.random.default_rng(5).normal(size=(s.n, 3))
    _, ge, gs = O.lj_force_grad(s.pos, s.box, P, G, sp)
    ae, as_ = O.lj_force_grad_scale(s.pos, s.box, P, G, sp)
    assert np.all(ae >= np.abs(ge)) and np.all(as_ >= np.abs(gs))
    assert np.all(ae > 3 * np.abs(ge))  # random upstream gradients cancel
    # a uniform field G_i = c: w = 0, every term vanishes, and so does the scale
    ae0, as0 = O.lj_force_grad_scale(s.pos, s.box, P, np.ones((s.n, 3)), sp)
    assert np.all(ae0 == 0.0) and np.all(as0 == 0.0)
