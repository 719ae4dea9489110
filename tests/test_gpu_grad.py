"""Force-matching derivatives on the GPU (through the C ABI) against the FP64 oracle.

md_forces_backward gives dL/dx, dL/deps and dL/dsigma for dL/dF = G on the pairs inside
their cutoffs (pair set fixed); md_energy_param_grad gives dE/deps and dE/dsigma.  Inputs:
Kob-Andersen binary mixture snapshots (fcc sites at rho* = 1.2, seeded 80:20 species
shuffle, Gaussian jitter), the workload shape of the force-matching experiment.
Bars: FP64 systems within 1e-11 of the oracle (relative, per atom against the RMS for
positions); mixed systems (FP32 pair terms) within 2e-5.
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
from paper_1305_4196_gb300.autograd import lj_forces  # noqa: E402

KA_EPS = np.array([[1.0, 1.5], [1.5, 0.5]])
KA_SIG = np.array([[1.0, 0.8], [0.8, 0.88]])
TOL = {"fp64": 1e-11, "mixed": 2e-5}
PREC = {"fp64": M.MD_FP64, "mixed": M.MD_MIXED}


def ka_snapshot(n_cells=10, seed=1, jitter=0.05):
    s = W.lj_fcc(n_cells, rho=1.2, seed=seed, jitter=jitter)
    sp = W.species_shuffle(s.n, 0.2, seed)
    return s, sp


def vec_error(g, gref):
    mag = np.sqrt((gref ** 2).sum(1))
    rms = np.sqrt((mag ** 2).mean())
    return float((np.sqrt(((g - gref) ** 2).sum(1)) / np.maximum(mag, rms)).max())


def make(s, sp, precision, rc):
    sysm = M.System(s.n, s.box, r_cut=float(rc.max()), skin=0.3, eps=KA_EPS, sigma=KA_SIG, mass=[1.0, 1.0],
                    precision=PREC[precision], rcut=rc)
    sysm.set_state(np.ascontiguousarray(s.pos), np.zeros_like(s.pos), sp)
    return sysm


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_backward_matches_oracle(precision):
    s, sp = ka_snapshot()
    rc = 2.5 * KA_SIG
    P = O.LJParams(KA_EPS, KA_SIG, rc, [1.0, 1.0])
    G = np.random.default_rng(2).normal(size=(s.n, 3))
    gx_ref, ge_ref, gs_ref = O.lj_force_grad(s.pos, s.box, P, G, sp)
    sysm = make(s, sp, precision, rc)
    gx, ge, gs = sysm.forces_backward(G)
    assert vec_error(gx, gx_ref) <= TOL[precision]
    assert np.array_equal(ge, ge.T) and np.array_equal(gs, gs.T)
    for t, tref in [(ge, ge_ref), (gs, gs_ref)]:
        assert np.abs(t - tref).max() <= TOL[precision] * np.abs(tref).max()
    # deterministic
    gx2, ge2, gs2 = sysm.forces_backward(G)
    assert np.array_equal(gx, gx2) and np.array_equal(ge, ge2) and np.array_equal(gs, gs2)


def test_backward_on_a_linear_block_grid():
    """6,912 atoms in a 17.9 sigma box: full lists take 6 cells per side (3 linearly
    numbered blocks per side, tiles of 4 of the 6 cells); FP64 derivatives at 1e-11."""
    s, sp = ka_snapshot(n_cells=12, seed=5)
    rc = 2.5 * KA_SIG
    P = O.LJParams(KA_EPS, KA_SIG, rc, [1.0, 1.0])
    G = np.random.default_rng(5).normal(size=(s.n, 3))
    sysm = make(s, sp, "fp64", rc)
    gx, ge, gs = sysm.forces_backward(G)
    assert sysm.info()["ncell"] == [6, 6, 6]
    gx_ref, ge_ref, gs_ref = O.lj_force_grad(s.pos, s.box, P, G, sp)
    assert vec_error(gx, gx_ref) <= TOL["fp64"]
    for t, tref in [(ge, ge_ref), (gs, gs_ref)]:
        assert np.abs(t - tref).max() <= TOL["fp64"] * np.abs(tref).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_energy_param_grad_matches_oracle(precision):
    s, sp = ka_snapshot(seed=3)
    rc = 2.5 * KA_SIG
    P = O.LJParams(KA_EPS, KA_SIG, rc, [1.0, 1.0])
    de_ref, ds_ref = O.lj_energy_param_grad(s.pos, s.box, P, sp)
    de, ds = make(s, sp, precision, rc).energy_param_grad()
    tol = 1e-11 if precision == "fp64" else 1e-5
    assert np.abs(de - de_ref).max() <= tol * np.abs(de_ref).max()
    assert np.abs(ds - ds_ref).max() <= tol * np.abs(ds_ref).max()


def test_set_params_forces_match_oracle():
    """Perturbed parameters (each value scaled by 1 +/- 10 %) with their scaled cutoffs."""
    s, sp = ka_snapshot(seed=4)
    rc0 = 2.5 * KA_SIG * 1.1
    sysm = make(s, sp, "fp64", rc0)
    sgn = np.where(W.uniform01(4, 9, 6) < 0.5, -1.0, 1.0)
    e = KA_EPS * (1 + 0.1 * np.array([[sgn[0], sgn[1]], [sgn[1], sgn[2]]]))
    g = KA_SIG * (1 + 0.1 * np.array([[sgn[3], sgn[4]], [sgn[4], sgn[5]]]))
    sysm.set_params(e, g, 2.5 * g)
    F = sysm.forces()
    Fref, _, _ = O.lj_forces(s.pos, s.box, O.LJParams(e, g, 2.5 * g, [1.0, 1.0]), sp)
    assert vec_error(F, Fref) <= 1e-12
    with pytest.raises(M.MDError):
        sysm.set_params(e, g, np.full((2, 2), 3.0))  # beyond the 2.75 the lists were sized for


def test_force_matching_gradient_by_finite_differences():
    """torch.autograd through the CUDA forward and backward (FP64 path): loss = mean squared
    force error against target forces of the reference parameters, at parameters perturbed
    by 10 %; dloss/d(eps, sigma) and dloss/dx against central differences of the GPU
    forward (fixed cutoff table, so the pair set does not change)."""
    s, sp = ka_snapshot(n_cells=8, seed=5)
    rc = np.full((2, 2), 2.3)
    dev = torch.device("cuda")
    sysm = make(s, sp, "fp64", rc)
    spt = torch.as_tensor(sp, dtype=torch.int32, device=dev)
    target = lj_forces(torch.as_tensor(s.pos, device=dev), torch.as_tensor(KA_EPS), torch.as_tensor(KA_SIG), sysm,
                       spt, rc).detach()
    eps = torch.tensor(KA_EPS * 1.1, requires_grad=True)
    sig = torch.tensor(KA_SIG * np.array([[0.95, 1.05], [1.05, 0.97]]), requires_grad=True)
    pos = torch.tensor(s.pos, device=dev, requires_grad=True)

    def loss_of(p, e, g):
        F = lj_forces(p, e, g, sysm, spt, rc)
        return ((F - target) ** 2).mean()

    loss = loss_of(pos, eps, sig)
    loss.backward()
    # central differences with step h: rounding error ~ eps_mach * loss / h, truncation
    # ~ h^2 * (third derivative) / 6, well below 1e-7 here
    h = 1e-5
    tol_abs = 20 * 2.2e-16 * loss.item() / h + 1e-7
    for table, grad in [("eps", eps.grad), ("sig", sig.grad)]:
        for a, b in [(0, 0), (0, 1), (1, 1)]:
            d = torch.zeros(2, 2, dtype=torch.float64)
            d[a, b] = d[b, a] = h
            e0, g0 = eps.detach(), sig.detach()
            lp = loss_of(pos.detach(), e0 + d if table == "eps" else e0, g0 + d if table == "sig" else g0).item()
            lm = loss_of(pos.detach(), e0 - d if table == "eps" else e0, g0 - d if table == "sig" else g0).item()
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grad[a, b].item()) <= 1e-6 * abs(fd) + tol_abs
    gpos = pos.grad.cpu().numpy()
    for i in [0, 17, 600]:
        for k in range(3):
            d = torch.zeros_like(pos)
            d[i, k] = h
            lp = loss_of(pos.detach() + d, eps.detach(), sig.detach()).item()
            lm = loss_of(pos.detach() - d, eps.detach(), sig.detach()).item()
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gpos[i, k]) <= 1e-6 * abs(fd) + tol_abs
    assert abs(gpos.sum(0)).max() <= 1e-10 * np.abs(gpos).sum()


def test_backward_needs_full_lists():
    s, sp = ka_snapshot(n_cells=8)
    sysm = M.System(s.n, s.box, r_cut=2.5, skin=0.3, eps=KA_EPS, sigma=KA_SIG, mass=[1.0, 1.0],
                    list_kind=M.MD_LIST_HALF_COLOUR8, rcut=2.5 * KA_SIG)
    sysm.set_state(np.ascontiguousarray(s.pos), np.zeros_like(s.pos), sp)
    with pytest.raises(M.MDError) as e:
        sysm.forces_backward(np.zeros((s.n, 3)))
    assert e.value.code == M.MD_ERR_ARG


def test_backward_cutoff_decided_by_the_definition():
    """Pairs at r_cut (1 -/+ 1e-7) on a mixed system: the FP32 backward pass takes the FP64
    cutoff decision, so it matches the oracle's gradient."""
    box = np.array([30.0, 30.0, 30.0])
    pos = W.threshold_pairs(216, box, 2.5, 1e-7, seed=14)
    sp = np.zeros(len(pos), dtype=np.int32)
    P = O.LJParams.single()
    s = M.System(len(pos), box, r_cut=2.5, skin=0.3, precision=M.MD_MIXED)
    s.set_state(np.ascontiguousarray(pos), np.zeros_like(pos), sp)
    G = np.random.default_rng(3).normal(size=(len(pos), 3))
    gx, ge, gs = s.forces_backward(G)
    gx_ref, ge_ref, gs_ref = O.lj_force_grad(pos, box, P, G, sp)
    assert np.abs(gx - gx_ref).max() <= 2e-5 * np.abs(gx_ref).max()
    assert abs(ge[0, 0] - ge_ref[0, 0]) <= 2e-5 * abs(ge_ref[0, 0])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_backward_at_the_force_matching_size(precision):
    """The force-matching workload at its stated size, in the launch configuration the
    benchmark times: 32,000 Kob-Andersen atoms (20^3 fcc cells at rho* = 1.2, L = 29.88),
    lists sized for cutoffs 10 % above 2.5 sigma_ab (8 cells per side, so 64 blocks whose
    4x4x4-cell tiles are smaller than the box), parameters perturbed by 10 %; dL/dx,
    dL/deps and dL/dsigma for a random upstream gradient, and dE/deps, dE/dsigma, element
    by element against the oracle's analytic gradient.  Bars as above, except that the
    mixed parameter derivatives dL/deps and dL/dsigma - sums of about 1.3 million pair
    terms of both signs - are held to the per-term bar 2e-5 times the sum of |term| (the
    oracle's scale of each sum): their terms cancel, so a bound relative to the result
    would demand more than FP32 pair terms carry."""
    s, sp = ka_snapshot(n_cells=20, seed=101)
    eps1 = KA_EPS * np.array([[1.1, 0.9], [0.9, 1.1]])
    sig1 = KA_SIG * np.array([[0.9, 1.1], [1.1, 0.9]])
    sysm = M.System(s.n, s.box, r_cut=2.5 * 1.1, skin=0.3, eps=KA_EPS, sigma=KA_SIG, mass=[1.0, 1.0],
                    precision=PREC[precision], rcut=2.5 * KA_SIG * 1.1)
    sysm.set_state(np.ascontiguousarray(s.pos), np.zeros_like(s.pos), sp)
    sysm.set_params(eps1, sig1, 2.5 * sig1)
    assert sysm.info()["ncell"] == [8, 8, 8]
    P = O.LJParams(eps1, sig1, 2.5 * sig1, [1.0, 1.0])
    G = np.random.default_rng(7).normal(size=(s.n, 3))
    gx, ge, gs = sysm.forces_backward(G)
    gx_ref, ge_ref, gs_ref = O.lj_force_grad(s.pos, s.box, P, G, sp)
    ae, as_ = O.lj_force_grad_scale(s.pos, s.box, P, G, sp)
    assert vec_error(gx, gx_ref) <= TOL[precision]
    for t, tref, scale in [(ge, ge_ref, ae), (gs, gs_ref, as_)]:
        if precision == "fp64":
            assert np.abs(t - tref).max() <= TOL[precision] * np.abs(tref).max()
        else:
            assert np.all(np.abs(t - tref) <= TOL[precision] * scale)
    de, ds = sysm.energy_param_grad()
    de_ref, ds_ref = O.lj_energy_param_grad(s.pos, s.box, P, sp)
    tol = 1e-11 if precision == "fp64" else 1e-5
    assert np.abs(de - de_ref).max() <= tol * np.abs(de_ref).max()
    assert np.abs(ds - ds_ref).max() <= tol * np.abs(ds_ref).max()
    F = sysm.forces()
    Fref = O.lj_forces(s.pos, s.box, P, sp)[0]
    assert vec_error(F, Fref) <= (1e-12 if precision == "fp64" else 2e-5)


def test_backward_on_the_coarser_grid():
    """The mixed backward pass on the coarser, linearly numbered grid a homogeneous system
    takes at its first build: a 296,352-atom liquid (42^3 fcc cells at rho* = 0.8442, 22
    instead of 24 cells per side); dL/dx element by element against the oracle, and
    dL/deps, dL/dsigma to the per-term bar (2e-5 of the sum of |term|)."""
    w = W.lj_fcc(42, seed=6, jitter=0.05)
    sysm = M.System(w.n, w.box, r_cut=2.5, skin=0.3, precision=M.MD_MIXED)
    sysm.set_state(w.pos, w.vel, w.species)
    sysm.forces()
    assert sysm.info()["ncell"] == [22, 22, 22]
    P = O.LJParams.single()
    G = np.random.default_rng(3).normal(size=(w.n, 3))
    gx, ge, gs = sysm.forces_backward(G)
    gx_ref, ge_ref, gs_ref = O.lj_force_grad(w.pos, w.box, P, G, w.species)
    ae, as_ = O.lj_force_grad_scale(w.pos, w.box, P, G, w.species)
    assert vec_error(gx, gx_ref) <= TOL["mixed"]
    for t, tref, scale in [(ge, ge_ref, ae), (gs, gs_ref, as_)]:
        assert np.all(np.abs(t - tref) <= TOL["mixed"] * scale)

