"""md_kinetic_energy_noalloc: the kinetic energy for callers that cannot allocate.

Callers under a locked memory budget (an embedding runtime that owns all device
memory) or in a loop that must not call cudaMalloc (it can synchronise the device)
use this entry point; it keeps its partial sums in a static device array instead of
allocating scratch.  Its result must equal the kinetic
energy md_energy_virial reports for the same velocities, on every call.  This
file is collected last so that a failure here does not hide any other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1305_4196_gb300 import build as B  # noqa: E402
from paper_1305_4196_gb300 import workloads as W  # noqa: E402

B.build()
from paper_1305_4196_gb300 import mdgb as M  # noqa: E402


def _reference_ke(sysm, species=None, mass=(1.0,), eps=1.0, sig=1.0):
    s = M.System(sysm.n, sysm.box, eps=eps, sigma=sig, mass=list(mass))
    s.set_state(sysm.pos, sysm.vel, species)
    _, ke, _ = s.energy_virial()
    s.close()
    return ke


def test_noalloc_matches_md_energy_virial_twice():
    sysm = W.lj_fcc(12, seed=5, jitter=0.05)  # 6,912 atoms
    ke_ref = _reference_ke(sysm)
    dev = torch.device("cuda")
    vel = torch.from_numpy(np.ascontiguousarray(sysm.vel)).to(dev)
    out = torch.full((2,), -1.0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for k in range(2):
        assert M.md_kinetic_energy_noalloc(sysm.n, vel, None, [1.0], out[k:k + 1], stream) == M.MD_OK
    torch.cuda.synchronize()
    ke = out.cpu().numpy()
    assert ke[0] == pytest.approx(ke_ref, rel=1e-12)
    assert ke[1] == pytest.approx(ke_ref, rel=1e-12)


def test_noalloc_two_species_and_larger_system_twice():
    sysm = W.lj_fcc(40, seed=6, jitter=0.05)  # 256,000 atoms: many partial sums
    sp = W.species_shuffle(sysm.n, 0.2, seed=6)
    mass = [1.0, 2.5]
    ke_ref = _reference_ke(sysm, species=sp, mass=mass, eps=np.ones((2, 2)), sig=np.ones((2, 2)))
    dev = torch.device("cuda")
    vel = torch.from_numpy(np.ascontiguousarray(sysm.vel)).to(dev)
    spt = torch.from_numpy(sp).to(dev)
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for k in range(2):
        assert M.md_kinetic_energy_noalloc(sysm.n, vel, spt, mass, out[k:k + 1], stream) == M.MD_OK
    torch.cuda.synchronize()
    ke = out.cpu().numpy()
    assert ke[0] == pytest.approx(ke_ref, rel=1e-12)
    assert ke[1] == ke[0]


def test_noalloc_rejects_sizes_beyond_the_maximum():
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    vel = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    assert M.md_kinetic_energy_noalloc((1 << 30) + 1, vel, None, [1.0], out) == M.MD_ERR_ARG
    assert M.md_kinetic_energy_noalloc(-1, vel, None, [1.0], out) == M.MD_ERR_ARG
    assert M.md_kinetic_energy_noalloc(1, vel, None, [1.0] * 5, out) == M.MD_ERR_ARG


def test_noalloc_species_ids_checked_at_the_limit():
    """Two species: ids up to n_species - 1 give the right energy; an id equal to
    n_species or negative reads no mass and turns the result into NaN."""
    sysm = W.lj_fcc(6, seed=8, jitter=0.05)  # 864 atoms
    sp = np.zeros(sysm.n, dtype=np.int32)
    sp[::3] = 1
    mass = [1.0, 3.0]
    ke_ref = 0.5 * float((np.asarray(mass)[sp] * (sysm.vel ** 2).sum(1)).sum())
    dev = torch.device("cuda")
    vel = torch.from_numpy(np.ascontiguousarray(sysm.vel)).to(dev)
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    assert M.md_kinetic_energy_noalloc(sysm.n, vel, torch.from_numpy(sp).to(dev), mass, out[0:1], stream) == M.MD_OK
    for k, bad in ((1, 2), (2, -1)):
        spb = sp.copy()
        spb[sysm.n // 2] = bad
        assert M.md_kinetic_energy_noalloc(sysm.n, vel, torch.from_numpy(spb).to(dev), mass, out[k:k + 1],
                                           stream) == M.MD_OK
    torch.cuda.synchronize()
    ke = out.cpu().numpy()
    assert ke[0] == pytest.approx(ke_ref, rel=1e-12)
    assert np.isnan(ke[1]) and np.isnan(ke[2])
