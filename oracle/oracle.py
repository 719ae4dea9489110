"""ctypes front end of the FP64 CPU oracle (md_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the package smoke check
and the benchmark's CPU-baseline leg, never by the library's product path.
It shares no code with the CUDA library.  build() compiles md_oracle.c with
gcc -O2 -ffp-contract=off so that every floating-point expression in it runs
exactly in the order written.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "md_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile md_oracle.c into _build/liboracle.so (only if the source is newer)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    # OpenMP for the all-cores baseline form; without it the same code runs on one thread
    r = subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        _lib = _configure(C.CDLL(build()))
        return _lib


def _configure(lib):
    """Declare the C signatures of md_oracle.c on a loaded library."""
    lib.orc_neighbor_pairs.restype = C.c_int64
    lib.orc_neighbor_pairs.argtypes = [C.c_int64, _dp, _dp, C.c_double, C.c_int, C.c_int64, C.c_void_p]
    lib.orc_lj_forces.restype = None
    lib.orc_lj_forces.argtypes = [C.c_int64, _dp, _dp, C.c_void_p, C.c_int32, _dp, _dp, _dp,
                                  C.c_int, _dp, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_lj_forces_pairs.restype = None
    lib.orc_lj_forces_pairs.argtypes = [C.c_int64, _dp, _dp, C.c_void_p, C.c_int32, _dp, _dp, _dp,
                                        C.c_int64, _ip, _dp, C.c_void_p, C.c_void_p]
    lib.orc_lj_forces_subset.restype = None
    lib.orc_lj_forces_subset.argtypes = [C.c_int64, _dp, _dp, C.c_void_p, C.c_int32, _dp, _dp, _dp,
                                         C.c_int64, _lp, _dp, C.c_void_p, C.c_void_p]
    lib.orc_kinetic.restype = C.c_double
    lib.orc_kinetic.argtypes = [C.c_int64, _dp, C.c_void_p, _dp]
    lib.orc_lj_grad.restype = None
    lib.orc_lj_grad.argtypes = [C.c_int64, _dp, _dp, C.c_void_p, C.c_int32, _dp, _dp, _dp, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    if hasattr(lib, "orc_lj_grad_abs"):
        lib.orc_lj_grad_abs.restype = None
        lib.orc_lj_grad_abs.argtypes = [C.c_int64, _dp, _dp, C.c_void_p, C.c_int32, _dp, _dp, _dp, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_tbsma_forces.restype = None
    lib.orc_tbsma_forces.argtypes = [C.c_int64, _dp, _dp, _dp, C.c_double, C.c_int, _dp, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p]
    for name in ("orc_run_nve", "orc_run_nve_omp"):
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = C.c_int64
        fn.argtypes = [C.c_int64, _dp, _dp, _ip, _dp, C.c_void_p, C.c_int32, _dp, _dp, _dp,
                       _dp, C.c_double, C.c_double, C.c_int32, C.c_int32, C.c_int64,
                       C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]
    if hasattr(lib, "orc_run_nve_tbsma"):
        lib.orc_run_nve_tbsma.restype = C.c_int64
        lib.orc_run_nve_tbsma.argtypes = [C.c_int64, _dp, _dp, _ip, _dp, _dp, C.c_double, C.c_double, C.c_double,
                                          C.c_double, C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p]
    if hasattr(lib, "orc_lj_forces_full_omp"):
        lib.orc_lj_forces_full_omp.restype = C.c_int32
        lib.orc_lj_forces_full_omp.argtypes = [C.c_int64, _dp, _dp, C.c_void_p, C.c_int32, _dp, _dp, _dp, _dp,
                                               C.c_void_p]
        lib.orc_threads.restype = C.c_int32
        lib.orc_threads.argtypes = []
    return lib


def build_variant(source_text: str, tag: str) -> str:
    """Compile a modified copy of md_oracle.c (used by the mutation tests)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    src = os.path.join(_OUT_DIR, f"variant_{tag}.c")
    lib = os.path.join(_OUT_DIR, f"libvariant_{tag}.so")
    with open(src, "w") as fh:
        fh.write(source_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", src, "-o", lib, "-lm"], check=True)
    return lib


class use_library:
    """Context manager: route this module's calls to another compiled oracle."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        _lib = _configure(C.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


class LJParams:
    """Pair parameters of an n-species Lennard-Jones model (symmetric n x n tables)."""

    def __init__(self, eps, sig, rc, mass):
        self.eps = np.ascontiguousarray(np.atleast_2d(np.asarray(eps, dtype=np.float64)))
        self.sig = np.ascontiguousarray(np.atleast_2d(np.asarray(sig, dtype=np.float64)))
        self.rc = np.ascontiguousarray(np.atleast_2d(np.asarray(rc, dtype=np.float64)))
        self.mass = np.ascontiguousarray(np.atleast_1d(np.asarray(mass, dtype=np.float64)))
        self.nsp = int(self.mass.shape[0])

    @staticmethod
    def single(eps=1.0, sig=1.0, rc=2.5, mass=1.0) -> "LJParams":
        return LJParams([[eps]], [[sig]], [[rc]], [mass])


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _sp(species):
    if species is None:
        return None
    s = _c(species, np.int32)
    return s, s.ctypes.data


def neighbor_pairs(pos, box, r_list, brute=False):
    """Sorted (P, 2) int32 array of pairs i < j with minimum-image distance < r_list."""
    lib = _load()
    pos = _c(pos, np.float64)
    box = _c(box, np.float64)
    n = pos.shape[0]
    cnt = lib.orc_neighbor_pairs(n, pos.ravel(), box, float(r_list), int(brute), 0, None)
    out = np.empty((max(cnt, 1), 2), dtype=np.int32)
    cnt2 = lib.orc_neighbor_pairs(n, pos.ravel(), box, float(r_list), int(brute), cnt, out.ctypes.data)
    assert cnt2 == cnt
    return out[:cnt]


def lj_forces(pos, box, params: LJParams, species=None, brute=False, per_atom=False):
    """(F (N,3), PE, virial[6]) of the whole system; with per_atom also PE per atom."""
    lib = _load()
    pos = _c(pos, np.float64)
    box = _c(box, np.float64)
    n = pos.shape[0]
    f = np.zeros((n, 3))
    pe = np.zeros(1)
    vir = np.zeros(6)
    pea = np.zeros(n) if per_atom else None
    sp = _sp(species)
    lib.orc_lj_forces(n, pos.ravel(), box, sp[1] if sp else None, params.nsp, params.eps.ravel(),
                      params.sig.ravel(), params.rc.ravel(), int(brute), f.ravel(),
                      pea.ctypes.data if pea is not None else None, pe.ctypes.data, vir.ctypes.data)
    if per_atom:
        return f, float(pe[0]), vir, pea
    return f, float(pe[0]), vir


class TBSMAParams:
    """Tight-binding second-moment potential of Cleri and Rosato (1993): A, xi (energy),
    p, q (dimensionless), r0 (nearest-neighbour distance) and the cutoff r_cut."""

    def __init__(self, A, xi, p, q, r0, rc):
        self.A, self.xi, self.p, self.q, self.r0, self.rc = (float(v) for v in (A, xi, p, q, r0, rc))

    def array(self):
        return np.array([self.A, self.xi, self.p, self.q, self.r0])

    @staticmethod
    def copper(rc=None):
        """Cu of Cleri and Rosato (eV, Angstrom): fitted to the fcc lattice constant 3.615 A and
        cohesive energy 3.544 eV with sums over five neighbour shells; the default cutoff lies
        halfway between the fifth and sixth shells, sqrt(5) r0 and sqrt(6) r0."""
        r0 = 3.615 / np.sqrt(2.0)
        return TBSMAParams(0.0855, 1.224, 10.960, 2.278, r0,
                           rc if rc is not None else 0.5 * (np.sqrt(5.0) + np.sqrt(6.0)) * r0)


def tbsma_forces(pos, box, params: TBSMAParams, brute=False, per_atom=False):
    """(F (N,3), E, virial[6]) of the whole system; with per_atom also (rho, E per atom)."""
    lib = _load()
    pos = _c(pos, np.float64)
    box = _c(box, np.float64)
    n = pos.shape[0]
    f = np.zeros((n, 3))
    e = np.zeros(1)
    vir = np.zeros(6)
    rho = np.zeros(n) if per_atom else None
    ea = np.zeros(n) if per_atom else None
    lib.orc_tbsma_forces(n, pos.ravel(), box, params.array(), params.rc, int(brute), f.ravel(),
                         rho.ctypes.data if per_atom else None, ea.ctypes.data if per_atom else None,
                         e.ctypes.data, vir.ctypes.data)
    if per_atom:
        return f, float(e[0]), vir, rho, ea
    return f, float(e[0]), vir


def lj_force_grad(pos, box, params: LJParams, G, species=None):
    """Reverse-mode derivatives of a scalar L(F) with dL/dF = G (N,3): returns
    (dL/dx (N,3), dL/deps (nsp,nsp), dL/dsig (nsp,nsp)) over the pairs inside their cutoffs
    (pair set held fixed).  Symmetric tables: entry [a][b] = [b][a] is the derivative with
    respect to the shared value of the species pair {a,b}."""
    lib = _load()
    pos = _c(pos, np.float64)
    box = _c(box, np.float64)
    G = _c(G, np.float64)
    n = pos.shape[0]
    gx = np.zeros((n, 3))
    ge = np.zeros((params.nsp, params.nsp))
    gs = np.zeros((params.nsp, params.nsp))
    sp = _sp(species)
    lib.orc_lj_grad(n, pos.ravel(), box, sp[1] if sp else None, params.nsp, params.eps.ravel(), params.sig.ravel(),
                    params.rc.ravel(), G.ctypes.data, gx.ctypes.data, ge.ctypes.data, gs.ctypes.data, None, None)
    return gx, ge, gs


def lj_force_grad_scale(pos, box, params: LJParams, G, species=None):
    """Sum over the pairs of |term| of dL/deps and dL/dsig (the tables of lj_force_grad):
    the scale that bounds the error of those sums when every term has a relative error."""
    lib = _load()
    pos = _c(pos, np.float64)
    box = _c(box, np.float64)
    G = _c(G, np.float64)
    n = pos.shape[0]
    scratch = np.zeros((n, 3))
    ge = np.zeros((params.nsp, params.nsp))
    gs = np.zeros((params.nsp, params.nsp))
    sp = _sp(species)
    lib.orc_lj_grad_abs(n, pos.ravel(), box, sp[1] if sp else None, params.nsp, params.eps.ravel(),
                        params.sig.ravel(), params.rc.ravel(), G.ctypes.data, scratch.ctypes.data, ge.ctypes.data,
                        gs.ctypes.data)
    return ge, gs


def lj_energy_param_grad(pos, box, params: LJParams, species=None):
    """(dE/deps, dE/dsig) as (nsp,nsp) tables (same convention as lj_force_grad)."""
    lib = _load()
    pos = _c(pos, np.float64)
    box = _c(box, np.float64)
    n = pos.shape[0]
    de = np.zeros((params.nsp, params.nsp))
    ds = np.zeros((params.nsp, params.nsp))
    sp = _sp(species)
    lib.orc_lj_grad(n, pos.ravel(), box, sp[1] if sp else None, params.nsp, params.eps.ravel(), params.sig.ravel(),
                    params.rc.ravel(), None, None, None, None, de.ctypes.data, ds.ctypes.data)
    return de, ds


def lj_forces_pairs(pos, box, params: LJParams, pairs, species=None):
    """(F, PE, virial) from an explicit pair set (each unordered pair once)."""
    lib = _load()
    pos = _c(pos, np.float64)
    box = _c(box, np.float64)
    pairs = _c(pairs, np.int32)
    n = pos.shape[0]
    f = np.zeros((n, 3))
    pe = np.zeros(1)
    vir = np.zeros(6)
    sp = _sp(species)
    lib.orc_lj_forces_pairs(n, pos.ravel(), box, sp[1] if sp else None, params.nsp, params.eps.ravel(),
                            params.sig.ravel(), params.rc.ravel(), pairs.shape[0], pairs.ravel(),
                            f.ravel(), pe.ctypes.data, vir.ctypes.data)
    return f, float(pe[0]), vir


def lj_forces_subset(pos, box, params: LJParams, idx, species=None):
    """(F (m,3), PE share (m,), virial share (m,6)) on the atoms idx, by direct summation."""
    lib = _load()
    pos = _c(pos, np.float64)
    box = _c(box, np.float64)
    idx = _c(idx, np.int64)
    n = pos.shape[0]
    m = idx.shape[0]
    f = np.zeros((m, 3))
    pe = np.zeros(m)
    vir = np.zeros((m, 6))
    sp = _sp(species)
    lib.orc_lj_forces_subset(n, pos.ravel(), box, sp[1] if sp else None, params.nsp, params.eps.ravel(),
                             params.sig.ravel(), params.rc.ravel(), m, idx, f.ravel(),
                             pe.ctypes.data, vir.ctypes.data)
    return f, pe, vir


def kinetic(vel, params: LJParams, species=None) -> float:
    lib = _load()
    vel = _c(vel, np.float64)
    sp = _sp(species)
    return float(lib.orc_kinetic(vel.shape[0], vel.ravel(), sp[1] if sp else None, params.mass))


def run_nve(pos, vel, box, params: LJParams, dt, skin, nsteps, species=None, image=None,
            policy=0, every_k=10, history=False, forces=None, all_cores=False):
    """Velocity-Verlet run; returns dict(pos, vel, image, rebuilds, forces[, pe, ke]).

    forces: the forces at pos (from an earlier run's result), used instead of evaluating
    them again, so that a run of k steps evaluates the forces exactly k times.
    all_cores: the full-sum forces of orc_lj_forces_full_omp on every host core."""
    lib = _load()
    x = _c(pos, np.float64).copy()
    v = _c(vel, np.float64).copy()
    n = x.shape[0]
    img = np.zeros((n, 3), dtype=np.int32) if image is None else _c(image, np.int32).copy()
    box = _c(box, np.float64)
    sp = _sp(species)
    pe_h = np.zeros(nsteps) if history else None
    ke_h = np.zeros(nsteps) if history else None
    f = np.zeros((n, 3)) if forces is None else _c(forces, np.float64).copy()
    fn = lib.orc_run_nve_omp if all_cores else lib.orc_run_nve
    nreb = fn(n, x.ravel(), v.ravel(), img.ravel(), box, sp[1] if sp else None, params.nsp,
              params.eps.ravel(), params.sig.ravel(), params.rc.ravel(), params.mass,
              float(dt), float(skin), int(policy), int(every_k), int(nsteps),
              f.ctypes.data, 0 if forces is None else 1,
              pe_h.ctypes.data if history else None, ke_h.ctypes.data if history else None)
    out = dict(pos=x, vel=v, image=img, rebuilds=int(nreb), forces=f)
    if history:
        out["pe"] = pe_h
        out["ke"] = ke_h
    return out


def run_nve_tbsma(pos, vel, box, params: "TBSMAParams", mass, dt, skin, nsteps, image=None,
                  policy=0, every_k=10, history=False):
    """Velocity-Verlet run with the many-body TB-SMA forces (one species of the given mass);
    returns dict(pos, vel, image, rebuilds[, pe, ke])."""
    lib = _load()
    x = _c(pos, np.float64).copy()
    v = _c(vel, np.float64).copy()
    n = x.shape[0]
    img = np.zeros((n, 3), dtype=np.int32) if image is None else _c(image, np.int32).copy()
    box = _c(box, np.float64)
    pe_h = np.zeros(nsteps) if history else None
    ke_h = np.zeros(nsteps) if history else None
    nreb = lib.orc_run_nve_tbsma(n, x.ravel(), v.ravel(), img.ravel(), box, params.array(), float(params.rc),
                                 float(mass), float(dt), float(skin), int(policy), int(every_k), int(nsteps),
                                 pe_h.ctypes.data if history else None, ke_h.ctypes.data if history else None)
    out = dict(pos=x, vel=v, image=img, rebuilds=int(nreb))
    if history:
        out["pe"] = pe_h
        out["ke"] = ke_h
    return out


def lj_forces_all_cores(pos, box, params: LJParams, species=None):
    """Forces and potential energy by full neighbour sums on every host core
    (orc_lj_forces_full_omp); returns (forces, pe, threads used)."""
    lib = _load()
    pos = _c(pos, np.float64)
    n = pos.shape[0]
    box = _c(box, np.float64)
    f = np.zeros((n, 3))
    pe = np.zeros(1)
    sp = _sp(species)
    th = lib.orc_lj_forces_full_omp(n, pos.ravel(), box, sp[1] if sp else None, params.nsp, params.eps.ravel(),
                                    params.sig.ravel(), params.rc.ravel(), f.ravel(), pe.ctypes.data)
    return f, float(pe[0]), int(th)


def threads() -> int:
    """Host threads the all-cores form uses."""
    return int(_load().orc_threads())
