"""Python binding of the mdgb C ABI (include/mdgb.h).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels behind libmdgb.so.  Functions keep the C names (md_create,
md_set_state, md_bin_cells, md_build_neighbors, md_forces, md_step,
md_energy_virial, md_get_state, md_get_neighbors, md_get_cells,
md_get_info, md_last_error, md_destroy) and accept numpy arrays (host
pointers) or torch CUDA tensors (device pointers).

Importing this module loads the library and raises if it is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MD_OK = 0
MD_ERR_ARG = -1
MD_ERR_BOX_TOO_SMALL = -2
MD_ERR_CELL_OVERFLOW = -3
MD_ERR_LIST_OVERFLOW = -4
MD_ERR_NONFINITE = -5
MD_ERR_SKIN_VIOLATION = -6
MD_ERR_CUDA = -7
MD_ERR_TIMEOUT = -8
MD_ERR_STATE = -9

MD_FP64 = 0
MD_MIXED = 1
MD_LIST_FULL = 0
MD_LIST_HALF_COLOUR8 = 1
MD_LIST_HALF_ATOMIC_FREE = 2
MD_REBUILD_SKIN_HALF = 0
MD_REBUILD_EVERY_K = 1

EXPORTED = ["md_create", "md_set_state", "md_bin_cells", "md_build_neighbors", "md_forces", "md_step",
            "md_energy_virial", "md_get_state", "md_get_neighbors", "md_get_cells", "md_get_info",
            "md_set_timing", "md_last_error", "md_destroy", "md_kinetic_energy_noalloc", "md_set_params",
            "md_forces_backward", "md_energy_param_grad", "md_set_tbsma", "md_colour_conflicts"]


class md_params(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("eps", C.POINTER(C.c_double)), ("sigma", C.POINTER(C.c_double)),
                ("rcut", C.POINTER(C.c_double)), ("mass", C.POINTER(C.c_double)), ("dt", C.c_double),
                ("precision", C.c_int32), ("list_kind", C.c_int32), ("rebuild", C.c_int32),
                ("rebuild_k", C.c_int32), ("stream", C.c_void_p)]


class md_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("ncell", C.c_int32 * 3), ("list_cap", C.c_int32), ("tile_cap", C.c_int32),
                ("n_builds", C.c_int64), ("n_steps", C.c_int64), ("list_entries", C.c_int64),
                ("max_list", C.c_int32), ("max_tile", C.c_int32), ("cell_width", C.c_double * 3),
                ("kernel_launches", C.c_int64), ("force_evals", C.c_int64), ("force_ms", C.c_double),
                ("timed_force_evals", C.c_int64), ("build_ms", C.c_double), ("timed_builds", C.c_int64),
                ("n_redos", C.c_int64)]


class MDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mdgb error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libmdgb.so is not built ({path}); run paper_1305_4196_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.md_create.argtypes = [C.c_int64, P, C.c_double, C.c_double, C.POINTER(md_params), C.POINTER(P)]
    lib.md_set_state.argtypes = [P, P, P, P, C.c_int]
    lib.md_bin_cells.argtypes = [P]
    lib.md_build_neighbors.argtypes = [P]
    lib.md_forces.argtypes = [P, P, C.c_int]
    lib.md_step.argtypes = [P, C.c_int32]
    lib.md_energy_virial.argtypes = [P, P, P, P]
    lib.md_get_state.argtypes = [P, P, P, P, C.c_int]
    lib.md_get_neighbors.argtypes = [P, C.POINTER(C.c_int64), P]
    lib.md_get_cells.argtypes = [P, P]
    lib.md_get_info.argtypes = [P, C.POINTER(md_info)]
    lib.md_set_timing.argtypes = [P, C.c_int]
    lib.md_kinetic_energy_noalloc.argtypes = [C.c_int64, P, P, C.POINTER(C.c_double), C.c_int32, P, P]
    lib.md_set_params.argtypes = [P, P, P, P]
    lib.md_forces_backward.argtypes = [P, P, C.c_int, P, P, P]
    lib.md_energy_param_grad.argtypes = [P, P, P]
    lib.md_set_tbsma.argtypes = [P] + [C.c_double] * 6
    lib.md_colour_conflicts.argtypes = [P, C.c_int32, C.POINTER(C.c_int64)]
    lib.md_last_error.argtypes = [P, C.c_char_p, C.c_int64]
    lib.md_destroy.argtypes = [P]
    lib.md_destroy.restype = None
    for name in EXPORTED:
        if name != "md_destroy":
            getattr(lib, name).restype = C.c_int
    return lib


_lib = _load()


def _ptr(a, dtype=None, count=None, name="array"):
    """(pointer, is_device) of a numpy array or torch tensor (None -> NULL).

    The C calls read or write a fixed number of elements of one type through the pointer,
    so the array must be contiguous, of element type `dtype` (a numpy dtype, when given)
    and hold at least `count` elements (when given); anything else raises before the call.
    """
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name} must be C-contiguous")
        kind, size, dev = a.dtype.name, a.size, False
        ptr = a.ctypes.data
    elif hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        kind, size, dev = str(a.dtype).replace("torch.", ""), a.numel(), bool(a.is_cuda)
        ptr = a.data_ptr()
    else:
        raise TypeError(f"unsupported array type {type(a)}")
    if dtype is not None and kind != np.dtype(dtype).name:
        raise TypeError(f"{name} must be {np.dtype(dtype).name}, not {kind}")
    if count is not None and size < count:
        raise ValueError(f"{name} holds {size} elements, the call uses {count}")
    return ptr, dev


def _same_side(*ptrs):
    """The one host/device flag of a call's arrays (None if all are NULL); a mix raises."""
    devs = {d for _, d in ptrs if d is not None}
    if len(devs) > 1:
        raise ValueError("mix of host and device arrays")
    return devs.pop() if devs else None


def _n_atoms(handle) -> int:
    info = md_info()
    _check(handle, _lib.md_get_info(handle, C.byref(info)))
    return int(info.n)


def _check(handle, code):
    if code != MD_OK:
        raise MDError(code, md_last_error(handle))


def md_last_error(handle) -> str:
    buf = C.create_string_buffer(512)
    _lib.md_last_error(handle, buf, 512)
    return buf.value.decode(errors="replace")


def md_create(n, box, r_cut, skin, eps, sigma, mass, dt, precision=MD_MIXED, list_kind=MD_LIST_FULL,
              rebuild=MD_REBUILD_SKIN_HALF, rebuild_k=10, rcut=None, stream=None):
    """Create a system; eps/sigma/rcut are n_species x n_species tables, mass has n_species entries."""
    eps = np.ascontiguousarray(np.atleast_2d(eps), dtype=np.float64)
    sigma = np.ascontiguousarray(np.atleast_2d(sigma), dtype=np.float64)
    mass = np.ascontiguousarray(np.atleast_1d(mass), dtype=np.float64)
    rc = None if rcut is None else np.ascontiguousarray(np.atleast_2d(rcut), dtype=np.float64)
    box = np.ascontiguousarray(box, dtype=np.float64)
    if box.shape != (3,):
        raise ValueError("box must hold the 3 sides")
    nsp = int(mass.shape[0])
    for name, table in (("eps", eps), ("sigma", sigma), ("rcut", rc)):
        if table is not None and table.size != nsp * nsp:
            raise ValueError(f"{name} must be an n_species x n_species table ({nsp} species)")
    dp = C.POINTER(C.c_double)
    p = md_params(int(mass.shape[0]), eps.ctypes.data_as(dp), sigma.ctypes.data_as(dp),
                  rc.ctypes.data_as(dp) if rc is not None else None, mass.ctypes.data_as(dp), float(dt),
                  int(precision), int(list_kind), int(rebuild), int(rebuild_k),
                  C.c_void_p(stream) if stream else None)
    out = C.c_void_p()
    code = _lib.md_create(int(n), box.ctypes.data, float(r_cut), float(skin), C.byref(p), C.byref(out))
    if code != MD_OK:
        raise MDError(code, "md_create failed")
    return out


def md_set_state(handle, pos, vel, species=None):
    n = _n_atoms(handle)
    args = (_ptr(pos, np.float64, 3 * n, "pos"), _ptr(vel, np.float64, 3 * n, "vel"),
            _ptr(species, np.int32, n, "species"))
    dev = _same_side(*args)
    _check(handle, _lib.md_set_state(handle, args[0][0], args[1][0], args[2][0], int(bool(dev))))


def md_bin_cells(handle):
    _check(handle, _lib.md_bin_cells(handle))


def md_build_neighbors(handle):
    _check(handle, _lib.md_build_neighbors(handle))


def md_forces(handle, f_out=None):
    fp, dev = _ptr(f_out, np.float64, 3 * _n_atoms(handle) if f_out is not None else None, "f_out")
    _check(handle, _lib.md_forces(handle, fp, int(bool(dev))))


def md_step(handle, n_steps):
    _check(handle, _lib.md_step(handle, int(n_steps)))


def md_energy_virial(handle):
    pe, ke = C.c_double(), C.c_double()
    vir = (C.c_double * 6)()
    _check(handle, _lib.md_energy_virial(handle, C.byref(pe), C.byref(ke), vir))
    return pe.value, ke.value, np.array(vir[:])


def md_get_state(handle, pos=None, vel=None, image=None):
    n = _n_atoms(handle)
    args = (_ptr(pos, np.float64, 3 * n, "pos"), _ptr(vel, np.float64, 3 * n, "vel"),
            _ptr(image, np.int32, 3 * n, "image"))
    dev = _same_side(*args)
    _check(handle, _lib.md_get_state(handle, args[0][0], args[1][0], args[2][0], int(bool(dev))))


def md_get_neighbors(handle):
    cnt = C.c_int64()
    _check(handle, _lib.md_get_neighbors(handle, C.byref(cnt), None))
    out = np.empty((max(cnt.value, 1), 2), dtype=np.int32)
    _check(handle, _lib.md_get_neighbors(handle, C.byref(cnt), out.ctypes.data))
    return out[:cnt.value]


def md_get_cells(handle, n):
    out = np.empty(int(n), dtype=np.int32)
    _check(handle, _lib.md_get_cells(handle, out.ctypes.data))
    return out


def md_get_info(handle) -> dict:
    info = md_info()
    _check(handle, _lib.md_get_info(handle, C.byref(info)))
    return {"n": info.n, "ncell": list(info.ncell), "list_cap": info.list_cap, "tile_cap": info.tile_cap,
            "n_builds": info.n_builds, "n_steps": info.n_steps, "list_entries": info.list_entries,
            "max_list": info.max_list, "max_tile": info.max_tile, "cell_width": list(info.cell_width),
            "kernel_launches": info.kernel_launches, "force_evals": info.force_evals, "force_ms": info.force_ms,
            "timed_force_evals": info.timed_force_evals, "build_ms": info.build_ms,
            "timed_builds": info.timed_builds, "n_redos": info.n_redos}


def md_set_timing(handle, enable=True):
    _check(handle, _lib.md_set_timing(handle, int(bool(enable))))


def md_kinetic_energy_noalloc(n, vel, species, mass, ke_out, stream=None):
    """Kinetic energy of device velocities into the device scalar ke_out, with no device
    allocation (see include/mdgb.h); returns the C status code."""
    mass = np.ascontiguousarray(np.atleast_1d(mass), dtype=np.float64)
    n = int(n)
    m = n if 0 < n <= 1 << 30 else None  # outside that range the call reads nothing
    vp, _ = _ptr(vel, np.float64, 3 * m if m else None, "vel")
    sp, _ = _ptr(species, np.int32, m, "species")
    op, _ = _ptr(ke_out, np.float64, 1, "ke_out")
    return _lib.md_kinetic_energy_noalloc(int(n), vp, sp, mass.ctypes.data_as(C.POINTER(C.c_double)),
                                          int(mass.shape[0]), op, C.c_void_p(stream) if stream else None)


def md_set_params(handle, eps, sigma, rcut=None, nsp=None):
    """New pair tables (n_species x n_species); nsp, when given, is checked against their size."""
    eps = np.ascontiguousarray(np.atleast_2d(eps), dtype=np.float64)
    sigma = np.ascontiguousarray(np.atleast_2d(sigma), dtype=np.float64)
    rc = None if rcut is None else np.ascontiguousarray(np.atleast_2d(rcut), dtype=np.float64)
    for name, table in (("eps", eps), ("sigma", sigma), ("rcut", rc)):
        if nsp is not None and table is not None and table.size != nsp * nsp:
            raise ValueError(f"{name} must be an n_species x n_species table ({nsp} species)")
    _check(handle, _lib.md_set_params(handle, eps.ctypes.data, sigma.ctypes.data,
                                      rc.ctypes.data if rc is not None else None))


def md_set_tbsma(handle, A, xi, p, q, r0, r_cut):
    _check(handle, _lib.md_set_tbsma(handle, float(A), float(xi), float(p), float(q), float(r0), float(r_cut)))


def md_forces_backward(handle, grad_f, grad_pos, nsp):
    """dL/dx into grad_pos (same kind of array as grad_f: numpy or CUDA tensor, N x 3) and
    (dL/deps, dL/dsigma) returned as nsp x nsp numpy tables."""
    n = _n_atoms(handle)
    (gp, dev), (op, dev2) = _ptr(grad_f, np.float64, 3 * n, "grad_f"), _ptr(grad_pos, np.float64, 3 * n, "grad_pos")
    if grad_pos is not None and bool(dev) != bool(dev2):
        raise ValueError("grad_f and grad_pos must both be host or both be device arrays")
    ge = np.zeros((nsp, nsp))
    gs = np.zeros((nsp, nsp))
    _check(handle, _lib.md_forces_backward(handle, gp, int(bool(dev)), op, ge.ctypes.data, gs.ctypes.data))
    return ge, gs


def md_energy_param_grad(handle, nsp):
    de = np.zeros((nsp, nsp))
    ds = np.zeros((nsp, nsp))
    _check(handle, _lib.md_energy_param_grad(handle, de.ctypes.data, ds.ctypes.data))
    return de, ds


def md_destroy(handle):
    _lib.md_destroy(handle)


class System:
    """Owning wrapper around one md_system handle (destroyed with the object)."""

    def __init__(self, n, box, r_cut=2.5, skin=0.3, eps=1.0, sigma=1.0, mass=1.0, dt=0.005,
                 precision=MD_MIXED, list_kind=MD_LIST_FULL, rebuild=MD_REBUILD_SKIN_HALF, rebuild_k=10,
                 rcut=None, stream=None):
        self.n = int(n)
        self.nsp = int(np.atleast_1d(mass).shape[0])
        self.handle = md_create(n, box, r_cut, skin, eps, sigma, mass, dt, precision, list_kind, rebuild,
                                rebuild_k, rcut, stream)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            md_destroy(h)
            self.handle = None

    def close(self):
        self.__del__()

    def set_state(self, pos, vel, species=None):
        md_set_state(self.handle, pos, vel, species)

    def bin_cells(self):
        md_bin_cells(self.handle)

    def build_neighbors(self):
        md_build_neighbors(self.handle)

    def forces(self, out=None):
        if out is None:
            out = np.empty((self.n, 3))
        md_forces(self.handle, out)
        return out

    def step(self, n_steps):
        md_step(self.handle, n_steps)

    def energy_virial(self):
        return md_energy_virial(self.handle)

    def get_state(self):
        pos, vel, img = np.empty((self.n, 3)), np.empty((self.n, 3)), np.empty((self.n, 3), dtype=np.int32)
        md_get_state(self.handle, pos, vel, img)
        return pos, vel, img

    def neighbors(self):
        return md_get_neighbors(self.handle)

    def cells(self):
        return md_get_cells(self.handle, self.n)

    def info(self):
        return md_get_info(self.handle)

    def set_timing(self, enable=True):
        md_set_timing(self.handle, enable)

    def set_params(self, eps, sigma, rcut=None):
        md_set_params(self.handle, eps, sigma, rcut, self.nsp)

    def colour_conflicts(self, n_phases=8):
        """Atoms claimed by two blocks of one phase (md_colour_conflicts): 0 for the 8 colours."""
        out = C.c_int64()
        _check(self.handle, _lib.md_colour_conflicts(self.handle, int(n_phases), C.byref(out)))
        return int(out.value)

    def set_tbsma(self, A, xi, p, q, r0, r_cut):
        """Cleri-Rosato tight-binding second-moment many-body potential (md_set_tbsma)."""
        md_set_tbsma(self.handle, A, xi, p, q, r0, r_cut)

    def forces_backward(self, grad_f, grad_pos=None):
        """(dL/dx, dL/deps, dL/dsigma) for dL/dF = grad_f (see md_forces_backward)."""
        if grad_pos is None:
            grad_pos = np.empty((self.n, 3)) if isinstance(grad_f, np.ndarray) else grad_f.new_empty((self.n, 3))
        ge, gs = md_forces_backward(self.handle, grad_f, grad_pos, self.nsp)
        return grad_pos, ge, gs

    def energy_param_grad(self):
        return md_energy_param_grad(self.handle, self.nsp)
