"""Python binding of the ensemble API (include/mdgb_batch.h): argument marshalling only."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import mdgb as _m

_lib = C.CDLL(_m.library_path())
_P = C.c_void_p
_lib.md_batch_create.argtypes = [C.c_int32, _P, _P, C.c_double, C.c_double, C.POINTER(_m.md_params), C.POINTER(_P)]
_lib.md_batch_set_state.argtypes = [_P, _P, _P, _P, C.c_int]
_lib.md_batch_step.argtypes = [_P, C.c_int32]
_lib.md_batch_forces.argtypes = [_P, _P, C.c_int]
_lib.md_batch_energies.argtypes = [_P, _P, _P]
_lib.md_batch_get_state.argtypes = [_P, _P, _P, _P, C.c_int]
_lib.md_batch_layout.argtypes = [_P, _P, _P, _P]
_lib.md_batch_autotune.argtypes = [_P, C.c_char_p]
_lib.md_batch_set_wait_budget.argtypes = [_P, C.c_int64, C.c_int32]
_lib.md_batch_last_error.argtypes = [_P, C.c_char_p, C.c_int64]
_lib.md_batch_destroy.argtypes = [_P]
_lib.md_batch_destroy.restype = None
for _f in ("md_batch_create", "md_batch_set_state", "md_batch_step", "md_batch_forces", "md_batch_energies",
           "md_batch_get_state", "md_batch_layout", "md_batch_autotune", "md_batch_last_error",
           "md_batch_set_wait_budget"):
    getattr(_lib, _f).restype = C.c_int


class Batch:
    """An ensemble of independent periodic LJ systems (one species, mixed precision)."""

    def __init__(self, n_atoms, boxes, r_cut=2.5, skin=0.3, eps=1.0, sigma=1.0, mass=1.0, dt=0.005, stream=None):
        self.n = np.ascontiguousarray(n_atoms, dtype=np.int64)
        self.nsys = int(self.n.shape[0])
        self.ntot = int(self.n.sum())
        boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(self.nsys, 3)
        self._keep = [np.array([float(eps)]), np.array([float(sigma)]), np.array([float(mass)])]
        dp = C.POINTER(C.c_double)
        p = _m.md_params(1, self._keep[0].ctypes.data_as(dp), self._keep[1].ctypes.data_as(dp), None,
                         self._keep[2].ctypes.data_as(dp), float(dt), _m.MD_MIXED, _m.MD_LIST_FULL,
                         _m.MD_REBUILD_SKIN_HALF, 10, C.c_void_p(stream) if stream else None)
        out = C.c_void_p()
        code = _lib.md_batch_create(self.nsys, self.n.ctypes.data, boxes.ctypes.data, float(r_cut), float(skin),
                                    C.byref(p), C.byref(out))
        if code != _m.MD_OK:
            raise _m.MDError(code, "md_batch_create failed")
        self.handle = out

    def _check(self, code):
        if code != _m.MD_OK:
            buf = C.create_string_buffer(512)
            _lib.md_batch_last_error(self.handle, buf, 512)
            raise _m.MDError(code, buf.value.decode(errors="replace"))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.md_batch_destroy(h)
            self.handle = None

    def close(self):
        self.__del__()

    def set_state(self, pos, vel, species=None):
        args = (_m._ptr(pos, np.float64, 3 * self.ntot, "pos"), _m._ptr(vel, np.float64, 3 * self.ntot, "vel"),
                _m._ptr(species, np.int32, self.ntot, "species"))
        dev = _m._same_side(*args)
        self._check(_lib.md_batch_set_state(self.handle, args[0][0], args[1][0], args[2][0], int(bool(dev))))

    def step(self, n_steps):
        self._check(_lib.md_batch_step(self.handle, int(n_steps)))

    def forces(self, out=None):
        if out is None:
            out = np.empty((self.ntot, 3))
        fp, dev = _m._ptr(out, np.float64, 3 * self.ntot, "out")
        self._check(_lib.md_batch_forces(self.handle, fp, int(bool(dev))))
        return out

    def energies(self):
        pe, ke = np.empty(self.nsys), np.empty(self.nsys)
        self._check(_lib.md_batch_energies(self.handle, pe.ctypes.data, ke.ctypes.data))
        return pe, ke

    def get_state(self):
        pos, vel = np.empty((self.ntot, 3)), np.empty((self.ntot, 3))
        img = np.empty((self.ntot, 3), dtype=np.int32)
        self._check(_lib.md_batch_get_state(self.handle, pos.ctypes.data, vel.ctypes.data, img.ctypes.data, 0))
        return pos, vel, img

    def layout(self):
        path, th, R = (np.empty(self.nsys, dtype=np.int32) for _ in range(3))
        self._check(_lib.md_batch_layout(self.handle, path.ctypes.data, th.ctypes.data, R.ctypes.data))
        return path, th, R

    def autotune(self, cache_path=None):
        self._check(_lib.md_batch_autotune(self.handle, cache_path.encode() if cache_path else None))

    def set_wait_budget(self, budget_cycles=0, held_system=-1):
        self._check(_lib.md_batch_set_wait_budget(self.handle, int(budget_cycles), int(held_system)))


def from_systems(systems, **kw) -> Batch:
    """A Batch for a list of workloads.System, with their state set."""
    b = Batch([s.n for s in systems], np.stack([s.box for s in systems]), **kw)
    b.set_state(np.ascontiguousarray(np.concatenate([s.pos for s in systems])),
                np.ascontiguousarray(np.concatenate([s.vel for s in systems])))
    return b
