"""The mixed path's FP64 decision band around r_cut^2, checked on the CPU.

A pair interacts when |r| < r_cut (Sec. I); the mixed kernels compute r^2 in FP32 and
take the FP64 decision only when the FP32 value lies within r_cut^2 (1 -/+ band).  That
is exact only if the FP32 error never exceeds the band.  Here the kernels' FP32
operations are replayed in numpy, one rounding at a time, for pairs at r_cut (1 -/+ 3e-6)
in many geometries, including the widest cells md_create can pick (close to 2 r_list)
and atoms that drifted skin/2 from where they were binned; the error must stay within
the bound the band is built from (half the band, less the threshold roundings), and
the bound must not be loose by more than a modest factor.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1305_4196_gb300 import build as B

F32 = np.float32


@pytest.fixture(scope="module")
def band_fn():
    B.build()
    lib = C.CDLL(B.LIB)
    f = lib.mdgb_cut_band
    f.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_int32, C.c_double, C.POINTER(C.c_double)]

    def band(frame, w, half_skin, R, rc):
        out = C.c_double()
        assert f(frame, w, half_skin, R, rc, C.byref(out)) == 0
        return out.value
    return band


def fma32(a, b, c):
    # a*b of two floats is exact in FP64; adding c rounds once in FP64, once more to FP32
    # (an FP64 intermediate rounding is ~1e-16 relative, far below what is measured here)
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)


def r2_fp32(d):
    dx, dy, dz = d[:, 0], d[:, 1], d[:, 2]
    return fma32(dz, dz, fma32(dy, dy, (dx * dx).astype(F32)))


def pairs_near_cutoff(rng, n, rc, rel):
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    r = rc * np.sqrt(1.0 + rng.uniform(-rel, rel, size=n))
    return u * r[:, None]


@pytest.mark.parametrize("w_over_rl", [1.0, 1.09, 1.5, 1.98])
@pytest.mark.parametrize("rc", [2.5, 1.1, 5.0])
def test_tile_frame_error_within_bound(band_fn, w_over_rl, rc):
    """md_system's block frame: coordinate = FP32(x - cell centre) + FP32 tile offset
    (t - 3/2) w, summed in FP32; displacement = FP32 difference; r^2 by two FMAs."""
    rng = np.random.default_rng(int(1000 * w_over_rl + 10 * rc))
    skin = 0.3
    w = w_over_rl * (rc + skin)
    n = 200000
    # atom i in one of the block's own cells (tile coordinate 1 or 2), bound to cell ci at
    # the build and since drifted by up to skin/2
    ci = rng.integers(1, 3, size=(n, 3))
    drift = rng.normal(size=(n, 3))
    drift *= (0.5 * skin * rng.uniform(0, 1, size=n) / np.linalg.norm(drift, axis=1))[:, None]
    base = 1000.0 * w  # the block's first tile cell starts here (absolute coordinates)
    xi_build = base + (ci + rng.uniform(0, 1, size=(n, 3))) * w
    xi = xi_build + drift
    xj = xi + pairs_near_cutoff(rng, n, rc, 3e-6)
    # j's build cell: where it was binned (its current position less a drift of up to skin/2)
    dj = rng.normal(size=(n, 3))
    dj *= (0.5 * skin * rng.uniform(0, 1, size=n) / np.linalg.norm(dj, axis=1))[:, None]
    cj = np.floor((xj - dj - base) / w).astype(int)
    ok = np.all((cj >= 0) & (cj <= 3), axis=1)  # inside the 4x4x4 tile
    xi, xj, ci, cj = xi[ok], xj[ok], ci[ok], cj[ok]

    def tile_coord(x, c):
        centre = base + (c + 0.5) * w
        xr = (x - centre).astype(F32)
        off = ((c - 1.5) * w).astype(F32)
        return (xr + off).astype(F32)

    d = (tile_coord(xi, ci) - tile_coord(xj, cj)).astype(F32)
    r2_32 = r2_fp32(d).astype(np.float64)
    r2 = ((xi - xj) ** 2).sum(1)
    rel = np.abs(r2_32 - r2) / rc ** 2
    bound = (band_fn(0, w, 0.5 * skin, 0, rc) - 3.0e-7) / 2.0
    assert ok.sum() > n // 4
    assert rel.max() <= bound, (rel.max(), bound)
    assert rel.max() >= bound / 20.0  # the bound is a worst case, but not a vacuous one


@pytest.mark.parametrize("R", [1, 2])
@pytest.mark.parametrize("w_over_rc", [1.0, 1.45, 1.9])
def test_cell_frame_error_within_bound(band_fn, R, w_over_rc):
    """The ensemble kernel: coordinates relative to the centre of this step's cell, the
    neighbour cell's shift k * FP32(w) added in FP32, FP32 difference, r^2 by two FMAs."""
    rc = 2.5
    w = w_over_rc * rc / R
    rng = np.random.default_rng(7 + R + int(10 * w_over_rc))
    n = 200000
    ci = rng.integers(0, 40, size=(n, 3))
    xi = (ci + rng.uniform(0, 1, size=(n, 3))) * w
    xj = xi + pairs_near_cutoff(rng, n, rc, 3e-6)
    cj = np.floor(xj / w).astype(int)
    k = cj - ci
    ok = np.all(np.abs(k) <= R, axis=1)
    xi, xj, ci, cj, k = xi[ok], xj[ok], ci[ok], cj[ok], k[ok]
    wf = F32(w)
    pi = (xi - (ci + 0.5) * w).astype(F32)
    pj = (xj - (cj + 0.5) * w).astype(F32)
    shift = (k.astype(F32) * wf).astype(F32)
    d = (pi - (pj + shift).astype(F32)).astype(F32)
    rel = np.abs(r2_fp32(d).astype(np.float64) - ((xi - xj) ** 2).sum(1)) / rc ** 2
    bound = (band_fn(1, w, 0.0, R, rc) - 3.0e-7) / 2.0
    assert ok.sum() > n // 4
    assert rel.max() <= bound, (rel.max(), bound)
    assert rel.max() >= bound / 20.0


def test_band_grows_with_the_cell_width(band_fn):
    b = [band_fn(0, w, 0.15, 0, 2.5) for w in (2.8, 4.0, 5.6)]
    assert b[0] <= b[1] <= b[2]
    assert 1e-6 < b[0] < 1e-5
