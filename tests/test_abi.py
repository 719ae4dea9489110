"""The C-ABI boundary on the CPU: exports, struct layout, argument errors, colour schedule.

No compute call is made here (there is no GPU in the CPU suite); md_create
is only driven into the argument checks that fail before any CUDA call.
"""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1305_4196_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_1305_4196_gb300 import mdgb
    return mdgb


def _declared():
    names = []
    for h in sorted(os.listdir(INCLUDE)):
        if h.endswith(".h"):
            txt = open(os.path.join(INCLUDE, h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:int64_t|int|void)\s+\**\s*(md\w+)\s*\(", txt, flags=re.M)
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 13
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in lib.EXPORTED:
        assert n in names


@pytest.mark.parametrize("compiler", [["gcc", "-std=c99"], ["g++", "-std=c++17", "-x", "c++"]])
def test_headers_compile_as_strict_c_and_cxx(compiler):
    """Every public header, alone and all together, is valid pedantic C99 and C++17 with no
    warning: a C caller needs no CUDA or C++ header to use the library."""
    import tempfile
    headers = sorted(h for h in os.listdir(INCLUDE) if h.endswith(".h"))
    with tempfile.TemporaryDirectory() as d:
        for name, body in [(h, f'#include "{h}"\n') for h in headers] + \
                [("all", "".join(f'#include "{h}"\n' for h in headers))]:
            src = os.path.join(d, name.replace(".h", "") + ".c")
            open(src, "w").write(body)
            subprocess.run(compiler + ["-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only", "-I", INCLUDE,
                                       src], check=True)


def test_plain_c_caller(lib):
    """A C program links libmdgb.so with no Python in between: it gets an argument error from
    md_create (before any CUDA call, so no GPU is needed) and computes the wave count of an
    8 x 8 x 8 periodic grid with the host tool md_waves, which must equal the binding's."""
    import tempfile
    from paper_1305_4196_gb300 import waves as WV
    src = r'''
#include <stdio.h>
#include <stdlib.h>
#include "mdgb.h"
#include "mdgb_waves.h"
int main(void) {
  double box[3] = {40.0, 40.0, 40.0}, eps = 1.0, sig = 1.0, mass = 1.0;
  md_params p = {1, &eps, &sig, NULL, &mass, 0.005, MD_MIXED, MD_LIST_FULL, MD_REBUILD_SKIN_HALF, 10, NULL};
  md_system *s = (md_system *)&p;
  int code = md_create(-1, box, 2.5, 0.3, &p, &s);
  int32_t n[3] = {8, 8, 8}, per[3] = {1, 1, 1};
  int32_t *w = malloc(sizeof(int32_t) * 512);
  int waves = md_waves(n, per, 27, w);
  printf("%d %d %d\n", code, s == NULL, waves);
  free(w);
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "caller.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "caller")
        libdir = os.path.dirname(B.LIB)
        subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", INCLUDE, c, "-o", exe, "-L", libdir, "-lmdgb",
                        "-Wl,-rpath," + libdir], check=True)
        got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert got == [lib.MD_ERR_ARG, 1, WV.waves([8, 8, 8], True)[1]]


def test_struct_layout_matches_binding(lib):
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "mdgb.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(md_params), offsetof(md_params, dt), offsetof(md_params, stream),
         sizeof(md_info), offsetof(md_info, cell_width));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", INCLUDE, c, "-o", exe], check=True)
        got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    P, I = lib.md_params, lib.md_info
    assert got == [C.sizeof(P), P.dt.offset, P.stream.offset, C.sizeof(I), I.cell_width.offset]


def test_argument_errors_before_any_cuda_call(lib):
    M = lib
    cases = [
        dict(n=10, box=[10, 10, 10], code=M.MD_ERR_BOX_TOO_SMALL),          # < 4 r_list per side
        dict(n=10, box=[40, 40, 11.1], code=M.MD_ERR_BOX_TOO_SMALL),
        dict(n=10, box=[40, 40, 40], sigma=-1.0, code=M.MD_ERR_ARG),
        dict(n=10, box=[40, 40, 40], mass=0.0, code=M.MD_ERR_ARG),
        dict(n=10, box=[40, 40, 40], dt=0.0, code=M.MD_ERR_ARG),
        dict(n=10, box=[40, 40, 40], precision=7, code=M.MD_ERR_ARG),
        dict(n=10, box=[40, 40, 40], list_kind=3, code=M.MD_ERR_ARG),
        dict(n=-1, box=[40, 40, 40], code=M.MD_ERR_ARG),
        dict(n=10, box=[40, 40, 40], eps=[[1.0, 2.0], [1.0, 1.0]], sigma=[[1, 1], [1, 1]], mass=[1, 1],
             code=M.MD_ERR_ARG),                                              # asymmetric table
    ]
    for c in cases:
        code = c.pop("code")
        kw = dict(r_cut=2.5, skin=0.3, eps=1.0, sigma=1.0, mass=1.0, dt=0.005)
        kw.update(c)
        with pytest.raises(M.MDError) as ei:
            M.md_create(kw.pop("n"), kw.pop("box"), **kw)
        assert ei.value.code == code, c


def _dbg(lib):
    L = lib._lib
    L.mdgb_grid_shape.argtypes = [C.c_void_p, C.c_double, C.c_int32, C.c_void_p]
    L.mdgb_num_blocks.argtypes = [C.c_void_p, C.c_void_p]
    L.mdgb_block_colour.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
    L.mdgb_tile_cells.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
    L.mdgb_coarse_cells.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int32, C.c_void_p]
    return L


@pytest.mark.parametrize("side,rho,per_block,fit,expect", [
    (134.3677, 0.8442, 224.0, 44, 42),    # 2,048,000-atom liquid
    (107.4942, 0.8442, 224.0, 36, 34),    # 1,048,576 atoms
    (214.9883, 0.8442, 224.0, 76, 68),    # 8,388,608 atoms
    (335.9193, 0.8442, 224.0, 116, 106),  # 32,000,000 atoms
    (67.1838, 0.8442, 224.0, 20, 20),     # 256,000 atoms: the fit is already coarser
    (151.1637, 0.864, 200.0, 52, 50),     # slab + nanoparticles, density the atoms see
    (14.94, 1.2, 224.0, 4, 4),            # whole-box tiles stay: never more cells
    (22.5, 0.1721, 224.0, 8, 6),          # a dilute gas: at least 6
])
def test_coarse_cells(lib, side, rho, per_block, fit, expect):
    """The coarser grid of a mixed full-list system: the smallest even count (at least 6)
    whose cells are at most (per_block / (8 rho))^(1/3) wide, never more than the fit.  The
    expected counts are worked by hand from that definition for the benchmark workloads."""
    L = _dbg(lib)
    out = C.c_int32(0)
    assert L.mdgb_coarse_cells(side, rho, per_block, fit, C.byref(out)) == 0
    nc = out.value
    assert nc == expect
    w_max = (per_block / (8 * rho)) ** (1 / 3)
    assert nc <= fit
    if nc < fit:
        assert nc % 2 == 0 and nc >= 6 and side / nc <= w_max
        # the next even count down would be too coarse (or below 6)
        assert nc == 6 or side / (nc - 2) > w_max
    assert L.mdgb_coarse_cells(side, rho, per_block, 3, C.byref(out)) == lib.MD_ERR_ARG
    assert L.mdgb_coarse_cells(side, 0.0, per_block, fit, C.byref(out)) == lib.MD_ERR_ARG
    assert L.mdgb_coarse_cells(float("nan"), rho, per_block, fit, C.byref(out)) == lib.MD_ERR_ARG


@pytest.mark.parametrize("box,rl", [((16.795962, 16.795962, 16.795962), 2.8),
                                    ((134.3677, 134.3677, 134.3677), 2.8),
                                    ((30.0, 41.0, 52.5), 2.8),
                                    ((20.0, 22.0, 17.0), 2.8)])
def test_grid_shape(lib, box, rl):
    """Sec. II.A: cells at least r_list wide, as many as a multiple of 4 allows (8 colour
    classes of 2x2x2 blocks); full lists take 6 where 6 fit and that rule gives 4."""
    L = _dbg(lib)
    for kind in (lib.MD_LIST_FULL, lib.MD_LIST_HALF_COLOUR8, lib.MD_LIST_HALF_ATOMIC_FREE):
        nc = np.zeros(3, dtype=np.int32)
        assert L.mdgb_grid_shape(np.array(box).ctypes.data, rl, kind, nc.ctypes.data) == 0
        for d in range(3):
            fit = int(np.floor(box[d] / rl))
            assert box[d] / nc[d] >= rl
            if kind == lib.MD_LIST_FULL and 6 <= fit < 8:
                assert nc[d] == 6
            else:
                assert nc[d] % 4 == 0 and box[d] / (nc[d] + 4) < rl
        if box[0] == 134.3677:
            assert nc.tolist() == [44, 44, 44]
        if box[0] == 16.795962:
            assert nc.tolist() == [4, 4, 4]
        if box[0] == 20.0:
            assert nc.tolist() == ([6, 6, 6] if kind == lib.MD_LIST_FULL else [4, 4, 4])
    nc = np.zeros(3, dtype=np.int32)
    assert L.mdgb_grid_shape(np.array(box).ctypes.data, rl, 7, nc.ctypes.data) == lib.MD_ERR_ARG


@pytest.mark.parametrize("nc", [(8, 8, 8), (6, 6, 6), (12, 10, 14)])
def test_tile_order_puts_half_shell_targets_first(lib, nc):
    """Sec. II.D.3: a half list of an own cell holds the cell itself and its 13 forward
    neighbours (dz > 0; dz = 0, dy > 0; dz = dy = 0, dx > 0).  The tile lists the 8 own
    cells first and then every other cell such a list reaches, so that the half-list
    kernel's reaction sums cover tile slots 0..42 only; the 21 cells after them are
    reached by no half list of the block (checked by brute force over the offsets)."""
    L = _dbg(lib)
    ncv = np.array(nc, dtype=np.int32)
    nb = np.zeros(1, dtype=np.int32)
    assert L.mdgb_num_blocks(ncv.ctypes.data, nb.ctypes.data) == 0
    buf = np.zeros(64, dtype=np.int32)
    fwd = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
           if dz > 0 or (dz == 0 and (dy > 0 or (dy == 0 and dx >= 0)))]
    assert len(fwd) == 14
    for b in sorted({0, int(nb[0]) // 2, int(nb[0]) - 1}):
        assert L.mdgb_tile_cells(ncv.ctypes.data, b, buf.ctypes.data) == 0
        cells = buf.tolist()
        coords = [(c % nc[0], (c // nc[0]) % nc[1], c // (nc[0] * nc[1])) for c in cells]
        reached = set()
        for (x, y, z) in coords[:8]:
            for dx, dy, dz in fwd:
                reached.add(((x + dx) % nc[0]) + nc[0] * (((y + dy) % nc[1]) + nc[1] * ((z + dz) % nc[2])))
        assert set(cells[:43]) == reached
        assert not reached & set(cells[43:])


@pytest.mark.parametrize("nc", [(4, 4, 4), (8, 12, 16), (44, 44, 44)])
def test_colour_schedule_tiles_disjoint(lib, nc):
    """Sec. II.A/II.B: tasks in one wave must not overlap.  Every block's 4x4x4 tile
    holds 64 distinct cells, own cells of all blocks partition the grid, and the
    tiles of any two blocks of one colour share no cell."""
    L = _dbg(lib)
    ncv = np.array(nc, dtype=np.int32)
    nb = np.zeros(1, dtype=np.int32)
    assert L.mdgb_num_blocks(ncv.ctypes.data, nb.ctypes.data) == 0
    nb = int(nb[0])
    ncell = nc[0] * nc[1] * nc[2]
    assert nb * 8 == ncell
    own_seen = np.zeros(ncell, dtype=np.int32)
    tiles = {c: [] for c in range(8)}
    buf = np.zeros(64, dtype=np.int32)
    col = np.zeros(1, dtype=np.int32)
    for b in range(nb):
        assert L.mdgb_tile_cells(ncv.ctypes.data, b, buf.ctypes.data) == 0
        assert len(set(buf.tolist())) == 64
        own_seen[buf[:8]] += 1
        assert L.mdgb_block_colour(ncv.ctypes.data, b, col.ctypes.data) == 0
        tiles[int(col[0])].append(buf.copy())
    assert np.all(own_seen == 1)
    for c in range(8):
        allc = np.concatenate(tiles[c])
        assert len(np.unique(allc)) == len(allc), f"colour {c} has overlapping tiles"
        assert len(tiles[c]) == nb // 8
        # blocks of one colour are contiguous in the block numbering
    # own cells of a block are its 2x2x2 cells: adjacent in every dimension
    assert L.mdgb_tile_cells(ncv.ctypes.data, nb, buf.ctypes.data) != 0  # out of range


@pytest.mark.parametrize("nc", [(6, 6, 6), (4, 6, 10), (46, 46, 46)])
def test_linear_block_numbering(lib, nc):
    """Grids with a side of 4k+2 cells (full lists) number their blocks linearly: the numbering
    is a bijection, every tile holds 64 distinct cells, own cells partition the grid, block
    b has coordinates (b mod nb_x, ...), and such grids have no colour classes."""
    L = _dbg(lib)
    ncv = np.array(nc, dtype=np.int32)
    nb = np.zeros(1, dtype=np.int32)
    assert L.mdgb_num_blocks(ncv.ctypes.data, nb.ctypes.data) == 0
    nb = int(nb[0])
    ncell = nc[0] * nc[1] * nc[2]
    assert nb * 8 == ncell
    own_seen = np.zeros(ncell, dtype=np.int32)
    buf = np.zeros(64, dtype=np.int32)
    nbx, nby = nc[0] // 2, nc[1] // 2
    for b in range(nb):
        assert L.mdgb_tile_cells(ncv.ctypes.data, b, buf.ctypes.data) == 0
        assert len(set(buf.tolist())) == 64
        own_seen[buf[:8]] += 1
        bx, by, bz = b % nbx, (b // nbx) % nby, b // (nbx * nby)
        lowest = 2 * bx + nc[0] * (2 * by + nc[1] * 2 * bz)
        assert int(buf[:8].min()) == lowest
    assert np.all(own_seen == 1)
    col = np.zeros(1, dtype=np.int32)
    assert L.mdgb_block_colour(ncv.ctypes.data, 0, col.ctypes.data) == lib.MD_ERR_ARG
    odd = np.array([5, 6, 6], dtype=np.int32)
    out = np.zeros(1, dtype=np.int32)
    assert L.mdgb_num_blocks(odd.ctypes.data, out.ctypes.data) == lib.MD_ERR_ARG


def test_binding_checks_arrays_before_the_call(lib):
    """The C calls read a fixed number of elements of one type through each pointer, so the
    binding refuses, before any call, arrays of another element type, too few elements,
    non-contiguous arrays, a mix of host and device arrays in one call, and md_create
    tables that do not match the species count."""
    import torch
    M = lib
    pos = np.zeros((10, 3))
    assert M._ptr(pos, np.float64, 30, "pos") == (pos.ctypes.data, False)
    with pytest.raises(TypeError):
        M._ptr(pos.astype(np.float32), np.float64, 30, "pos")
    with pytest.raises(ValueError):
        M._ptr(pos, np.float64, 33, "pos")
    with pytest.raises(ValueError):
        M._ptr(np.zeros((3, 10)).T, np.float64, 30, "pos")
    t = torch.zeros(10, dtype=torch.int32)
    assert M._ptr(t, np.int32, 10, "species") == (t.data_ptr(), False)
    with pytest.raises(TypeError):
        M._ptr(t.to(torch.int64), np.int32, 10, "species")
    with pytest.raises(ValueError):
        M._ptr(t, np.int32, 11, "species")
    assert M._ptr(None, np.int32, 10, "species") == (None, None)
    assert M._same_side((1, False), (None, None), (2, False)) is False
    assert M._same_side((None, None)) is None
    with pytest.raises(ValueError):
        M._same_side((1, False), (2, True))
    kw = dict(r_cut=2.5, skin=0.3, dt=0.005)
    with pytest.raises(ValueError):
        M.md_create(10, [40, 40], eps=1.0, sigma=1.0, mass=1.0, **kw)
    with pytest.raises(ValueError):
        M.md_create(10, [40, 40, 40], eps=1.0, sigma=np.ones((2, 2)), mass=[1.0, 1.0], **kw)


def test_binding_marshals_valid_arrays(lib, monkeypatch):
    """With valid arrays every marshalling function reaches its C call with the arrays'
    pointers and one host/device flag (a recording stand-in for the library, no GPU)."""
    import torch
    M = lib
    n = 7
    calls = {}

    class Fake:
        def md_get_info(self, handle, info):
            C.cast(info, C.POINTER(M.md_info)).contents.n = n
            return M.MD_OK

        def __getattr__(self, name):
            def call(*args):
                calls[name] = args
                return M.MD_OK
            return call

    monkeypatch.setattr(M, "_lib", Fake())
    pos, vel = np.zeros((n, 3)), np.zeros((n, 3))
    sp, img = np.zeros(n, dtype=np.int32), np.zeros((n, 3), dtype=np.int32)
    M.md_set_state("h", pos, vel, sp)
    assert calls["md_set_state"] == ("h", pos.ctypes.data, vel.ctypes.data, sp.ctypes.data, 0)
    M.md_set_state("h", pos, None)
    assert calls["md_set_state"] == ("h", pos.ctypes.data, None, None, 0)
    M.md_get_state("h", pos, vel, img)
    assert calls["md_get_state"] == ("h", pos.ctypes.data, vel.ctypes.data, img.ctypes.data, 0)
    M.md_forces("h", None)
    assert calls["md_forces"] == ("h", None, 0)
    M.md_forces("h", pos)
    assert calls["md_forces"] == ("h", pos.ctypes.data, 0)
    M.md_forces_backward("h", pos, vel, 1)
    assert calls["md_forces_backward"][:4] == ("h", pos.ctypes.data, 0, vel.ctypes.data)
    t = torch.zeros((n, 3), dtype=torch.float64)
    M.md_set_state("h", t, t)
    assert calls["md_set_state"] == ("h", t.data_ptr(), t.data_ptr(), None, 0)
    with pytest.raises(ValueError):
        M.md_set_state("h", np.zeros((n - 1, 3)), vel)
    with pytest.raises(TypeError):
        M.md_get_state("h", pos, vel, np.zeros((n, 3), dtype=np.int64))
    with pytest.raises(TypeError):
        M.md_set_state("h", pos, vel, np.zeros(n, dtype=np.int64))
    with pytest.raises(ValueError):
        M.md_set_params("h", np.ones((2, 2)), np.ones((2, 2)), None, nsp=1)
    M.md_set_params("h", 1.0, 1.0, None, nsp=1)
    assert "md_set_params" in calls
