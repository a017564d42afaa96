"""Row tiles of the single-pass search (row_tile_end and tiles_max in
csrc/sph_internal.cuh), host build: on random and adversarial rows of cells,
the tiles cover each row exactly and in order, hold 1..TILE_ROWS particles
within TILE_SPAN consecutive cells, are cut greedily, and never outnumber the
bound the tile buffers are sized by (len / TILE_ROWS + nx / TILE_SPAN + 1 per
row; tiles_max over a grid)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def tc(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("tc") / "libtc.so")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-shared",
                           "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"),
                           os.path.join(HERE, "native", "tile_cut_shim.cu"), "-o", out])
    lib = ctypes.CDLL(out)
    lib.tc_cut_row.restype = ctypes.c_int
    lib.tc_cut_row.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    lib.tc_tiles_max.restype = ctypes.c_longlong
    lib.tc_tiles_max.argtypes = [ctypes.c_longlong] * 3
    return lib


def cut(tc, counts, base=0):
    """Tile ends of one row whose cells hold `counts` particles, the row
    starting at sorted index `base`."""
    cs = np.ascontiguousarray(np.concatenate([[0], np.cumsum(counts)]) + base, dtype=np.int32)
    nx = len(counts)
    cap = int(cs[-1] - cs[0]) + 1
    ends = np.zeros(cap, dtype=np.int32)
    k = tc.tc_cut_row(cs.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), nx,
                      ends.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), cap)
    return cs, ends[:k]


def check_row(tc, counts, base=0):
    rows, span = tc.tc_tile_rows(), tc.tc_tile_span()
    cs, ends = cut(tc, counts, base)
    nx, total = len(counts), int(cs[-1] - cs[0])
    if total == 0:
        assert len(ends) == 0
        return 0
    starts = np.concatenate([[cs[0]], ends[:-1]])
    assert ends[-1] == cs[-1]                        # the row is covered to its end
    sizes = ends - starts
    assert (sizes >= 1).all() and (sizes <= rows).all()
    # cell of sorted position p: the last cell whose start is <= p among non-empty cells
    cell_of = lambda p: int(np.searchsorted(cs[1:], p, side="right"))
    for s, e in zip(starts, ends):
        c0, c1 = cell_of(s), cell_of(e - 1)
        assert c1 - c0 < span, (s, e, c0, c1)
        if e != cs[-1]:
            # greedy: the tile stops only at TILE_ROWS particles or where the
            # next particle would leave the span
            assert e - s == rows or e == cs[min(c0 + span, nx)], (s, e)
    assert len(ends) <= total // rows + nx // span + 1
    return len(ends)


def test_empty_and_single_cell_rows(tc):
    assert check_row(tc, [0]) == 0
    assert check_row(tc, [0] * 17) == 0
    assert check_row(tc, [1]) == 1
    assert check_row(tc, [32]) == 1
    assert check_row(tc, [33]) == 2
    assert check_row(tc, [1000]) == 32  # 31 full tiles and the rest


def test_span_limit_and_full_tiles(tc):
    # 4 cells of 8 fill one tile exactly; a fifth cell starts a new tile
    assert check_row(tc, [8] * 4) == 1
    assert check_row(tc, [8] * 5) == 2
    # sparse cells: the span, not the particle count, ends each tile
    assert check_row(tc, [1] * 40) == 10
    assert check_row(tc, [1, 0, 0, 0] * 10) == 10


def test_random_rows(tc):
    rng = np.random.default_rng(11)
    for trial in range(3000):
        nx = int(rng.integers(1, 160))
        kind = trial % 5
        if kind == 0:
            counts = rng.poisson(18.0, nx)                      # the jittered-lattice mean
        elif kind == 1:
            counts = rng.poisson(0.7, nx)                       # sparse spray
        elif kind == 2:
            counts = rng.integers(0, 70, nx) * (rng.random(nx) < 0.3)   # clustered
        elif kind == 3:
            counts = np.where(rng.random(nx) < 0.5, 31, 1)      # just under a tile per cell
        else:
            counts = rng.geometric(0.05, nx) - 1                # heavy tail
        check_row(tc, counts.astype(np.int64), base=int(rng.integers(0, 1 << 20)))


def test_grid_total_within_tiles_max(tc):
    rng = np.random.default_rng(12)
    for trial in range(40):
        nx, nrow = int(rng.integers(1, 60)), int(rng.integers(1, 80))
        lam = [0.3, 3.0, 18.0, 60.0][trial % 4]
        counts = rng.poisson(lam, (nrow, nx))
        total, base = 0, 0
        for r in range(nrow):
            total += check_row(tc, counts[r], base)
            base += int(counts[r].sum())
        n, ncell = int(counts.sum()), nx * nrow
        assert total <= tc.tc_tiles_max(n, ncell, nrow)
