"""The C-ABI library loads on a machine without a GPU and exports every entry
point declared in include/*.h (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2401_08586_gb300 import build as lib_build
from paper_2401_08586_gb300 import sph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sph_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    lib_build.build()
    return ctypes.CDLL(lib_build.LIB)


def test_header_declares_core_calls():
    names = declared_functions()
    for core in ("sph_bin_cells", "sph_nnps_query", "sph_density_sum", "sph_grid_free", "sph_last_error"):
        assert core in names


def test_every_declared_symbol_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    assert set(declared_functions()) <= set(sph.exported_symbols()) | set(getattr(sph, "EXTRA_SYMBOLS", ()))


def test_host_only_calls(lib):
    sph.load()
    assert sph.sph_version() >= 100
    tau16, tau32 = sph.sph_precision_bands()
    assert 0 < tau32 < tau16 < 0.1


def test_invalid_params_rejected_without_gpu():
    """Parameter validation happens before any CUDA call."""
    p = sph.make_params(4, 0.01)  # dim 4 is invalid
    with pytest.raises(sph.SphError) as ei:
        sph.sph_bin_cells(p, 0, 10, stream=0)
    assert ei.value.code == sph.SPH_ERR_INVALID
    p = sph.make_params(3, -1.0)
    with pytest.raises(sph.SphError) as ei:
        sph.sph_bin_cells(p, 0, 10, stream=0)
    assert ei.value.code == sph.SPH_ERR_INVALID
    p = sph.make_params(3, 0.01, cell_size=0.015)  # smaller than kh
    with pytest.raises(sph.SphError):
        sph.sph_bin_cells(p, 0, 10, stream=0)
