"""Division by an invariant divisor (csrc/fastdiv.h), host build: exact
against the division operator for divisors and dividends across the 32-bit
range, including the values the grids use (cells per axis and per layer)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def fd(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("fd") / "libfd.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                           os.path.join(HERE, "native", "fastdiv_shim.cpp"), "-o", out])
    lib = ctypes.CDLL(out)
    lib.fd_check.restype = ctypes.c_longlong
    lib.fd_check.argtypes = [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32), ctypes.c_longlong]
    return lib


def check(fd, d, n):
    n = np.ascontiguousarray(n, dtype=np.uint32)
    return fd.fd_check(d, n.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), n.size)


def test_exhaustive_small(fd):
    n = np.arange(0, 1 << 20, dtype=np.uint32)
    for d in list(range(1, 300)) + [1 << 20, (1 << 20) - 1, 1521, 39 * 39, 67 * 67]:
        assert check(fd, d, n) == 0, d


def test_random_full_range(fd):
    rng = np.random.default_rng(0)
    n = np.concatenate([rng.integers(0, 1 << 32, size=200000, dtype=np.uint64).astype(np.uint32),
                        np.array([0, 1, (1 << 31) - 1, 1 << 31, (1 << 32) - 1], dtype=np.uint32)])
    ds = rng.integers(1, 1 << 32, size=200, dtype=np.uint64).tolist() + [2, 3, 7, 1 << 31, (1 << 32) - 1]
    for d in ds:
        assert check(fd, int(d), n) == 0, d
