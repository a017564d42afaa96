"""FP64 CPU oracle for the RCLL neighbour search and SPH density path.

TEST INFRASTRUCTURE ONLY.  Imported by tests/, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py``; the product package never
imports, links or runs anything here.  The arithmetic lives in
``sph_oracle.c`` (plain FP64, no fused multiply-add); this module only moves
numpy arrays across ctypes.

Functions and the passage each follows (arXiv 2401.08586):
  kernel_w / kernel_alpha -- cubic B-spline kernel, Eq. 3.
  allpairs                -- all-list search (Section "SPH method", Fig. 3a).
  cll                     -- cell link-list search (same section, Fig. 3b).
  density                 -- summation density with W from Eq. 3 (self term included).
  cll_rows / density_rows -- the same for a listed subset of rows (sampled checks).
  gradient_a5             -- normalised first-order gradient, Appendix Eq. A5.
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(_build.build())
    lib.oracle_kernel_alpha.restype = ctypes.c_double
    lib.oracle_kernel_alpha.argtypes = [ctypes.c_int, ctypes.c_double]
    lib.oracle_kernel_w.restype = ctypes.c_double
    lib.oracle_kernel_w.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
    lib.oracle_kernel_dwdr.restype = ctypes.c_double
    lib.oracle_kernel_dwdr.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
    lib.oracle_kernel_w_array.restype = None
    lib.oracle_kernel_w_array.argtypes = [ctypes.c_int, ctypes.c_int64, _f64p, ctypes.c_double, _f64p]
    lib.oracle_allpairs.restype = ctypes.c_int64
    lib.oracle_allpairs.argtypes = [ctypes.c_int, ctypes.c_int64, _f64p, ctypes.c_double,
                                    _i64p, _i32p, ctypes.c_int64]
    lib.oracle_cll.restype = ctypes.c_int64
    lib.oracle_cll.argtypes = [ctypes.c_int, ctypes.c_int64, _f64p, ctypes.c_double, ctypes.c_int,
                               _i64p, _i32p, ctypes.c_int64]
    lib.oracle_cll_rows.restype = ctypes.c_int64
    lib.oracle_cll_rows.argtypes = [ctypes.c_int, ctypes.c_int64, _f64p, ctypes.c_double, ctypes.c_int,
                                    _i64p, ctypes.c_int64, _i64p, _i32p, ctypes.c_int64]
    lib.oracle_density_rows.restype = None
    lib.oracle_density_rows.argtypes = [ctypes.c_int, _f64p, ctypes.c_double, ctypes.c_double, _i64p,
                                        ctypes.c_int64, _i64p, _i32p, _f64p]
    lib.oracle_density.restype = None
    lib.oracle_density.argtypes = [ctypes.c_int, ctypes.c_int64, _f64p, ctypes.c_double,
                                   ctypes.c_double, _i64p, _i32p, ctypes.c_int, _f64p]
    lib.oracle_gradient_a5.restype = None
    lib.oracle_gradient_a5.argtypes = [ctypes.c_int, ctypes.c_int64, _f64p, ctypes.c_double,
                                       _f64p, _i64p, _i32p, _f64p]
    lib.oracle_openmp_max_threads.restype = ctypes.c_int
    lib.oracle_openmp_max_threads.argtypes = []
    _lib = lib
    return lib


def _ptr(a, t):
    return a.ctypes.data_as(t)


def _coords(xyz):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    if xyz.ndim != 2 or xyz.shape[1] not in (2, 3):
        raise ValueError("xyz must be an (N, 2) or (N, 3) array")
    return xyz


def kernel_alpha(dim, h):
    """alpha_d of Eq. 3."""
    return _load().oracle_kernel_alpha(int(dim), float(h))


def kernel_w(dim, R, h):
    """W(R, h) of Eq. 3, elementwise over R."""
    R = np.ascontiguousarray(np.atleast_1d(R), dtype=np.float64)
    out = np.empty_like(R)
    _load().oracle_kernel_w_array(int(dim), R.size, _ptr(R, _f64p), float(h), _ptr(out, _f64p))
    return out


def kernel_dwdr(dim, R, h):
    """dW/dR of Eq. 3 (the derivative the Appendix A5 gradient uses), elementwise over R."""
    lib = _load()
    R = np.atleast_1d(np.asarray(R, dtype=np.float64))
    return np.array([lib.oracle_kernel_dwdr(int(dim), float(r), float(h)) for r in R])


def _csr(fn, xyz, kh, *extra):
    xyz = _coords(xyz)
    n, dim = xyz.shape
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    nnz = fn(dim, n, _ptr(xyz, _f64p), float(kh), *extra, _ptr(row_ptr, _i64p), None, 0)
    if nnz < 0:
        raise ValueError("domain too large for the oracle's cell grid")
    col = np.zeros(max(nnz, 1), dtype=np.int32)
    nnz2 = fn(dim, n, _ptr(xyz, _f64p), float(kh), *extra, _ptr(row_ptr, _i64p),
              _ptr(col, _i32p), col.size)
    assert nnz2 == nnz
    return row_ptr, col[:nnz]


def allpairs(xyz, kh):
    """All-list neighbour CSR (row_ptr int64[N+1], col int32[nnz]); rows in
    input order, columns ascending, self excluded, strict r^2 < kh^2."""
    return _csr(_load().oracle_allpairs, xyz, kh)


def cll(xyz, kh, threads=1):
    """Cell link-list neighbour CSR, same contract as :func:`allpairs`."""
    return _csr(_load().oracle_cll, xyz, kh, int(threads))


def cll_counts(xyz, kh, threads=1):
    """Row pointer of the cell link-list CSR only (no column array)."""
    xyz = _coords(xyz)
    n, dim = xyz.shape
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    nnz = _load().oracle_cll(dim, n, _ptr(xyz, _f64p), float(kh), int(threads), _ptr(row_ptr, _i64p), None, 0)
    if nnz < 0:
        raise ValueError("domain too large for the oracle's cell grid")
    return row_ptr


def cll_rows(xyz, kh, rows, threads=1):
    """Neighbour lists (ascending input indices) of the listed particles only:
    CSR with one row per entry of ``rows``."""
    xyz = _coords(xyz)
    n, dim = xyz.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= n):
        raise ValueError("row index out of range")
    rp = np.zeros(rows.size + 1, dtype=np.int64)
    lib = _load()
    nnz = lib.oracle_cll_rows(dim, n, _ptr(xyz, _f64p), float(kh), int(threads), _ptr(rows, _i64p), rows.size,
                              _ptr(rp, _i64p), None, 0)
    if nnz < 0:
        raise ValueError("grid too large")
    col = np.empty(max(nnz, 1), dtype=np.int32)
    lib.oracle_cll_rows(dim, n, _ptr(xyz, _f64p), float(kh), int(threads), _ptr(rows, _i64p), rows.size,
                        _ptr(rp, _i64p), _ptr(col, _i32p), col.size)
    return rp, col[:nnz]


def density_rows(xyz, h, rows, row_ptr, col, mass=1.0):
    """FP64 summation density of the listed particles, given their rows."""
    xyz = _coords(xyz)
    dim = xyz.shape[1]
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    rho = np.empty(rows.size, dtype=np.float64)
    _load().oracle_density_rows(dim, _ptr(xyz, _f64p), float(h), float(mass), _ptr(rows, _i64p), rows.size,
                                _ptr(row_ptr, _i64p), _ptr(col, _i32p), _ptr(rho, _f64p))
    return rho


def density(xyz, h, row_ptr, col, mass=1.0, threads=1):
    """FP64 summation density for every particle (self term included)."""
    xyz = _coords(xyz)
    n, dim = xyz.shape
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    rho = np.empty(n, dtype=np.float64)
    _load().oracle_density(dim, n, _ptr(xyz, _f64p), float(h), float(mass), _ptr(row_ptr, _i64p),
                           _ptr(col, _i32p), int(threads), _ptr(rho, _f64p))
    return rho


def gradient_a5(xyz, h, f, row_ptr, col):
    """Appendix Eq. A5 gradient of the particle field f, shape (N, dim)."""
    xyz = _coords(xyz)
    n, dim = xyz.shape
    f = np.ascontiguousarray(f, dtype=np.float64)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    grad = np.empty((n, dim), dtype=np.float64)
    _load().oracle_gradient_a5(dim, n, _ptr(xyz, _f64p), float(h), _ptr(f, _f64p),
                               _ptr(row_ptr, _i64p), _ptr(col, _i32p), _ptr(grad, _f64p))
    return grad


def max_threads():
    """Threads the oracle's OpenMP runtime would use by default."""
    return _load().oracle_openmp_max_threads()
