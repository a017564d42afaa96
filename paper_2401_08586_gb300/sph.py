"""ctypes binding of libsph (include/sph.h): argument marshalling only.

Every entry point of the C ABI is exposed under the same name and takes the
same arguments; torch tensors are accepted wherever the C call takes a device
pointer (their ``data_ptr()`` is passed) and streams default to torch's current
stream.  All the computation happens in the CUDA library; if ``libsph.so`` is
missing or no GPU is present the calls raise instead of falling back.

Convenience wrappers (:class:`Grid`, :func:`neighbours`) only allocate the torch
output tensors and sequence the C calls.
"""
import ctypes
import os

import numpy as np

from . import build as _build

SPH_OK = 0
SPH_PENDING = 1
SPH_ERR_INVALID = -1
SPH_ERR_CAPACITY = -2
SPH_ERR_BUDGET = -3
SPH_ERR_CUDA = -4
SPH_ERR_TIMEOUT = -5
SPH_ERR_DEVICE_CHECK = -6
SPH_ERR_NOMEM = -7
SPH_ERR_NOT_FOUND = -8

SPH_ORDER_CELL = 0
SPH_ORDER_CANONICAL = 1
SPH_PREC_FP16_RCLL = 0
SPH_PREC_FP64_CLL = 1

_ERRNAMES = {v: k for k, v in dict(globals()).items() if k.startswith("SPH_ERR_") or k in ("SPH_OK", "SPH_PENDING")}


class SphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_ERRNAMES.get(code, "SPH_ERR"), code, msg))
        self.code = code


class sph_params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("order", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("have_box", ctypes.c_int32), ("h", ctypes.c_double), ("kh", ctypes.c_double),
                ("cell_size", ctypes.c_double), ("box_lo", ctypes.c_double * 3),
                ("box_hi", ctypes.c_double * 3), ("mass", ctypes.c_double)]


class sph_grid_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ncell", ctypes.c_int64), ("nk", ctypes.c_int32 * 3),
                ("dim", ctypes.c_int32), ("lo", ctypes.c_double * 3), ("cell_size", ctypes.c_double),
                ("cell_start", ctypes.c_void_p), ("orig_id", ctypes.c_void_p), ("rank", ctypes.c_void_p),
                ("stat_fp32_pairs", ctypes.c_int64), ("stat_fp64_pairs", ctypes.c_int64)]


class sph_batch_out(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("col_capacity", ctypes.c_int64),
                ("rho", ctypes.c_void_p), ("orig_id", ctypes.c_void_p),
                ("sys_first", ctypes.POINTER(ctypes.c_int64)), ("nnz", ctypes.c_int64)]


class sph_batch_stats(ctypes.Structure):
    _fields_ = [("runs", ctypes.c_int64), ("graph_captures", ctypes.c_int64), ("graph_replays", ctypes.c_int64),
                ("tuned_staging", ctypes.c_int32), ("tuned_candidates", ctypes.c_int32),
                ("tuned_shape", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("fp32_pairs", ctypes.c_int64), ("fp64_pairs", ctypes.c_int64),
                ("direct_launches", ctypes.c_int64), ("graph_launched", ctypes.c_int64)]


class sph_server_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("streams", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("small_n", ctypes.c_int64), ("max_wait_ns", ctypes.c_int64), ("large_n", ctypes.c_int64),
                ("large_sm_percent", ctypes.c_int32), ("reserve_pool", ctypes.c_int32)]


class sph_request(ctypes.Structure):
    _fields_ = [("params", sph_params), ("xyz", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("xyz_on_device", ctypes.c_int32), ("want_density", ctypes.c_int32)]


class sph_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("rho", ctypes.c_void_p),
                ("orig_id", ctypes.c_void_p), ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64)]


class sph_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("batched_requests", ctypes.c_int64), ("held_bytes", ctypes.c_int64),
                ("peak_held_bytes", ctypes.c_int64), ("queued", ctypes.c_int64)]


class sph_precision_counts(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int64), ("neighbours", ctypes.c_int64), ("wrong_fp16_abs", ctypes.c_int64),
                ("wrong_fp32_abs", ctypes.c_int64), ("wrong_fp16_rcll", ctypes.c_int64),
                ("wrong_tiered", ctypes.c_int64)]


SPH_BATCH_OPT_GRAPH = 1
SPH_BATCH_OPT_STAGING = 2

_lib = None
_vp = ctypes.c_void_p


def lib_path():
    return _build.LIB


def load(build_if_missing=False):
    """Load libsph.so (building it first if asked).  Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libsph.so is not built (%s); run __graft_entry__.build()" % path)
        _build.build()
    lib = ctypes.CDLL(path)
    sig = {
        "sph_bin_cells": [ctypes.POINTER(sph_params), _vp, ctypes.c_int64, _vp, ctypes.POINTER(_vp)],
        "sph_nnps_query": [_vp, _vp, _vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), _vp, _vp],
        "sph_density_sum": [_vp, _vp, _vp, _vp, _vp],
        "sph_grid_info_get": [_vp, ctypes.POINTER(sph_grid_info)],
        "sph_grid_export": [_vp, _vp, _vp, _vp, _vp],
        "sph_grid_export_rel": [_vp, _vp, _vp, _vp],
        "sph_density_half": [_vp, _vp, _vp],
        "sph_grid_check": [_vp, _vp],
        "sph_grid_free": [_vp],
        "sph_last_error": [],
        "sph_precision_bands": [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
        "sph_version": [],
        "sph_search_host": [ctypes.POINTER(sph_params), _vp, ctypes.c_int64, _vp, ctypes.POINTER(ctypes.c_int64),
                            ctypes.POINTER(_vp), _vp],
        "sph_grid_csr": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                         ctypes.POINTER(ctypes.c_int64)],
        "sph_grid_csr_copy": [_vp, _vp, _vp, _vp],
        "sph_nnps_query_half": [_vp, _vp, _vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), _vp, _vp],
        "sph_search_host_async": [ctypes.POINTER(sph_params), _vp, ctypes.c_int64, _vp, ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(_vp), _vp],
        "sph_search_host_finish": [_vp, ctypes.POINTER(ctypes.c_int64)],
        "sph_profile_enable": [ctypes.c_int],
        "sph_profile_reset": [],
        "sph_profile_select": [ctypes.c_char_p],
        "sph_device_fp64_rate": [ctypes.POINTER(ctypes.c_double)],
        "sph_profile_read": [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)],
        "sph_launch_count": [],
        "sph_grid_set_option": [_vp, ctypes.c_int, ctypes.c_int64],
        "sph_nnps_query_static": [_vp, _vp, _vp, ctypes.c_int64, _vp, _vp],
        "sph_advance": [_vp, _vp, _vp, ctypes.c_double, _vp],
        "sph_gradient_a5": [_vp, _vp, _vp, _vp, _vp, _vp],
        "sph_precision_study": [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(sph_precision_counts), _vp],
        "sph_batch_run": [ctypes.POINTER(_vp), ctypes.POINTER(sph_params), ctypes.POINTER(_vp),
                          ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.POINTER(sph_batch_out), _vp],
        "sph_batch_get_stats": [_vp, ctypes.POINTER(sph_batch_stats)],
        "sph_batch_create": [ctypes.POINTER(_vp)],
        "sph_batch_set_option": [_vp, ctypes.c_int, ctypes.c_int64],
        "sph_batch_free": [_vp],
        "sph_server_create": [ctypes.POINTER(sph_server_cfg), ctypes.POINTER(_vp)],
        "sph_serve_submit": [_vp, ctypes.POINTER(sph_request), ctypes.POINTER(ctypes.c_uint64)],
        "sph_serve_poll": [_vp, ctypes.c_uint64, ctypes.POINTER(sph_result)],
        "sph_serve_wait": [_vp, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(sph_result)],
        "sph_result_copy": [_vp, ctypes.c_uint64, _vp, _vp, _vp, _vp, _vp],
        "sph_result_release": [_vp, ctypes.c_uint64],
        "sph_server_get_stats": [_vp, ctypes.POINTER(sph_server_stats)],
        "sph_server_destroy": [_vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name == "sph_last_error" else ctypes.c_int
    lib.sph_launch_count.restype = ctypes.c_int64
    _lib = lib
    return lib


def exported_symbols():
    """Names of the C-ABI entry points this binding expects."""
    return ["sph_bin_cells", "sph_nnps_query", "sph_density_sum", "sph_grid_info_get",
            "sph_grid_export", "sph_grid_export_rel", "sph_density_half", "sph_grid_check", "sph_grid_free", "sph_last_error",
            "sph_precision_bands", "sph_version", "sph_search_host", "sph_grid_csr", "sph_grid_csr_copy",
            "sph_nnps_query_half", "sph_search_host_async", "sph_search_host_finish",
            "sph_profile_enable", "sph_profile_select", "sph_profile_reset", "sph_profile_read",
            "sph_launch_count", "sph_grid_set_option", "sph_nnps_query_static", "sph_device_fp64_rate",
            "sph_advance", "sph_gradient_a5", "sph_precision_study", "sph_batch_create", "sph_batch_run", "sph_batch_get_stats", "sph_batch_set_option", "sph_batch_free",
            "sph_server_create", "sph_serve_submit", "sph_serve_poll", "sph_serve_wait", "sph_result_copy",
            "sph_result_release", "sph_server_get_stats", "sph_server_destroy"]


def sph_nnps_query_static(grid, row_ptr, col, col_capacity, rho=None, stream=None):
    """The search without any device allocation (working memory is a fixed
    array inside the library); see include/sph.h for its limits."""
    _check(load().sph_nnps_query_static(grid, _ptr(row_ptr), _ptr(col), int(col_capacity), _ptr(rho),
                                        _stream(stream)))


SPH_OPT_FUSED = 1
SPH_OPT_STAGING = 2
SPH_OPT_TILE_SHAPE = 3
SPH_OPT_TEST_LOOKBACK = 4
SPH_OPT_SM_SHARE = 5


def sph_grid_set_option(grid, option, value):
    _check(load().sph_grid_set_option(grid, int(option), int(value)))


def _check(rc):
    if rc < 0:
        raise SphError(rc, load().sph_last_error().decode())
    return rc


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- the C entry points, same names ----------------------------------------

def sph_bin_cells(params, xyz, n, stream=None, grid=None):
    """Returns the (possibly new) grid handle (an int)."""
    g = _vp(grid)
    _check(load().sph_bin_cells(ctypes.byref(params), _ptr(xyz), int(n), _stream(stream), ctypes.byref(g)))
    return g.value


def sph_nnps_query(grid, row_ptr, col=None, col_capacity=0, want_nnz=True, rho=None, stream=None):
    """Returns nnz (an int) when want_nnz, else None."""
    nnz = ctypes.c_int64(-1)
    _check(load().sph_nnps_query(grid, _ptr(row_ptr), _ptr(col), int(col_capacity),
                                 ctypes.byref(nnz) if want_nnz else None, _ptr(rho), _stream(stream)))
    return nnz.value if want_nnz else None


def sph_density_sum(grid, row_ptr, col, rho, stream=None):
    _check(load().sph_density_sum(grid, _ptr(row_ptr), _ptr(col), _ptr(rho), _stream(stream)))


def sph_grid_info_get(grid):
    info = sph_grid_info()
    _check(load().sph_grid_info_get(grid, ctypes.byref(info)))
    return info


def sph_grid_export(grid, orig_id=None, rank=None, cell_start=None, stream=None):
    _check(load().sph_grid_export(grid, _ptr(orig_id), _ptr(rank), _ptr(cell_start), _stream(stream)))


def sph_density_half(grid, rho, stream=None):
    _check(load().sph_density_half(grid, _ptr(rho), _stream(stream)))


def sph_grid_export_rel(grid, rel16=None, rel32=None, stream=None):
    _check(load().sph_grid_export_rel(grid, _ptr(rel16), _ptr(rel32), _stream(stream)))


def sph_grid_check(grid, stream=None):
    return _check(load().sph_grid_check(grid, _stream(stream)))


def sph_grid_free(grid):
    if grid:
        _check(load().sph_grid_free(grid))


def sph_last_error():
    return load().sph_last_error().decode()


def sph_precision_bands():
    """(tau16, tau32) of the FP16 test and FP32 re-decision, in units of u^2."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().sph_precision_bands(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def sph_version():
    return load().sph_version()


def sph_search_host(params, xyz_host, n, rho_host=None, stream=None, grid=None):
    """xyz_host / rho_host: host numpy arrays or pinned CPU torch tensors
    (float64 n x dim / float32 n).  Returns (grid handle, nnz)."""
    g = _vp(grid)
    nnz = ctypes.c_int64(-1)
    _check(load().sph_search_host(ctypes.byref(params), _host_ptr(xyz_host), int(n), _host_ptr(rho_host),
                                  ctypes.byref(nnz), ctypes.byref(g), _stream(stream)))
    return g.value, nnz.value


def sph_nnps_query_half(grid, row_ptr, col=None, col_capacity=0, rho=None, stream=None):
    """Half-stencil neighbour list (include/sph.h); returns nnz."""
    nnz = ctypes.c_int64(-1)
    _check(load().sph_nnps_query_half(grid, _ptr(row_ptr), _ptr(col), int(col_capacity), ctypes.byref(nnz), _ptr(rho),
                                      _stream(stream)))
    return nnz.value


def sph_grid_csr_copy(grid, row_ptr=None, col=None, stream=None):
    """Copy the grid-owned CSR of the last sph_search_host into row_ptr / col
    (pinned CPU or CUDA tensors, or host numpy arrays); synchronises."""
    _check(load().sph_grid_csr_copy(grid, _host_ptr(row_ptr), _host_ptr(col), _stream(stream)))


def sph_search_host_async(params, xyz_host, n, rho_host=None, stream=None, grid=None):
    """Queue a host-buffer search (include/sph.h); returns the grid handle.
    xyz_host / rho_host must stay alive until sph_search_host_finish."""
    g = _vp(grid)
    _check(load().sph_search_host_async(ctypes.byref(params), _host_ptr(xyz_host), int(n), _host_ptr(rho_host), None,
                                        ctypes.byref(g), _stream(stream)))
    return g.value


def sph_search_host_finish(grid):
    """Wait for the grid's queued host-buffer search; returns nnz."""
    nnz = ctypes.c_int64(-1)
    _check(load().sph_search_host_finish(grid, ctypes.byref(nnz)))
    return nnz.value


def sph_grid_csr(grid):
    """(row_ptr, col, rho) device addresses and nnz of the grid-owned CSR."""
    a, b, c = _vp(), _vp(), _vp()
    nnz = ctypes.c_int64()
    _check(load().sph_grid_csr(grid, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(nnz)))
    return a.value, b.value, c.value, nnz.value


def sph_profile_enable(on=True):
    _check(load().sph_profile_enable(1 if on else 0))


def sph_profile_select(kernels=None):
    """Time only the listed kernel tags (comma-separated string or list; None: all)."""
    if kernels is not None and not isinstance(kernels, str):
        kernels = ",".join(kernels)
    _check(load().sph_profile_select(None if kernels is None else kernels.encode()))


def sph_device_fp64_rate():
    """Measured FP64 FMA throughput of the current device, FLOP/s."""
    v = ctypes.c_double(0.0)
    _check(load().sph_device_fp64_rate(ctypes.byref(v)))
    return v.value


def sph_profile_reset():
    _check(load().sph_profile_reset())


def sph_profile_read(kernel):
    """(total milliseconds, launches) of one kernel tag since the last reset."""
    ms = ctypes.c_double()
    cnt = ctypes.c_int64()
    _check(load().sph_profile_read(kernel.encode(), ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value


def sph_launch_count():
    return load().sph_launch_count()


def _host_ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


# ---- convenience ------------------------------------------------------------

def sph_gradient_a5(grid, row_ptr, col, f, grad, stream=None):
    """Appendix Eq. A5 gradient of f over the grid's CSR into grad (n x dim)."""
    _check(load().sph_gradient_a5(grid, _ptr(row_ptr), _ptr(col), _ptr(f), _ptr(grad), _stream(stream)))


def sph_precision_study(grid, row_begin=0, row_end=None, stream=None):
    """Wrong-decision counts of reduced-precision neighbour tests (dict)."""
    c = sph_precision_counts()
    if row_end is None:
        row_end = 1 << 62
    _check(load().sph_precision_study(grid, int(row_begin), int(row_end), ctypes.byref(c), _stream(stream)))
    return {k: getattr(c, k) for k, _ in sph_precision_counts._fields_}


def sph_advance(grid, xyz_new, vel, dt, stream=None):
    """Eq. 8-9 time step of a binned grid (see include/sph.h)."""
    _check(load().sph_advance(grid, _ptr(xyz_new), _ptr(vel), float(dt), _stream(stream)))


def sph_batch_run(batch, params_list, xyz_list, out, stream=None):
    """One batched run.  batch: workspace handle (None on first use); params_list:
    sph_params per system; xyz_list: (n_s, dim) float64 CUDA tensors; out: a
    filled sph_batch_out.  Returns the (possibly new) workspace handle."""
    nsys = len(params_list)
    P = (sph_params * nsys)(*params_list)
    X = (_vp * nsys)(*[_ptr(x) for x in xyz_list])
    N = (ctypes.c_int64 * nsys)(*[int(x.shape[0]) for x in xyz_list])
    h = _vp(batch)
    _check(load().sph_batch_run(ctypes.byref(h), P, X, N, nsys, ctypes.byref(out), _stream(stream)))
    return h.value


def sph_batch_create():
    h = _vp()
    _check(load().sph_batch_create(ctypes.byref(h)))
    return h.value


def sph_batch_get_stats(batch):
    st = sph_batch_stats()
    _check(load().sph_batch_get_stats(batch, ctypes.byref(st)))
    return st


def sph_batch_set_option(batch, option, value):
    _check(load().sph_batch_set_option(batch, int(option), int(value)))


def sph_batch_free(batch):
    _check(load().sph_batch_free(batch))


class Batch:
    """Workspace of batched runs plus torch-allocated outputs.

    ``run(systems)`` takes a list of (xyz CUDA tensor, sph_params) and returns
    (row_ptr, col, rho, orig_id, sys_first): the block-diagonal cell-order CSR
    of the concatenation (see include/sph.h).  The output tensors are views of
    buffers the workspace keeps and reuses (so a repeated run of the same
    shapes replays its recorded CUDA graph); the next run overwrites them.
    The column buffer grows, by a count-only run, when it is too small."""

    def __init__(self):
        self.handle = None
        self.handle = sph_batch_create()
        self._rp = self._col = self._rho = self._orig = None
        self._first = None

    def _buffers(self, ntot, nsys, dev, density):
        import torch
        if self._rp is None or self._rp.numel() != ntot + 1 or self._rp.device != dev:
            self._rp = torch.empty(ntot + 1, dtype=torch.int64, device=dev)
            self._orig = torch.empty(max(ntot, 1), dtype=torch.int32, device=dev)
            self._rho = None
        if density and self._rho is None:
            self._rho = torch.empty(max(ntot, 1), dtype=torch.float32, device=dev)
        if self._first is None or len(self._first) != nsys + 1:
            self._first = (ctypes.c_int64 * (nsys + 1))()

    def run(self, systems, density=True, stream=None, capacity=None):
        import torch
        xs = [x.contiguous() for x, _ in systems]
        ps = [p for _, p in systems]
        ntot = sum(int(x.shape[0]) for x in xs)
        dev = xs[0].device
        self._buffers(ntot, len(xs), dev, density)
        rho = self._rho if density else None
        if capacity is not None and (self._col is None or self._col.numel() < capacity):
            self._col = torch.empty(max(int(capacity), 1), dtype=torch.int32, device=dev)
        if self._col is None:
            out = sph_batch_out(_ptr(self._rp), None, 0, None, _ptr(self._orig), self._first, 0)
            sph_batch_run(self.handle, ps, xs, out, stream)
            self._col = torch.empty(max(int(out.nnz * 1.05) + 1024, 1), dtype=torch.int32, device=dev)
        while True:
            out = sph_batch_out(_ptr(self._rp), _ptr(self._col), self._col.numel(), _ptr(rho), _ptr(self._orig),
                                self._first, 0)
            try:
                sph_batch_run(self.handle, ps, xs, out, stream)
                break
            except SphError as e:
                if e.code != SPH_ERR_CAPACITY:
                    raise
                self._col = torch.empty(int(out.nnz * 1.05) + 1024, dtype=torch.int32, device=dev)
        self._keep = xs
        nnz = int(out.nnz)
        return (self._rp, self._col[:nnz], (rho[:ntot] if density else None), self._orig[:ntot],
                list(self._first))

    def stats(self):
        return sph_batch_get_stats(self.handle)

    def set_option(self, option, value):
        sph_batch_set_option(self.handle, option, value)

    def close(self):
        if self.handle is not None:
            sph_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sph_server_create(cfg):
    h = _vp()
    _check(load().sph_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def sph_serve_submit(server, req):
    t = ctypes.c_uint64(0)
    _check(load().sph_serve_submit(server, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def sph_serve_poll(server, ticket):
    """The finished request's sph_result, or None while it is pending."""
    res = sph_result()
    rc = load().sph_serve_poll(server, ticket, ctypes.byref(res))
    if rc == SPH_PENDING:
        return None
    _check(rc)
    return res


def sph_serve_wait(server, ticket, timeout_ns=-1):
    res = sph_result()
    rc = load().sph_serve_wait(server, ticket, int(timeout_ns), ctypes.byref(res))
    if rc == SPH_PENDING:
        return None
    _check(rc)
    return res


def sph_result_copy(server, ticket, row_ptr=None, col=None, rho=None, orig_id=None, stream=None):
    _check(load().sph_result_copy(server, ticket, _ptr(row_ptr), _ptr(col), _ptr(rho), _ptr(orig_id),
                                  _stream(stream)))


def sph_result_release(server, ticket):
    _check(load().sph_result_release(server, ticket))


def sph_server_get_stats(server):
    st = sph_server_stats()
    _check(load().sph_server_get_stats(server, ctypes.byref(st)))
    return st


def sph_server_destroy(server):
    _check(load().sph_server_destroy(server))


class Server:
    """Request server (see include/sph.h).  ``submit`` keeps a reference to
    the coordinates until the request is released."""

    def __init__(self, budget_bytes, streams=0, max_batch=0, small_n=0, max_wait_ns=0, large_n=0,
                 large_sm_percent=0, reserve_pool=0):
        self.handle = None
        self.handle = sph_server_create(sph_server_cfg(int(budget_bytes), streams, max_batch, small_n, max_wait_ns,
                                                       large_n, large_sm_percent, reserve_pool))
        self._keep = {}

    def submit(self, xyz, params, density=True):
        """xyz: float64 array (numpy on the host, or a CUDA tensor)."""
        if isinstance(xyz, np.ndarray):
            xyz = np.ascontiguousarray(xyz, dtype=np.float64)
            ptr, on_dev = xyz.ctypes.data, 0
        else:
            xyz = xyz.contiguous()
            ptr, on_dev = xyz.data_ptr(), 1
        req = sph_request(params, ptr if xyz.shape[0] else None, int(xyz.shape[0]), on_dev, int(density))
        t = sph_serve_submit(self.handle, req)
        self._keep[t] = xyz
        return t

    def poll(self, ticket):
        return sph_serve_poll(self.handle, ticket)

    def wait(self, ticket, timeout_s=None):
        return sph_serve_wait(self.handle, ticket, -1 if timeout_s is None else int(timeout_s * 1e9))

    def fetch(self, ticket, stream=None):
        """Copies of a finished request's results as CUDA tensors:
        (row_ptr, col, rho or None, orig_id or None)."""
        import torch
        res = self.wait(ticket)
        if res.status != SPH_OK:
            raise SphError(res.status, "request %d failed" % ticket)
        rp = torch.empty(res.n + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(max(res.nnz, 1), dtype=torch.int32, device="cuda")
        rho = torch.empty(max(res.n, 1), dtype=torch.float32, device="cuda") if res.rho else None
        orig = torch.empty(max(res.n, 1), dtype=torch.int32, device="cuda") if res.orig_id else None
        sph_result_copy(self.handle, ticket, rp, col, rho, orig, stream)
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return rp, col[:res.nnz], (rho[:res.n] if rho is not None else None), (orig[:res.n] if orig is not None else None)

    def release(self, ticket):
        sph_result_release(self.handle, ticket)
        self._keep.pop(ticket, None)

    def stats(self):
        return sph_server_get_stats(self.handle)

    def close(self):
        if self.handle is not None:
            sph_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_params(dim, h, kh=None, order=SPH_ORDER_CELL, precision=SPH_PREC_FP16_RCLL, mass=1.0,
                cell_size=0.0, box=None):
    p = sph_params()
    p.dim = int(dim)
    p.order = int(order)
    p.precision = int(precision)
    p.h = float(h)
    p.kh = float(2.0 * h if kh is None else kh)
    p.cell_size = float(cell_size)
    p.mass = float(mass)
    if box is not None:
        p.have_box = 1
        lo, hi = box
        for k in range(dim):
            p.box_lo[k] = float(lo[k])
            p.box_hi[k] = float(hi[k])
    return p


class Grid:
    """A binned particle system on the current CUDA device.

    ``xyz`` is an (N, dim) float64 CUDA tensor; it is referenced (not copied),
    so it is kept alive here.
    """

    def __init__(self, xyz, h, kh=None, order=SPH_ORDER_CELL, precision=SPH_PREC_FP16_RCLL, mass=1.0,
                 cell_size=0.0, box=None, stream=None):
        import torch
        if not (isinstance(xyz, torch.Tensor) and xyz.is_cuda and xyz.dtype == torch.float64):
            raise TypeError("xyz must be a float64 CUDA tensor")
        self.xyz = xyz.contiguous()
        self.params = make_params(self.xyz.shape[1], h, kh, order, precision, mass, cell_size, box)
        self.handle = None
        self.handle = sph_bin_cells(self.params, self.xyz, self.xyz.shape[0], stream, None)

    def gradient(self, row_ptr, col, f, stream=None):
        """Appendix Eq. A5 gradient (n x dim float64 CUDA tensor) of the field
        f (float64, input order) over the CSR of :meth:`query`."""
        import torch
        g = torch.empty((self.n, self.xyz.shape[1]), dtype=torch.float64, device=self.xyz.device)
        sph_gradient_a5(self.handle, row_ptr, col, f.contiguous(), g, stream)
        return g

    def advance(self, xyz_new, vel, dt, stream=None):
        """Eq. 8-9 step: positions after the step and the velocities (CUDA
        float64 tensors, input order)."""
        self.xyz = xyz_new.contiguous()
        self._vel = vel.contiguous()
        sph_advance(self.handle, self.xyz, self._vel, dt, stream)

    def rebin(self, xyz=None, stream=None):
        if xyz is not None:
            self.xyz = xyz.contiguous()
        sph_bin_cells(self.params, self.xyz, self.xyz.shape[0], stream, self.handle)

    @property
    def n(self):
        return self.xyz.shape[0]

    def info(self):
        return sph_grid_info_get(self.handle)

    def orig_id(self, stream=None):
        """int32[N] tensor: sorted position -> input index."""
        import torch
        out = torch.empty(self.n, dtype=torch.int32, device=self.xyz.device)
        sph_grid_export(self.handle, out, None, None, stream)
        return out

    def density_half(self, stream=None):
        """float32[N] tensor: the summation density over a half stencil
        (no neighbour list), in sorted order (row r is input orig_id[r])."""
        import torch
        rho = torch.empty(self.n, dtype=torch.float32, device=self.xyz.device)
        sph_density_half(self.handle, rho, stream)
        return rho

    def relative_coordinates(self, stream=None):
        """(rel16, rel32) in sorted order: float16[N, 4] (x, y, z, then the
        bits of the cell x index modulo 2^16) and float32[N, 4] (x, y, z, 0)
        tensors of the stored cell-relative coordinates."""
        import torch
        r16 = torch.empty((self.n, 4), dtype=torch.int16, device=self.xyz.device)
        r32 = torch.empty((self.n, 4), dtype=torch.float32, device=self.xyz.device)
        sph_grid_export_rel(self.handle, r16, r32, stream)
        return r16.view(torch.float16), r32

    def rank(self, stream=None):
        """int32[N] tensor: input index -> sorted position."""
        import torch
        out = torch.empty(self.n, dtype=torch.int32, device=self.xyz.device)
        sph_grid_export(self.handle, None, out, None, stream)
        return out

    def cell_start(self, stream=None):
        import torch
        out = torch.empty(int(self.info().ncell) + 1, dtype=torch.int32, device=self.xyz.device)
        sph_grid_export(self.handle, None, None, out, stream)
        return out

    def query(self, density=True, col_capacity=None, stream=None):
        """Run the search; returns (row_ptr int64[N+1], col int32[nnz], rho float32[N] or None)."""
        import torch
        dev = self.xyz.device
        row_ptr = torch.empty(self.n + 1, dtype=torch.int64, device=dev)
        if col_capacity is None:
            nnz = sph_nnps_query(self.handle, row_ptr, None, 0, True, None, stream)
            col_capacity = nnz
        col = torch.empty(max(int(col_capacity), 1), dtype=torch.int32, device=dev)
        rho = torch.empty(self.n, dtype=torch.float32, device=dev) if density else None
        nnz = sph_nnps_query(self.handle, row_ptr, col, col.numel(), True, rho, stream)
        return row_ptr, col[:nnz], rho

    def density(self, row_ptr, col, stream=None):
        import torch
        rho = torch.empty(self.n, dtype=torch.float32, device=self.xyz.device)
        sph_density_sum(self.handle, row_ptr, col, rho, stream)
        return rho

    def check(self, stream=None):
        return sph_grid_check(self.handle, stream)

    def close(self):
        if self.handle:
            sph_grid_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def neighbours(xyz, h, kh=None, order=SPH_ORDER_CANONICAL, precision=SPH_PREC_FP16_RCLL, density=True,
               mass=1.0):
    """One-shot search on a CUDA float64 tensor: returns (row_ptr, col, rho)."""
    g = Grid(xyz, h, kh, order, precision, mass)
    try:
        return g.query(density=density)
    finally:
        g.close()
