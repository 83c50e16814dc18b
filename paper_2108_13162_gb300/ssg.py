"""ctypes binding of libssg.so (include/ssg.h), same names as the C ABI.

Argument marshalling only: every step of the sub-structured CG runs in the
library's CUDA kernels.  Device vectors are passed as ``torch.Tensor``
(float64, CUDA, contiguous) through ``data_ptr()``; host arrays as numpy
arrays.  The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2108_13162_gb300.build``): there is no fallback, a missing
library raises.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

SSG_OK = 0
SSG_E_INVALID = 1
SSG_E_OOM = 2
SSG_E_CUDA = 3
SSG_E_BREAKDOWN = 4
SSG_E_NOT_CONVERGED = 5
SSG_E_TIMEOUT = 6
SSG_FP64 = 0
SSG_MIXED = 1
SSG_FP64_JACOBI = 2
SSG_MIXED_JACOBI = 3
SSG_WEIGHT_INV_MULT = 0
SSG_WEIGHT_OWNER = 1
SSG_DRIVER_GRAPH = 0
SSG_DRIVER_HOST = 1
SSG_BAND_ROW = 0
SSG_BAND_COL = 1
SSG_BAND_AUTO = 0
SSG_BAND_STAGED = -1

# every entry point declared in include/ssg.h
EXPORTS = (
    "ssg_create",
    "ssg_set_stream",
    "ssg_set_driver",
    "ssg_set_mixed",
    "ssg_set_rhs_block",
    "ssg_set_unroll",
    "ssg_destroy",
    "ssg_partition",
    "ssg_partition_fe",
    "ssg_partition_batch",
    "ssg_solve_batch",
    "ssg_get_sizes",
    "ssg_copy_maps",
    "ssg_scatter",
    "ssg_gather",
    "ssg_spmv_assembled",
    "ssg_spmv_assembled_f32",
    "ssg_autotune",
    "ssg_spmm_assembled",
    "ssg_spmm_assembled_f32",
    "ssg_wdot",
    "ssg_solve",
    "ssg_solve_host",
    "ssg_set_values",
    "ssg_pattern_grad",
    "ssg_fv7_values",
    "ssg_fv7_adjoint",
    "ssg_system_destroy",
    "ssg_error_string",
    "ssg_last_error",
    "ssg_wdot_noalloc",
    "ssg_set_batch_graph",
    "ssg_measure_fp64_rate",
    "ssg_set_slice_sort",
    "ssg_set_weights",
    "ssg_set_cluster_solve",
    "ssg_get_cluster_solve",
    "ssg_get_layout",
    "ssg_get_iface_layout",
    "ssg_autotune_block",
    "ssg_band_split",
    "ssg_band_get",
    "ssg_band_spmv",
    "ssg_band_set_variant",
    "ssg_band_autotune",
    "ssg_band_check_timeout",
    "ssg_band_destroy",
)


class ssg_sizes(C.Structure):
    _fields_ = [
        ("n", C.c_int32),
        ("P", C.c_int32),
        ("nnz", C.c_int64),
        ("nloc", C.c_int64),
        ("ngamma", C.c_int32),
        ("max_mult", C.c_int32),
        ("ncopies", C.c_int64),
    ]


class ssg_stats(C.Structure):
    _fields_ = [
        ("status", C.c_int32),
        ("iters", C.c_int32),
        ("outer", C.c_int32),
        ("block", C.c_int32),
        ("relres", C.c_double),
        ("true_relres", C.c_double),
        ("solve_ms", C.c_double),
        ("kernel_launches", C.c_int64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


TUNE_CANDIDATES = 6  # SSG_TUNE_CANDIDATES


class ssg_tune(C.Structure):
    _fields_ = [
        ("fp64_choice", C.c_int32),
        ("fp32_choice", C.c_int32),
        ("fp64_blocks_per_sm", C.c_int32 * TUNE_CANDIDATES),
        ("fp64_l2_ahead", C.c_int32 * TUNE_CANDIDATES),
        ("fp32_blocks_per_sm", C.c_int32 * TUNE_CANDIDATES),
        ("fp32_l2_ahead", C.c_int32 * TUNE_CANDIDATES),
        ("fp64_us", C.c_double * TUNE_CANDIDATES),
        ("fp32_us", C.c_double * TUNE_CANDIDATES),
    ]

    def as_dict(self):
        return {f: (list(getattr(self, f)) if not isinstance(getattr(self, f), int) else getattr(self, f))
                for f, _ in self._fields_}


TUNE_BLOCK_CANDIDATES = 6  # SSG_TUNE_BLOCK_CANDIDATES


class ssg_tune_block(C.Structure):
    _fields_ = [
        ("k", C.c_int32),
        ("fp64_choice", C.c_int32),
        ("fp32_choice", C.c_int32),
        ("nc", C.c_int32 * TUNE_BLOCK_CANDIDATES),
        ("l2_ahead", C.c_int32 * TUNE_BLOCK_CANDIDATES),
        ("fp64_us", C.c_double * TUNE_BLOCK_CANDIDATES),
        ("fp32_us", C.c_double * TUNE_BLOCK_CANDIDATES),
    ]

    def as_dict(self):
        return {f: (list(getattr(self, f)) if not isinstance(getattr(self, f), int) else getattr(self, f))
                for f, _ in self._fields_}


class ssg_band_tune(C.Structure):
    _fields_ = [
        ("variant", C.c_int32),
        ("rule_variant", C.c_int32),
        ("code", C.c_int32 * 7),
        ("us", C.c_float * 7),
    ]

    def as_dict(self):
        return {"variant": self.variant, "rule_variant": self.rule_variant,
                "us": {int(c): float(u) for c, u in zip(self.code, self.us) if u > 0}}


class SSGError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s failed: %s (%s)" % (where, _lib_or_none_str(status), last_error()))


_lib = None


def _lib_or_none_str(status):
    try:
        return lib().ssg_error_string(status).decode()
    except Exception:  # noqa: BLE001
        return "status %d" % status


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libssg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libssg.so is not built (%s); run __graft_entry__.build()" % path)
        L = C.CDLL(path)
        vp = C.c_void_p
        i32 = C.c_int32
        L.ssg_create.argtypes = [C.POINTER(vp), C.c_int, vp]
        L.ssg_set_stream.argtypes = [vp, vp]
        L.ssg_set_driver.argtypes = [vp, C.c_int]
        L.ssg_set_mixed.argtypes = [vp, C.c_double, C.c_int32]
        L.ssg_set_rhs_block.argtypes = [vp, C.c_int32]
        L.ssg_set_unroll.argtypes = [vp, C.c_int32]
        L.ssg_destroy.argtypes = [vp]
        L.ssg_partition.argtypes = [vp, i32, vp, vp, vp, vp, i32, C.POINTER(vp)]
        L.ssg_partition_batch.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, C.POINTER(vp)]
        L.ssg_partition_fe.argtypes = [vp, i32, i32, i32, vp, vp, vp, i32, C.POINTER(vp)]
        L.ssg_solve_batch.argtypes = [vp, vp, vp, i32, C.c_double, i32, i32, C.POINTER(ssg_stats)]
        L.ssg_get_sizes.argtypes = [vp, C.POINTER(ssg_sizes)]
        L.ssg_copy_maps.argtypes = [vp] * 12
        L.ssg_scatter.argtypes = [vp, vp, vp]
        L.ssg_gather.argtypes = [vp, vp, vp]
        L.ssg_spmv_assembled.argtypes = [vp, vp, vp, vp]
        L.ssg_spmv_assembled_f32.argtypes = [vp, vp, vp, vp]
        L.ssg_wdot.argtypes = [vp, vp, vp, vp]
        L.ssg_spmm_assembled.argtypes = [vp, i32, vp, vp]
        L.ssg_autotune.argtypes = [vp, i32, C.POINTER(ssg_tune)]
        L.ssg_set_values.argtypes = [vp, vp]
        L.ssg_pattern_grad.argtypes = [vp, i32, vp, vp, vp]
        L.ssg_fv7_values.argtypes = [vp, i32, i32, i32, vp, vp]
        L.ssg_fv7_adjoint.argtypes = [vp, i32, i32, i32, vp, vp, vp]
        L.ssg_spmm_assembled_f32.argtypes = [vp, i32, vp, vp]
        L.ssg_solve.argtypes = [vp, i32, vp, vp, i32, C.c_double, i32, i32, C.POINTER(ssg_stats)]
        L.ssg_solve_host.argtypes = [vp, i32, vp, vp, i32, C.c_double, i32, i32, C.POINTER(ssg_stats)]
        L.ssg_system_destroy.argtypes = [vp]
        L.ssg_wdot_noalloc.argtypes = [vp, vp, vp, C.c_int64, vp, vp]
        L.ssg_set_batch_graph.argtypes = [vp, C.c_int32]
        L.ssg_set_slice_sort.argtypes = [vp, C.c_int32]
        L.ssg_set_weights.argtypes = [vp, C.c_int32]
        L.ssg_set_cluster_solve.argtypes = [vp, C.c_int64, C.c_int32]
        L.ssg_get_cluster_solve.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
        L.ssg_autotune_block.argtypes = [vp, C.c_int32, C.c_int32, C.POINTER(ssg_tune_block)]
        L.ssg_get_layout.argtypes = [vp, np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")]
        L.ssg_get_iface_layout.argtypes = [vp, np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")]
        L.ssg_measure_fp64_rate.argtypes = [vp, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                            C.POINTER(C.c_double)]
        L.ssg_band_split.argtypes = [vp, i32, i32, vp, vp, vp, i32, C.POINTER(vp)]
        L.ssg_band_get.argtypes = [vp, i32, vp, vp, vp, vp]
        L.ssg_band_spmv.argtypes = [vp, vp, vp]
        L.ssg_band_set_variant.argtypes = [vp, i32]
        L.ssg_band_autotune.argtypes = [vp, i32, C.POINTER(ssg_band_tune)]
        L.ssg_band_check_timeout.argtypes = [vp]
        L.ssg_band_destroy.argtypes = [vp]
        L.ssg_error_string.argtypes = [C.c_int]
        L.ssg_error_string.restype = C.c_char_p
        L.ssg_last_error.argtypes = []
        L.ssg_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("ssg_error_string", "ssg_last_error"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def last_error() -> str:
    return lib().ssg_last_error().decode(errors="replace")


def _check(rc, where, ok=(SSG_OK,)):
    if rc not in ok:
        raise SSGError(rc, where)
    return rc


def _ptr(t):
    """Device (torch) or host (numpy) buffer -> address; None -> NULL."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags.c_contiguous
        return t.ctypes.data
    assert t.is_contiguous(), "tensors passed to the library must be contiguous"
    return t.data_ptr()


def _dev_f64(t):
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


# ------------------------------------------------------------------ thin wrappers (same names)
def ssg_create(device: int = 0, stream=None):
    h = C.c_void_p()
    _check(lib().ssg_create(C.byref(h), device, stream), "ssg_create")
    return h


def ssg_set_stream(ctx, stream):
    return _check(lib().ssg_set_stream(ctx, stream), "ssg_set_stream")


def ssg_set_driver(ctx, driver: int):
    return _check(lib().ssg_set_driver(ctx, driver), "ssg_set_driver")


def ssg_set_mixed(ctx, inner_rtol: float, max_outer: int):
    return _check(lib().ssg_set_mixed(ctx, inner_rtol, max_outer), "ssg_set_mixed")


def ssg_set_rhs_block(ctx, kmax: int):
    return _check(lib().ssg_set_rhs_block(ctx, kmax), "ssg_set_rhs_block")


def ssg_set_unroll(ctx, iters: int):
    return _check(lib().ssg_set_unroll(ctx, int(iters)), "ssg_set_unroll")


def ssg_destroy(ctx):
    return lib().ssg_destroy(ctx)


def ssg_partition(ctx, n, rowptr, colidx, val, part, P):
    rowptr = np.ascontiguousarray(rowptr, np.int32)
    colidx = np.ascontiguousarray(colidx, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    part = np.ascontiguousarray(part, np.int32)
    if rowptr.size != n + 1 or part.size != n or colidx.size != val.size or colidx.size < rowptr[-1]:
        raise ValueError("CSR/partition arrays have inconsistent sizes")
    h = C.c_void_p()
    _check(
        lib().ssg_partition(ctx, n, _ptr(rowptr), _ptr(colidx), _ptr(val), _ptr(part), P, C.byref(h)),
        "ssg_partition",
    )
    return h


def ssg_partition_fe(ctx, n, elem, kel, epart, P):
    elem = np.ascontiguousarray(elem, np.int32)
    kel = np.ascontiguousarray(kel, np.float64)
    epart = np.ascontiguousarray(epart, np.int32)
    ne, nv = elem.shape
    if kel.shape != (ne, nv, nv) or epart.size != ne:
        raise ValueError("element arrays have inconsistent sizes")
    h = C.c_void_p()
    _check(lib().ssg_partition_fe(ctx, n, ne, nv, _ptr(elem), _ptr(kel), _ptr(epart), P, C.byref(h)),
           "ssg_partition_fe")
    return h


def ssg_partition_batch(ctx, sys_node_off, sys_sub_off, sys_nrhs, rowptr, colidx, val, part):
    node_off = np.ascontiguousarray(sys_node_off, np.int32)
    sub_off = np.ascontiguousarray(sys_sub_off, np.int32)
    nrhs = np.ascontiguousarray(sys_nrhs, np.int32)
    rowptr = np.ascontiguousarray(rowptr, np.int32)
    colidx = np.ascontiguousarray(colidx, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    part = np.ascontiguousarray(part, np.int32)
    nsys = nrhs.size
    n = int(node_off[-1])
    if node_off.size != nsys + 1 or sub_off.size != nsys + 1 or rowptr.size != n + 1 or part.size != n \
            or colidx.size != val.size or colidx.size < rowptr[-1]:
        raise ValueError("batch tables / CSR arrays have inconsistent sizes")
    h = C.c_void_p()
    _check(lib().ssg_partition_batch(ctx, nsys, _ptr(node_off), _ptr(sub_off), _ptr(nrhs), _ptr(rowptr),
                                     _ptr(colidx), _ptr(val), _ptr(part), C.byref(h)), "ssg_partition_batch")
    return h


def ssg_solve_batch(sys, nstats, b, x, x_is_guess=False, rtol=1e-8, max_iter=0, mode=SSG_FP64):
    """Batch solve (device buffers); returns (status, stats per (system, right-hand side))."""
    st = (ssg_stats * nstats)()
    rc = lib().ssg_solve_batch(sys, _dev_f64(b), _dev_f64(x), int(bool(x_is_guess)), rtol, max_iter, mode, st)
    _check(rc, "ssg_solve_batch", ok=(SSG_OK, SSG_E_BREAKDOWN, SSG_E_NOT_CONVERGED))
    return rc, [st[i].as_dict() for i in range(nstats)]


def ssg_get_sizes(sys):
    s = ssg_sizes()
    _check(lib().ssg_get_sizes(sys, C.byref(s)), "ssg_get_sizes")
    return s


def ssg_copy_maps(sys):
    s = ssg_get_sizes(sys)
    out = {
        "off": np.zeros(s.P + 1, np.int32),
        "nint": np.zeros(s.P, np.int32),
        "l2g": np.zeros(s.nloc, np.int32),
        "mult": np.zeros(s.n, np.int32),
        "lrowptr": np.zeros(s.nloc + 1, np.int32),
        "lcol": np.zeros(s.nnz, np.int32),
        "lval": np.zeros(s.nnz, np.float64),
        "gamma": np.zeros(s.ngamma, np.int32),
        "iptr": np.zeros(s.ngamma + 1, np.int32),
        "icopy": np.zeros(s.ncopies, np.int32),
        "own": np.zeros(s.n, np.int32),
    }
    keys = ("off", "nint", "l2g", "mult", "lrowptr", "lcol", "lval", "gamma", "iptr", "icopy", "own")
    _check(lib().ssg_copy_maps(sys, *[_ptr(out[k]) for k in keys]), "ssg_copy_maps")
    return out


def ssg_scatter(sys, x_glob, x_loc):
    return _check(lib().ssg_scatter(sys, _dev_f64(x_glob), _dev_f64(x_loc)), "ssg_scatter")


def ssg_gather(sys, x_loc, x_glob):
    return _check(lib().ssg_gather(sys, _dev_f64(x_loc), _dev_f64(x_glob)), "ssg_gather")


def ssg_spmv_assembled(sys, x_loc, y_loc, xSx=None):
    return _check(
        lib().ssg_spmv_assembled(sys, _dev_f64(x_loc), _dev_f64(y_loc), None if xSx is None else _dev_f64(xSx)),
        "ssg_spmv_assembled",
    )


def _dev_f32(t):
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return t.data_ptr()


def ssg_spmv_assembled_f32(sys, x_loc, y_loc, xSx=None):
    return _check(
        lib().ssg_spmv_assembled_f32(sys, _dev_f32(x_loc), _dev_f32(y_loc), None if xSx is None else _dev_f64(xSx)),
        "ssg_spmv_assembled_f32",
    )


def ssg_autotune(sys, reps=20):
    t = ssg_tune()
    _check(lib().ssg_autotune(sys, reps, C.byref(t)), "ssg_autotune")
    return t.as_dict()


def ssg_autotune_block(sys, k=16, reps=20):
    t = ssg_tune_block()
    _check(lib().ssg_autotune_block(sys, int(k), int(reps), C.byref(t)), "ssg_autotune_block")
    return t.as_dict()


def ssg_band_split(ctx, kind, n, rowptr, colidx, val, nb):
    rowptr = np.ascontiguousarray(rowptr, np.int32)
    colidx = np.ascontiguousarray(colidx, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    if rowptr.size != n + 1 or colidx.size != val.size or colidx.size < rowptr[-1]:
        raise ValueError("CSR arrays have inconsistent sizes")
    h = C.c_void_p()
    _check(lib().ssg_band_split(ctx, kind, n, _ptr(rowptr), _ptr(colidx), _ptr(val), nb, C.byref(h)),
           "ssg_band_split")
    return h


def ssg_band_get(band, p, n_rows_total):
    """Band p's CSR arrays (host): returns (N_p, displ, rowptr, colidx, val).
    n_rows_total: the band's row count, N_p (band-row) or n (band-column),
    is found from a first call with NULL arrays."""
    sz = np.zeros(3, np.int64)
    _check(lib().ssg_band_get(band, p, _ptr(sz), None, None, None), "ssg_band_get")
    rows = int(sz[0]) if n_rows_total is None else n_rows_total
    rp = np.zeros(rows + 1, np.int32)
    ci = np.zeros(max(int(sz[2]), 1), np.int32)
    va = np.zeros(max(int(sz[2]), 1), np.float64)
    _check(lib().ssg_band_get(band, p, _ptr(sz), _ptr(rp), _ptr(ci), _ptr(va)), "ssg_band_get")
    nz = int(sz[2])
    return int(sz[0]), int(sz[1]), rp, ci[:nz].copy(), va[:nz].copy()


def ssg_band_spmv(band, x, y):
    return _check(lib().ssg_band_spmv(band, _dev_f64(x), _dev_f64(y)), "ssg_band_spmv")


def ssg_band_set_variant(band, variant):
    return _check(lib().ssg_band_set_variant(band, variant), "ssg_band_set_variant")


def ssg_band_autotune(band, reps=20):
    t = ssg_band_tune()
    _check(lib().ssg_band_autotune(band, reps, C.byref(t)), "ssg_band_autotune")
    return t.as_dict()


def ssg_band_check_timeout(band):
    """Status of the bounded-wait failure path (SSG_E_TIMEOUT when it works)."""
    return lib().ssg_band_check_timeout(band)


def ssg_band_destroy(band):
    return _check(lib().ssg_band_destroy(band), "ssg_band_destroy")


def ssg_spmm_assembled(sys, k, x_loc, y_loc):
    return _check(lib().ssg_spmm_assembled(sys, k, _dev_f64(x_loc), _dev_f64(y_loc)), "ssg_spmm_assembled")


def ssg_spmm_assembled_f32(sys, k, x_loc, y_loc):
    return _check(lib().ssg_spmm_assembled_f32(sys, k, _dev_f32(x_loc), _dev_f32(y_loc)), "ssg_spmm_assembled_f32")


def ssg_set_values(sys, val):
    return _check(lib().ssg_set_values(sys, _dev_f64(val)), "ssg_set_values")


def ssg_pattern_grad(sys, k, lam, x, g):
    return _check(lib().ssg_pattern_grad(sys, k, _dev_f64(lam), _dev_f64(x), _dev_f64(g)), "ssg_pattern_grad")


def ssg_fv7_values(sys, nx, ny, nz, logk, val):
    return _check(lib().ssg_fv7_values(sys, nx, ny, nz, _dev_f64(logk), _dev_f64(val)), "ssg_fv7_values")


def ssg_fv7_adjoint(sys, nx, ny, nz, logk, g, glogk):
    return _check(lib().ssg_fv7_adjoint(sys, nx, ny, nz, _dev_f64(logk), _dev_f64(g), _dev_f64(glogk)),
                  "ssg_fv7_adjoint")


def ssg_wdot(sys, u_loc, v_loc, out):
    return _check(lib().ssg_wdot(sys, _dev_f64(u_loc), _dev_f64(v_loc), _dev_f64(out)), "ssg_wdot")


def ssg_solve(sys, k, b, x, x_is_guess=False, rtol=1e-8, max_iter=0, mode=SSG_FP64):
    """Device solve; returns (status, [stats per RHS])."""
    st = (ssg_stats * k)()
    rc = lib().ssg_solve(sys, k, _dev_f64(b), _dev_f64(x), int(bool(x_is_guess)), rtol, max_iter, mode, st)
    _check(rc, "ssg_solve", ok=(SSG_OK, SSG_E_BREAKDOWN, SSG_E_NOT_CONVERGED))
    return rc, [st[i].as_dict() for i in range(k)]


def ssg_solve_host(sys, k, b_host, x_host, x_is_guess=False, rtol=1e-8, max_iter=0, mode=SSG_FP64):
    """Host-buffer solve (copies inside the call); returns (status, stats)."""
    assert b_host.dtype == np.float64 and x_host.dtype == np.float64
    st = (ssg_stats * k)()
    rc = lib().ssg_solve_host(sys, k, _ptr(b_host), _ptr(x_host), int(bool(x_is_guess)), rtol, max_iter, mode, st)
    _check(rc, "ssg_solve_host", ok=(SSG_OK, SSG_E_BREAKDOWN, SSG_E_NOT_CONVERGED))
    return rc, [st[i].as_dict() for i in range(k)]


def noalloc_wdot_args(u_loc, v_loc, mult_loc, out):
    """Checks the arguments of ssg_wdot_noalloc before anything reaches the
    library, which cannot see buffer lengths or devices: u_loc, v_loc (float64)
    and mult_loc (uint8) must be contiguous with one common length, out a
    float64 tensor of at least one element, and all four on the current CUDA
    device.  Raises TypeError (wrong kind of tensor) or ValueError (lengths,
    layout, device); returns nloc."""
    import torch

    named = (("u_loc", u_loc, torch.float64), ("v_loc", v_loc, torch.float64),
             ("mult_loc", mult_loc, torch.uint8), ("out", out, torch.float64))
    for name, t, dt in named:
        if not isinstance(t, torch.Tensor):
            raise TypeError("%s must be a torch tensor" % name)
        if t.dtype != dt:
            raise TypeError("%s must have dtype %s, not %s" % (name, dt, t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    n = u_loc.numel()
    if v_loc.numel() != n or mult_loc.numel() != n:
        raise ValueError("u_loc, v_loc and mult_loc must have the same length (%d, %d, %d)"
                         % (n, v_loc.numel(), mult_loc.numel()))
    if out.numel() < 1:
        raise ValueError("out must hold at least one element")
    for name, t, _ in named:
        if not t.is_cuda:
            raise TypeError("%s must be a CUDA tensor" % name)
    dev = torch.cuda.current_device()
    for name, t, _ in named:
        if t.device.index != dev:
            raise ValueError("%s is on cuda:%d, the current device is cuda:%d" % (name, t.device.index, dev))
    return n


def ssg_wdot_noalloc(u_loc, v_loc, mult_loc, out, stream=None):
    """Weighted dot with no device allocation in the library (see ssg.h)."""
    n = noalloc_wdot_args(u_loc, v_loc, mult_loc, out)
    return _check(
        lib().ssg_wdot_noalloc(u_loc.data_ptr(), v_loc.data_ptr(), mult_loc.data_ptr(), n, out.data_ptr(), stream),
        "ssg_wdot_noalloc",
    )


def ssg_set_batch_graph(sys, one_graph: bool):
    return _check(lib().ssg_set_batch_graph(sys, int(bool(one_graph))), "ssg_set_batch_graph")


def ssg_measure_fp64_rate(ctx, iters: int = 20000, reps: int = 3):
    """(TFLOP/s, best launch ms) of the FP64 FMA rate probe (see ssg.h)."""
    t = C.c_double()
    ms = C.c_double()
    _check(lib().ssg_measure_fp64_rate(ctx, int(iters), int(reps), C.byref(t), C.byref(ms)), "ssg_measure_fp64_rate")
    return t.value, ms.value


def ssg_set_slice_sort(ctx, window: int):
    return _check(lib().ssg_set_slice_sort(ctx, int(window)), "ssg_set_slice_sort")


def ssg_set_cluster_solve(ctx, max_nloc: int, ctas: int = 0):
    return _check(lib().ssg_set_cluster_solve(ctx, int(max_nloc), int(ctas)), "ssg_set_cluster_solve")


def ssg_get_cluster_solve(ctx) -> tuple:
    """(max_nloc, CTAs per cluster) of the one-cluster solve (see ssg.h)."""
    n = C.c_int64(0)
    c = C.c_int32(0)
    _check(lib().ssg_get_cluster_solve(ctx, C.byref(n), C.byref(c)), "ssg_get_cluster_solve")
    return int(n.value), int(c.value)


def ssg_set_weights(sys, mode: int):
    return _check(lib().ssg_set_weights(sys, int(mode)), "ssg_set_weights")


def ssg_get_layout(sys) -> dict:
    """The interior slice layout of a system (see ssg.h)."""
    out = np.zeros(4, np.int64)
    _check(lib().ssg_get_layout(sys, out), "ssg_get_layout")
    return {"slice_slots": int(out[0]), "slice_entries": int(out[1]), "sorted_subdomains": int(out[2]),
            "max_window": int(out[3]), "padding_ratio": float(out[0]) / max(int(out[1]), 1)}


def ssg_get_iface_layout(sys) -> dict:
    """The interface layout of a system's products (see ssg.h)."""
    out = np.zeros(3, np.int64)
    _check(lib().ssg_get_iface_layout(sys, out), "ssg_get_iface_layout")
    return {"iface_slots": int(out[0]), "group_slots": int(out[1]), "groups": bool(out[2])}


def ssg_system_destroy(sys):
    return lib().ssg_system_destroy(sys)


def ssg_error_string(status: int) -> str:
    return lib().ssg_error_string(status).decode()


def ssg_last_error() -> str:
    return last_error()


# ------------------------------------------------------------------ convenience object
@dataclass
class Sizes:
    n: int
    P: int
    nnz: int
    nloc: int
    ngamma: int
    max_mult: int
    ncopies: int


class Context:
    """Owns an ssg_ctx on a CUDA device; work goes to the given torch stream
    (default: the current stream at creation)."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the sub-structured CG library needs a CUDA device")
        torch.cuda.set_device(device)
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.device = device
        self.h = ssg_create(device, C.c_void_p(stream.cuda_stream))

    def set_driver(self, driver: int):
        ssg_set_driver(self.h, driver)

    def set_unroll(self, iters: int):
        """CG iterations per pass of a single-vector loop graph's body (systems partitioned afterwards)."""
        ssg_set_unroll(self.h, iters)

    def set_slice_sort(self, window: int = 0):
        """Interior slice layout: 0 auto, 1 none, > 1 sorting window, -1 whole subdomain
        (systems partitioned afterwards)."""
        ssg_set_slice_sort(self.h, window)

    def set_cluster_solve(self, max_nloc: int = 12288, ctas: int = 0):
        """Single-vector FP64 solves of systems with at most max_nloc local entries
        run as one thread-block cluster (0: never) of ctas CTAs (0: the device's
        largest; systems partitioned afterwards)."""
        ssg_set_cluster_solve(self.h, max_nloc, ctas)

    def cluster_solve(self) -> tuple:
        """(max_nloc, CTAs per cluster; 0 when the device places none)."""
        return ssg_get_cluster_solve(self.h)

    def set_mixed(self, inner_rtol: float = 1e-4, max_outer: int = 30):
        ssg_set_mixed(self.h, inner_rtol, max_outer)

    def set_rhs_block(self, kmax: int = 16):
        """Right-hand sides of one solve call that iterate together (1, 2, 4, 8, 16)."""
        ssg_set_rhs_block(self.h, kmax)

    def close(self):
        """Free the context once no System created on it is alive (the C
        library refuses earlier; a System keeps its Context referenced)."""
        if getattr(self, "h", None):
            if ssg_destroy(self.h) == SSG_OK:
                self.h = None

    def __del__(self):
        self.close()


class Batch:
    """Independent systems solved together (ssg_partition_batch / ssg_solve_batch).

    systems: list of (A, part, P, nrhs) with part in 0..P-1 per system."""

    def __init__(self, ctx: Context, systems):
        import scipy.sparse as sp

        self.ctx = ctx
        ns = [A.n for A, _, _, _ in systems]
        Ps = [P for _, _, P, _ in systems]
        self.nrhs = [int(k) for _, _, _, k in systems]
        self.node_off = np.concatenate([[0], np.cumsum(ns)]).astype(np.int32)
        self.sub_off = np.concatenate([[0], np.cumsum(Ps)]).astype(np.int32)
        U = sp.block_diag([A.to_scipy() for A, _, _, _ in systems], format="csr")
        U.sort_indices()
        part = np.concatenate([np.asarray(pt, np.int32) + self.sub_off[s]
                               for s, (_, pt, _, _) in enumerate(systems)])
        self.h = ssg_partition_batch(ctx.h, self.node_off, self.sub_off, self.nrhs, U.indptr, U.indices, U.data, part)
        self.rhs_off = np.concatenate([[0], np.cumsum([k * n for k, n in zip(self.nrhs, ns)])]).astype(np.int64)
        s = ssg_get_sizes(self.h)
        self.sizes = Sizes(s.n, s.P, s.nnz, s.nloc, s.ngamma, s.max_mult, s.ncopies)

    def set_weights(self, mode: int = SSG_WEIGHT_INV_MULT):
        """Weights of the weighted dots of every system of the batch."""
        ssg_set_weights(self.h, mode)

    def autotune_block(self, reps=20):
        """Tune every column group's K-vector product."""
        return ssg_autotune_block(self.h, 16, reps)

    def solve(self, b, x=None, rtol=1e-8, max_iter=0, mode=SSG_FP64):
        """b: float64 CUDA tensor of rhs_off[-1] values (system s's right-hand
        side j at rhs_off[s] + j * n_s); returns (x, status, stats)."""
        import torch

        if b.numel() != int(self.rhs_off[-1]) or (x is not None and x.numel() != b.numel()):
            raise ValueError("b (and x) must hold %d values" % int(self.rhs_off[-1]))
        guess = x is not None
        xx = torch.zeros_like(b) if x is None else x.clone()
        rc, st = ssg_solve_batch(self.h, int(sum(self.nrhs)), b.contiguous(), xx, guess, rtol, max_iter, mode)
        return xx, rc, st

    def close(self):
        if getattr(self, "h", None):
            ssg_system_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


class Band:
    """Band-row (kind SSG_BAND_ROW) or band-column (SSG_BAND_COL) splitting of
    A into nb bands (ssg_band_split), with its product y = A x."""

    def __init__(self, ctx: Context, A, kind, nb):
        self.ctx = ctx
        self.n = A.n
        self.kind = kind
        self.nb = nb
        self.h = ssg_band_split(ctx.h, kind, A.n, A.rowptr, A.colidx, A.val, nb)

    def band(self, p):
        """(N_p, displ, rowptr, colidx, val) of band p (host arrays)."""
        return ssg_band_get(self.h, p, None if self.kind == SSG_BAND_ROW else self.n)

    def spmv(self, x, out=None):
        import torch

        out = torch.empty(self.n, dtype=torch.float64, device=x.device) if out is None else out
        ssg_band_spmv(self.h, x, out)
        return out

    def set_variant(self, variant):
        ssg_band_set_variant(self.h, variant)

    def autotune(self, reps=20):
        return ssg_band_autotune(self.h, reps)

    def close(self):
        if getattr(self, "h", None):
            ssg_band_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


class System:
    """A partitioned system (ssg_partition, or ssg_partition_fe through
    ``from_elements``) with device-side operators."""

    def __init__(self, ctx: Context | None, A, part, P, _handle=None):
        self.ctx = ctx
        self.h = _handle if _handle is not None else ssg_partition(None if ctx is None else ctx.h, A.n, A.rowptr,
                                                                    A.colidx, A.val, part, P)
        s = ssg_get_sizes(self.h)
        self.sizes = Sizes(s.n, s.P, s.nnz, s.nloc, s.ngamma, s.max_mult, s.ncopies)

    @classmethod
    def from_elements(cls, ctx: Context | None, n, elem, kel, epart, P):
        """Sub-structures from finite elements: elem (ne, nv) node ids (-1 for
        an eliminated node), kel (ne, nv, nv) element matrices, epart (ne)."""
        return cls(ctx, None, None, P, _handle=ssg_partition_fe(None if ctx is None else ctx.h, n, elem, kel, epart, P))

    def maps(self):
        return ssg_copy_maps(self.h)

    def _empty_loc(self):
        import torch

        return torch.empty(self.sizes.nloc, dtype=torch.float64, device="cuda:%d" % self.ctx.device)

    def scatter(self, x_glob, out=None):
        out = self._empty_loc() if out is None else out
        ssg_scatter(self.h, x_glob, out)
        return out

    def gather(self, x_loc, out=None):
        import torch

        out = torch.empty(self.sizes.n, dtype=torch.float64, device=x_loc.device) if out is None else out
        ssg_gather(self.h, x_loc, out)
        return out

    def spmv(self, x_loc, out=None, xSx=None):
        out = self._empty_loc() if out is None else out
        ssg_spmv_assembled(self.h, x_loc, out, xSx)
        return out

    def layout(self):
        return ssg_get_layout(self.h)

    def iface_layout(self):
        return ssg_get_iface_layout(self.h)

    def set_weights(self, mode: int = SSG_WEIGHT_INV_MULT):
        """Weights of the weighted dots: SSG_WEIGHT_INV_MULT (1/m) or SSG_WEIGHT_OWNER."""
        ssg_set_weights(self.h, mode)

    def autotune_block(self, k=16, reps=20):
        """Tune the k-vector product of the several-right-hand-side solves."""
        return ssg_autotune_block(self.h, k, reps)

    def autotune(self, reps=20):
        """Pick the fastest single-vector SpMV instances for this system."""
        return ssg_autotune(self.h, reps)

    def spmm(self, x_loc, out=None):
        """Product with k vectors: x_loc is an (nloc, k) CUDA tensor (row-major,
        i.e. interleaved), float64 or float32; k = 2, 4, 8 or 16."""
        import torch

        k = x_loc.shape[1]
        out = torch.empty_like(x_loc) if out is None else out
        if x_loc.dtype == torch.float32:
            ssg_spmm_assembled_f32(self.h, k, x_loc, out)
        else:
            ssg_spmm_assembled(self.h, k, x_loc, out)
        return out

    def spmv_prec(self, x_loc, out, prec="fp64", xSx=None):
        """Sub-structured SpMV in FP64 (prec="fp64") or FP32 ("fp32")."""
        if prec == "fp32":
            ssg_spmv_assembled_f32(self.h, x_loc, out, xSx)
        else:
            ssg_spmv_assembled(self.h, x_loc, out, xSx)
        return out

    def wdot(self, u, v, out=None):
        import torch

        out = torch.empty(1, dtype=torch.float64, device=u.device) if out is None else out
        ssg_wdot(self.h, u, v, out)
        return out

    def solve(self, b, x=None, rtol=1e-8, max_iter=0, mode=SSG_FP64):
        """b: CUDA float64 (n,) or (k, n) tensor; returns (x, status, stats)."""
        import torch

        bb = b.reshape(-1, self.sizes.n).contiguous()
        k = bb.shape[0]
        guess = x is not None
        xx = torch.zeros_like(bb) if x is None else x.reshape(-1, self.sizes.n).contiguous()
        rc, st = ssg_solve(self.h, k, bb, xx, guess, rtol, max_iter, mode)
        return xx.reshape(b.shape), rc, st

    def solve_host(self, b_host, x_host, rtol=1e-8, max_iter=0, mode=SSG_FP64, x_is_guess=False):
        k = b_host.size // self.sizes.n
        return ssg_solve_host(self.h, k, b_host, x_host, x_is_guess, rtol, max_iter, mode)

    def close(self):
        if getattr(self, "h", None):
            ssg_system_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()
