"""FP64 CPU oracle for the sub-structured CG (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it, and it
never calls the CUDA library.  The arithmetic lives in ``ssg_oracle.c``
(plain C, -O2 -ffp-contract=off); this module builds it with gcc and wraps it
with ctypes and numpy arrays.  ``cond_from_lanczos`` is the one piece written
here: it forms the Lanczos tridiagonal matrix from the CG coefficients and
takes its extreme eigenvalues with numpy (a library primitive).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ssg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

OK, INVALID, OOM, BREAKDOWN, NOT_CONVERGED = 0, 1, 2, 4, 5
WEIGHT_INV_MULT, WEIGHT_OWNER = 0, 1  # weights of the weighted dots (Partition.set_weights)

_lib = None

_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


_CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c99"]


def build(force: bool = False) -> str:
    """Compile ssg_oracle.c into _build/liboracle.so (gcc, no FMA contraction),
    with OpenMP for or_sub_cg_omp where the compiler has it (without it that
    function runs on one thread with the same results)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        try:
            subprocess.check_call(["gcc"] + _CFLAGS + ["-fopenmp", "-o", tmp, _SRC, "-lm"],
                                  stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(["gcc"] + _CFLAGS + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def compile_variant(src_text: str, tag: str) -> str:
    """Compile a modified copy of the oracle source (used by the tests that
    plant a mistake in the oracle to show that the pins catch it)."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_BUILD, "variant_%s.c" % tag)
    out = os.path.join(_BUILD, "libvariant_%s_%d.so" % (tag, os.getpid()))
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc"] + _CFLAGS + ["-o", out, src, "-lm"])
    return out


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


class use_library:
    """Context manager: route this module's calls to another build of the
    oracle source (a planted-mistake variant) and restore afterwards."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = _bind(C.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(C.CDLL(_LIB))
    return _lib


def _bind(L):
    if L is not None:
        L.or_spmv.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p]
        L.or_spmv.restype = None
        dp = C.POINTER(C.c_double)
        L.or_cg.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, C.c_double, C.c_int32,
                            C.POINTER(C.c_int32), C.POINTER(C.c_double), dp, dp, dp]
        L.or_cg.restype = C.c_int
        L.or_partition.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _i32p, C.c_int32, C.POINTER(C.c_int)]
        L.or_partition.restype = C.c_void_p
        L.or_partition_fe.argtypes = [C.c_int32, C.c_int32, C.c_int32, _i32p, _f64p, _i32p, C.c_int32,
                                      C.POINTER(C.c_int)]
        L.or_partition_fe.restype = C.c_void_p
        L.or_part_free.argtypes = [C.c_void_p]
        L.or_part_sizes.argtypes = [C.c_void_p, np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")]
        L.or_part_copy.argtypes = [C.c_void_p] + [_i32p] * 6 + [_f64p] + [_i32p] * 4 + [_f64p]
        L.or_scatter.argtypes = [C.c_void_p, _f64p, _f64p]
        L.or_gather.argtypes = [C.c_void_p, _f64p, _f64p]
        L.or_sub_spmv.argtypes = [C.c_void_p, _f64p, _f64p]
        L.or_wdot.argtypes = [C.c_void_p, _f64p, _f64p]
        L.or_wdot.restype = C.c_double
        L.or_set_weights.argtypes = [C.c_void_p, C.c_int]
        L.or_set_weights.restype = C.c_int
        L.or_sub_cg.argtypes = [C.c_void_p, _f64p, _f64p, C.c_double, C.c_int32, C.POINTER(C.c_int32),
                                C.POINTER(C.c_double), dp, dp, dp]
        L.or_sub_cg.restype = C.c_int
        L.or_sub_spmv32.argtypes = [C.c_void_p, np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS"),
                                    np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")]
        L.or_sub_cg_mixed.argtypes = [C.c_void_p, _f64p, _f64p, C.c_double, C.c_int32, C.c_double, C.c_int32,
                                      C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_double)]
        L.or_sub_cg_mixed.restype = C.c_int
        L.or_pcg.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, C.c_double, C.c_int32,
                             C.POINTER(C.c_int32), C.POINTER(C.c_double)]
        L.or_pcg.restype = C.c_int
        L.or_sub_pcg.argtypes = [C.c_void_p, _f64p, _f64p, C.c_double, C.c_int32, C.POINTER(C.c_int32),
                                 C.POINTER(C.c_double)]
        L.or_sub_pcg.restype = C.c_int
        L.or_sub_pcg_mixed.argtypes = [C.c_void_p, _f64p, _f64p, C.c_double, C.c_int32, C.c_double, C.c_int32,
                                       C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_double)]
        L.or_sub_pcg_mixed.restype = C.c_int
        L.or_sub_cg_omp.argtypes = [C.c_void_p, _f64p, _f64p, C.c_double, C.c_int32, C.c_int32,
                                    C.POINTER(C.c_int32), C.POINTER(C.c_double)]
        L.or_sub_cg_omp.restype = C.c_int
        L.or_omp_max_threads.argtypes = []
        L.or_omp_max_threads.restype = C.c_int
        L.or_cholesky_solve.argtypes = [C.c_int32, _f64p, _f64p, _f64p]
        L.or_cholesky_solve.restype = C.c_int
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        vp = C.c_void_p
        for f in (L.or_band_row, L.or_band_col):
            f.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_int32, C.c_int32, i64p, vp, vp, vp]
            f.restype = C.c_int
        for f in (L.or_band_row_spmv, L.or_band_col_spmv):
            f.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_int32, _f64p, _f64p]
            f.restype = C.c_int
    return L


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def spmv(A, x):
    """Global CSR product y = A x (Section 1.2 storage, rows summed left to right)."""
    x = _c(x, np.float64)
    y = np.empty(A.n, np.float64)
    lib().or_spmv(A.n, _c(A.rowptr, np.int32), _c(A.colidx, np.int32), _c(A.val, np.float64), x, y)
    return y


@dataclass
class CGResult:
    x: np.ndarray
    status: int
    iters: int
    relres: float
    alpha: np.ndarray
    beta: np.ndarray
    res_hist: np.ndarray


def _hist(n):
    a = np.zeros(max(n, 1), np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def cg(A, b, rtol, max_iter, x0=None) -> CGResult:
    """Algorithm 3 with M = I on the global matrix (see ssg_oracle.c: or_cg)."""
    b = _c(b, np.float64).ravel()
    x = np.zeros(A.n) if x0 is None else _c(x0, np.float64).ravel().copy()
    it = C.c_int32()
    rr = C.c_double()
    ha, pa = _hist(max_iter)
    hb, pb = _hist(max_iter)
    hr, pr = _hist(max_iter)
    st = lib().or_cg(A.n, _c(A.rowptr, np.int32), _c(A.colidx, np.int32), _c(A.val, np.float64), b, x,
                     rtol, max_iter, C.byref(it), C.byref(rr), pa, pb, pr)
    k = it.value
    return CGResult(x, st, k, rr.value, ha[:k].copy(), hb[:k].copy(), hr[:k].copy())


@dataclass
class Maps:
    """Sub-structure data as computed by the oracle partitioner."""

    n: int
    P: int
    nnz: int
    nloc: int
    ngamma: int
    ncopies: int
    off: np.ndarray
    nint: np.ndarray
    l2g: np.ndarray
    mult: np.ndarray
    lrowptr: np.ndarray
    lcol: np.ndarray
    lval: np.ndarray
    gamma: np.ndarray
    iptr: np.ndarray
    icopy: np.ndarray
    own: np.ndarray
    w: np.ndarray


class Partition:
    """Handle on the oracle's sub-structure data (or_partition, or
    or_partition_fe through ``from_elements``)."""

    def __init__(self, A, part, P, _handle=None):
        self.A = A
        st = C.c_int()
        self._L = lib()
        if _handle is None:
            self._rp = _c(A.rowptr, np.int32)
            self._ci = _c(A.colidx, np.int32)
            self._va = _c(A.val, np.float64)
            self._pa = _c(part, np.int32)
            h = self._L.or_partition(A.n, self._rp, self._ci, self._va, self._pa, int(P), C.byref(st))
            self.status = st.value
        else:
            h = _handle
            self.status = OK
        self.h = h
        if not h:
            raise ValueError("oracle partition rejected the input (status %d)" % st.value)
        sz = np.zeros(6, np.int64)
        self._L.or_part_sizes(h, sz)
        n, P_, nnz, nloc, ng, nc = (int(v) for v in sz)
        m = Maps(
            n, P_, nnz, nloc, ng, nc,
            np.zeros(P_ + 1, np.int32), np.zeros(P_, np.int32), np.zeros(nloc, np.int32), np.zeros(n, np.int32),
            np.zeros(nloc + 1, np.int32), np.zeros(nnz, np.int32), np.zeros(nnz, np.float64),
            np.zeros(ng, np.int32), np.zeros(ng + 1, np.int32), np.zeros(nc, np.int32), np.zeros(n, np.int32),
            np.zeros(nloc, np.float64),
        )
        self._L.or_part_copy(h, m.off, m.nint, m.l2g, m.mult, m.lrowptr, m.lcol, m.lval, m.gamma, m.iptr,
                           m.icopy, m.own, m.w)
        self.maps = m

    @classmethod
    def from_elements(cls, n, elem, kel, epart, P):
        """Sub-structures from finite elements (or_partition_fe): elem (ne, nv)
        node ids (-1: eliminated), kel (ne, nv, nv) element matrices, epart (ne)
        subdomain of every element."""
        elem = _c(elem, np.int32)
        ne, nv = elem.shape
        st = C.c_int()
        h = lib().or_partition_fe(int(n), int(ne), int(nv), elem.ravel(), _c(kel, np.float64).ravel(),
                                  _c(epart, np.int32), int(P), C.byref(st))
        if not h:
            raise ValueError("oracle element partition rejected the input (status %d)" % st.value)
        return cls(None, None, P, _handle=h)

    def __del__(self):
        if getattr(self, "h", None):
            self._L.or_part_free(self.h)
            self.h = None

    def scatter(self, xg):
        out = np.empty(self.maps.nloc)
        self._L.or_scatter(self.h, _c(xg, np.float64).ravel(), out)
        return out

    def gather(self, xl):
        out = np.empty(self.maps.n)
        self._L.or_gather(self.h, _c(xl, np.float64), out)
        return out

    def spmv(self, xl):
        """Sub-structured SpMV on concatenated local vectors (Section 3.4.1)."""
        out = np.empty(self.maps.nloc)
        self._L.or_sub_spmv(self.h, _c(xl, np.float64), out)
        return out

    def wdot(self, u, v) -> float:
        return float(self._L.or_wdot(self.h, _c(u, np.float64), _c(v, np.float64)))

    def set_weights(self, mode: int):
        """Weights of every weighted dot of this partition (or_set_weights):
        WEIGHT_INV_MULT (1/m, the default) or WEIGHT_OWNER (1 on the owner copy,
        0 on the others)."""
        if self._L.or_set_weights(self.h, int(mode)) != 0:
            raise ValueError("weight mode must be WEIGHT_INV_MULT or WEIGHT_OWNER")

    def cg(self, b, rtol, max_iter, x0=None) -> CGResult:
        """Sub-structured CG (Algorithm 3, M = I) on global b / x."""
        b = _c(b, np.float64).ravel()
        x = np.zeros(self.maps.n) if x0 is None else _c(x0, np.float64).ravel().copy()
        it = C.c_int32()
        rr = C.c_double()
        ha, pa = _hist(max_iter)
        hb, pb = _hist(max_iter)
        hr, pr = _hist(max_iter)
        st = self._L.or_sub_cg(self.h, b, x, rtol, max_iter, C.byref(it), C.byref(rr), pa, pb, pr)
        k = it.value
        return CGResult(x, st, k, rr.value, ha[:k].copy(), hb[:k].copy(), hr[:k].copy())


def omp_max_threads() -> int:
    """Threads or_sub_cg_omp uses by default (1 when built without OpenMP)."""
    return int(lib().or_omp_max_threads())


def _cg_omp(self, b, rtol, max_iter, nthreads=0, x0=None) -> CGResult:
    """Sub-structured CG with the subdomains shared among OpenMP threads
    (ssg_oracle.c: or_sub_cg_omp); nthreads 0 = all."""
    b = _c(b, np.float64).ravel()
    x = np.zeros(self.maps.n) if x0 is None else _c(x0, np.float64).ravel().copy()
    it = C.c_int32()
    rr = C.c_double()
    st = self._L.or_sub_cg_omp(self.h, b, x, rtol, max_iter, int(nthreads), C.byref(it), C.byref(rr))
    e = np.zeros(0)
    return CGResult(x, st, it.value, rr.value, e, e, e)


Partition.cg_omp = _cg_omp


@dataclass
class MixedResult:
    x: np.ndarray
    status: int
    iters: int
    outer: int
    relres: float


def _mixed(self, b, rtol, max_iter, inner_rtol=1e-4, max_outer=30, x0=None) -> MixedResult:
    """FP32 inner CG inside FP64 iterative refinement (ssg_oracle.c: or_sub_cg_mixed)."""
    b = _c(b, np.float64).ravel()
    x = np.zeros(self.maps.n) if x0 is None else _c(x0, np.float64).ravel().copy()
    it = C.c_int32()
    ou = C.c_int32()
    rr = C.c_double()
    st = self._L.or_sub_cg_mixed(self.h, b, x, rtol, max_iter, inner_rtol, max_outer, C.byref(it), C.byref(ou),
                                 C.byref(rr))
    return MixedResult(x, st, it.value, ou.value, rr.value)


Partition.cg_mixed = _mixed


def _spmv32(self, xl):
    """FP32 sub-structured SpMV (values rounded to FP32, FP32 arithmetic)."""
    out = np.empty(self.maps.nloc, np.float32)
    self._L.or_sub_spmv32(self.h, np.ascontiguousarray(xl, np.float32), out)
    return out


Partition.spmv32 = _spmv32


@dataclass
class PCGResult:
    x: np.ndarray
    status: int
    iters: int
    relres: float


def pcg(A, b, rtol, max_iter, x0=None) -> PCGResult:
    """Algorithm 3 with M = diag(A) on the global matrix (ssg_oracle.c: or_pcg)."""
    b = _c(b, np.float64).ravel()
    x = np.zeros(A.n) if x0 is None else _c(x0, np.float64).ravel().copy()
    it = C.c_int32()
    rr = C.c_double()
    st = lib().or_pcg(A.n, _c(A.rowptr, np.int32), _c(A.colidx, np.int32), _c(A.val, np.float64), b, x, rtol,
                      max_iter, C.byref(it), C.byref(rr))
    return PCGResult(x, st, it.value, rr.value)


def _sub_pcg(self, b, rtol, max_iter, x0=None) -> PCGResult:
    """Sub-structured Algorithm 3 with M = diag(S) (ssg_oracle.c: or_sub_pcg)."""
    b = _c(b, np.float64).ravel()
    x = np.zeros(self.maps.n) if x0 is None else _c(x0, np.float64).ravel().copy()
    it = C.c_int32()
    rr = C.c_double()
    st = self._L.or_sub_pcg(self.h, b, x, rtol, max_iter, C.byref(it), C.byref(rr))
    return PCGResult(x, st, it.value, rr.value)


Partition.pcg = _sub_pcg


def _sub_pcg_mixed(self, b, rtol, max_iter, inner_rtol=1e-4, max_outer=30, x0=None) -> "MixedResult":
    """Mixed refinement with diagonal-preconditioned FP32 inner solves
    (ssg_oracle.c: or_sub_pcg_mixed)."""
    b = _c(b, np.float64).ravel()
    x = np.zeros(self.maps.n) if x0 is None else _c(x0, np.float64).ravel().copy()
    it = C.c_int32()
    ou = C.c_int32()
    rr = C.c_double()
    st = self._L.or_sub_pcg_mixed(self.h, b, x, rtol, max_iter, inner_rtol, max_outer, C.byref(it), C.byref(ou),
                                  C.byref(rr))
    return MixedResult(x, st, it.value, ou.value, rr.value)


Partition.pcg_mixed = _sub_pcg_mixed


@dataclass
class Band:
    """Band p of a band-row (Algorithm 1) or band-column (Algorithm 2)
    splitting: an np x n (row) or n x np (column) CSR matrix starting at
    row / column ``displ`` of A."""

    kind: str
    p: int
    np: int
    displ: int
    rowptr: np.ndarray
    colidx: np.ndarray
    val: np.ndarray


def band(A, kind, nb, p) -> Band:
    """Band p of nb (0-based) of the band-row (kind "row", or_band_row) or
    band-column (kind "col", or_band_col) splitting of A."""
    f = lib().or_band_row if kind == "row" else lib().or_band_col
    args = (A.n, _c(A.rowptr, np.int32), _c(A.colidx, np.int32), _c(A.val, np.float64), int(nb), int(p))
    sz = np.zeros(3, np.int64)
    if f(*args, sz, None, None, None) != OK:
        raise ValueError("oracle band splitting rejected the input")
    npr, displ, nz = (int(v) for v in sz)
    rows = npr if kind == "row" else A.n
    br = np.zeros(rows + 1, np.int32)
    bc = np.zeros(max(nz, 1), np.int32)
    bv = np.zeros(max(nz, 1), np.float64)
    f(*args, sz, br.ctypes.data, bc.ctypes.data, bv.ctypes.data)
    return Band(kind, int(p), npr, displ, br, bc[:nz].copy(), bv[:nz].copy())


def band_spmv(A, kind, nb, x):
    """y = A x through the band-row or band-column splitting with nb bands
    (or_band_row_spmv / or_band_col_spmv)."""
    f = lib().or_band_row_spmv if kind == "row" else lib().or_band_col_spmv
    y = np.zeros(A.n, np.float64)
    st = f(A.n, _c(A.rowptr, np.int32), _c(A.colidx, np.int32), _c(A.val, np.float64), int(nb),
           _c(x, np.float64), y)
    if st != OK:
        raise ValueError("oracle band product rejected the input (status %d)" % st)
    return y


def cholesky_solve(Adense, b):
    """Textbook dense Cholesky solve (or_cholesky_solve)."""
    A = _c(Adense, np.float64)
    n = A.shape[0]
    x = np.zeros(n)
    st = lib().or_cholesky_solve(n, A, _c(b, np.float64).ravel(), x)
    if st != OK:
        raise np.linalg.LinAlgError("oracle Cholesky: not positive definite")
    return x


def cond_from_lanczos(alpha, beta):
    """Estimate kappa(A) from CG coefficients via the Lanczos tridiagonal T.

    T[j, j] = 1/alpha_j + beta_{j-1}/alpha_{j-1},  T[j, j+1] = sqrt(beta_j)/alpha_j
    (the standard CG-Lanczos relation); kappa_est = lambda_max(T)/lambda_min(T).
    """
    a = np.asarray(alpha, np.float64)
    bt = np.asarray(beta, np.float64)
    k = a.size
    if k == 0:
        return 1.0
    d = 1.0 / a
    d[1:] += bt[:-1] / a[:-1]
    e = np.sqrt(bt[:-1]) / a[:-1]
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    ev = np.linalg.eigvalsh(T)
    return float(ev[-1] / ev[0])
