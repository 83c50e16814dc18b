"""Pins for the oracle pieces the GPU tests lean on besides the FP64 method:
the FP32 sub-structured product (the checker of the FP32 kernels and of the
mixed-precision mode), the condition-number estimate from the CG coefficients
(which scales every "2 kappa rtol" bound), the finite-volume generators (the
reference of the differentiable assembly), and the inner iteration counts of
the mixed refinement.  Each is checked against facts the mathematics fixes,
not against its own formula, and planted mistakes must each break a pin.

FP32 product (Section 3.4.1 in FP32 arithmetic):
  F1 exact on integer data: with small integer values and an integer x every
     FP32 product and partial sum is exact, so the sub-structured FP32 product
     equals the global integer product A x (int64) exactly.
  F2 rounding bound against the global FP64 product:
     |y32_i - (A x)_i| <= 4 (L_i + m_i) 2^-24 (|A||x|)_i.
  F3 every copy of a node carries bitwise the same value.
  F4 every local row is an FP32 sum in local CSR order, evaluated here column
     by column over all rows at once; the interface sums in ascending
     subdomain order.
Condition estimate (Lanczos tridiagonal from alpha_k, beta_k):
  K1 the 1D Laplacian of size n after n iterations: kappa = cot^2(pi/(2(n+1))).
  K2 a diagonal matrix with d distinct values: after d iterations kappa =
     max/min; for k < d the estimate grows with k and stays below it (the Ritz
     values lie inside the spectrum).
Generators (cell-centred finite volumes, harmonic faces, boundary faces 2k):
  G1 fv3d_7pt on 2x2x2 cells with constant kappa, written out by hand.
  G2 fv3d_7pt on 2x2x2 cells, one cell with another kappa.
  G3 fv3d_7pt on a line of three cells along x, y and z, three kappas.
  G4 fv2d_5pt on 2x2 cells and on a line of three cells.
Mixed inner iterations:
  M1 a matrix with d distinct eigenvalues (d <= 4, kappa <= 27), refinement
     capped at two steps and rtol 1e-13, so that both inner solves run to
     the inner tolerance 1e-4 (rtol ||b|| / ||r|| stays below it): each FP32
     inner solve ends after exactly d iterations (CG's finite termination),
     2 d in all.  (Uncapped, the last refinement's tolerance rtol ||b|| / ||r||
     is loose, and where it stops depends on rounding.)
"""

import inspect
import math
import os

import numpy as np
import pytest

import oracle
import synth.problems as problems
from synth import (
    CSR,
    box_partition_3d,
    config_problem,
    fe2d_p1_jittered,
    fv2d_5pt,
    fv3d_7pt,
    laplace1d,
    pair_blocks,
    random_spd,
    rcb_partition,
)

U32 = 2.0**-24
U = 2.0**-53


# ---------------------------------------------------------------- FP32 product
def _cases():
    rng = np.random.default_rng(11)
    out = []
    kap = np.exp(rng.standard_normal((4, 3, 5)))
    out.append(("fv3d_5x3x4_2x2x2", fv3d_7pt(5, 3, 4, kap), box_partition_3d(5, 3, 4, 2, 2, 2), 8))
    A, coords, _ = fe2d_p1_jittered(9, rng)
    out.append(("fe_9_rcb4", A, rcb_partition(coords, 2, rng), 4))
    A = random_spd(48, 5.0, rng)
    out.append(("rand48_P5", A, rng.integers(0, 5, 48).astype(np.int32), 5))
    return out


CASES = _cases()


def _integer_version(A):
    """Same pattern, symmetric small integer values, positive diagonal."""
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    off = -(1 + (rows + A.colidx) % 3).astype(np.float64)
    val = np.where(rows == A.colidx, 0.0, off)
    diag = 1.0 + np.bincount(rows, weights=np.abs(val), minlength=A.n)
    val = np.where(rows == A.colidx, diag[rows], val)
    return CSR(A.n, A.rowptr, A.colidx, val)


def _columnwise_fp32(m, xl32):
    """F4's evaluation: k-th entries of all local rows at once, FP32 products
    and sums, then each interface node's copies summed in ascending order."""
    val32 = m.lval.astype(np.float32)
    lens = np.diff(m.lrowptr)
    sub = np.searchsorted(m.off, np.arange(m.nloc), side="right") - 1
    acc = np.zeros(m.nloc, np.float32)
    for k in range(int(lens.max(initial=0))):
        rows = np.nonzero(lens > k)[0]
        e = m.lrowptr[rows] + k
        prod = val32[e] * xl32[m.off[sub[rows]] + m.lcol[e]]
        acc[rows] = acc[rows] + prod
    y = acc.copy()
    for g in range(m.ngamma):
        cs = m.icopy[m.iptr[g]:m.iptr[g + 1]]
        S = np.float32(0.0)
        for c in cs:
            S = np.float32(S + acc[c])
        y[cs] = S
    return y


def pin_spmv32(A, part, P, seed=2):
    rng = np.random.default_rng(seed)
    # F1: integer data, exact
    Ai = _integer_version(A)
    Pt = oracle.Partition(Ai, part, P)
    m = Pt.maps
    xi = rng.integers(-8, 9, A.n)
    y_int = Ai.to_scipy().astype(np.int64) @ xi.astype(np.int64)
    yl = Pt.spmv32(xi.astype(np.float32)[m.l2g])
    assert np.array_equal(yl.astype(np.int64), y_int[m.l2g])
    # F2 + F3 + F4 on the real values
    Pt = oracle.Partition(A, part, P)
    m = Pt.maps
    x32 = rng.uniform(-1, 1, A.n).astype(np.float32)
    xl32 = x32[m.l2g]
    yl = Pt.spmv32(xl32)
    assert yl.dtype == np.float32
    x64 = x32.astype(np.float64)
    y_ref = A.to_scipy() @ x64
    absAx = abs(A.to_scipy()) @ np.abs(x64)
    L = np.diff(A.rowptr)
    bound = 4.0 * (L + m.mult) * U32 * absAx + 1e-300
    y_own = yl[m.own].astype(np.float64)
    assert np.all(np.abs(y_own - y_ref) <= bound)
    assert np.array_equal(yl.view(np.int32), yl[m.own][m.l2g].view(np.int32))
    assert np.array_equal(yl.view(np.int32), _columnwise_fp32(m, xl32).view(np.int32))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_spmv32_pins(case):
    pin_spmv32(*case[1:])


def _run_spmv32_pins():
    failures = []
    for c in CASES:
        try:
            pin_spmv32(*c[1:])
        except Exception as e:  # noqa: BLE001 - any failure counts as caught
            failures.append((c[0], type(e).__name__))
    return failures


SPMV32_MUTATIONS = {
    # the interface assembly keeps only the last copy's value
    "spmv32_last_copy": ("float S = 0.0f;\n        for (int32_t c = h->iptr[g]; c < h->iptr[g + 1]; ++c) S += yl[h->icopy[c]];",
                         "float S = 0.0f;\n        for (int32_t c = h->iptr[g]; c < h->iptr[g + 1]; ++c) S = yl[h->icopy[c]];"),
    # row index used where the column index belongs
    "spmv32_wrong_index": ("acc += val32[k] * xl[o + h->lcol[k]];", "acc += val32[k] * xl[o + li];"),
    # rows accumulated in double, not FP32
    "spmv32_double_accumulation": (
        "float acc = 0.0f;\n            for (int32_t k = h->lrowptr[o + li]; k < h->lrowptr[o + li + 1]; ++k) acc += val32[k] * xl[o + h->lcol[k]];",
        "double acc = 0.0;\n            for (int32_t k = h->lrowptr[o + li]; k < h->lrowptr[o + li + 1]; ++k) acc += (double)val32[k] * xl[o + h->lcol[k]];"),
    # no interface assembly at all
    "spmv32_no_assembly": (
        "        float S = 0.0f;\n        for (int32_t c = h->iptr[g]; c < h->iptr[g + 1]; ++c) S += yl[h->icopy[c]];\n        for (int32_t c = h->iptr[g]; c < h->iptr[g + 1]; ++c) yl[h->icopy[c]] = S;",
        "        (void)g;"),
}


@pytest.mark.parametrize("name", sorted(SPMV32_MUTATIONS))
def test_spmv32_planted_mistake_is_caught(name):
    old, new = SPMV32_MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, "mutation anchor not found: %s" % name
    path = oracle.compile_variant(src.replace(old, new), name)
    try:
        with oracle.use_library(path):
            failures = _run_spmv32_pins()
    finally:
        os.remove(path)
    assert failures, "planted mistake %s slipped through every pin" % name


# ---------------------------------------------------------------- condition estimate
def _diag(d):
    n = d.size
    return CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.asarray(d, np.float64))


def pin_cond(cond=oracle.cond_from_lanczos):
    rng = np.random.default_rng(19)
    # K1: 1D Laplacian, eigenvalues 4 sin^2(j pi / (2(n+1))), j = 1..n
    for n in (8, 20, 40):
        b = rng.uniform(-1, 1, n)
        r = oracle.cg(laplace1d(n), b, 0.0, n)
        assert r.iters == n
        exact = 1.0 / math.tan(math.pi / (2 * (n + 1))) ** 2
        assert abs(cond(r.alpha, r.beta) - exact) <= 1e-9 * exact
    # K2: diagonal with d distinct values, each repeated
    values = np.array([1.0, 2.0, 5.0, 10.0, 30.0, 100.0])
    d = rng.permutation(np.repeat(values, 10))
    b = rng.uniform(-1, 1, d.size)
    A = _diag(d)
    prev = 0.0
    for k in range(1, values.size + 1):
        r = oracle.cg(A, b, 0.0, k)
        est = cond(r.alpha, r.beta)
        assert prev - 1e-12 <= est <= 100.0 * (1 + 1e-12)
        prev = est
    assert abs(prev - 100.0) <= 1e-10 * 100.0


def test_cond_from_lanczos_pins():
    pin_cond()


COND_MUTATIONS = {
    # off-diagonal of T divided by the next alpha
    "offdiag_index": ("e = np.sqrt(bt[:-1]) / a[:-1]", "e = np.sqrt(bt[:-1]) / a[1:]"),
    # off-diagonal without the square root
    "offdiag_no_sqrt": ("e = np.sqrt(bt[:-1]) / a[:-1]", "e = bt[:-1] / a[:-1]"),
    # the beta term of the diagonal divided by the wrong alpha
    "diag_beta_index": ("d[1:] += bt[:-1] / a[:-1]", "d[1:] += bt[:-1] / a[1:]"),
    # the beta term of the diagonal dropped
    "diag_no_beta": ("d[1:] += bt[:-1] / a[:-1]", "d = d"),
}


@pytest.mark.parametrize("name", sorted(COND_MUTATIONS))
def test_cond_planted_mistake_is_caught(name):
    old, new = COND_MUTATIONS[name]
    src = inspect.getsource(oracle.cond_from_lanczos)
    assert src.count(old) == 1, name
    ns = {"np": np}
    exec(src.replace(old, new), ns)
    with pytest.raises(AssertionError):
        pin_cond(ns["cond_from_lanczos"])


# ---------------------------------------------------------------- finite-volume generators
def _dense(A):
    D = np.zeros((A.n, A.n))
    for i in range(A.n):
        for k in range(A.rowptr[i], A.rowptr[i + 1]):
            D[i, A.colidx[k]] = A.val[k]
    return D


def _expected(n, pairs, face, boundary):
    """Dense matrix from a hand-made list of interior faces (a, b) with their
    coefficients, plus each cell's total boundary coefficient."""
    E = np.zeros((n, n))
    for (a, b), t in zip(pairs, face):
        E[a, b] = E[b, a] = -t
        E[a, a] += t
        E[b, b] += t
    for i in range(n):
        E[i, i] += boundary[i]
    return E


# interior faces of the 2x2x2 grid, cell id ix + 2 iy + 4 iz
PAIRS_222 = [(0, 1), (2, 3), (4, 5), (6, 7),   # x
             (0, 2), (1, 3), (4, 6), (5, 7),   # y
             (0, 4), (1, 5), (2, 6), (3, 7)]   # z
# interior faces of the 2x2 grid, cell id ix + 2 iy
PAIRS_22 = [(0, 1), (2, 3), (0, 2), (1, 3)]


def pin_fv(f3=fv3d_7pt, f2=fv2d_5pt):
    # G1: constant kappa 2: interior faces 2, three boundary faces of 4 per cell
    A = f3(2, 2, 2, np.full((2, 2, 2), 2.0))
    assert A.nnz == 8 + 2 * 12
    assert np.array_equal(_dense(A), _expected(8, PAIRS_222, [2.0] * 12, [12.0] * 8))
    # G2: cell 0 has kappa 3, the rest 1: faces at cell 0 are 2*3*1/(3+1) = 1.5
    k = np.ones((2, 2, 2))
    k[0, 0, 0] = 3.0
    face = [1.5 if 0 in p else 1.0 for p in PAIRS_222]
    bnd = [3 * 2 * 3.0] + [3 * 2 * 1.0] * 7
    assert np.array_equal(_dense(f3(2, 2, 2, k)), _expected(8, PAIRS_222, face, bnd))
    # G3: three cells in a line along each axis, kappa 1, 2, 4: faces 4/3, 8/3;
    # the end cells have five boundary faces, the middle one four
    line = np.array([1.0, 2.0, 4.0])
    E = _expected(3, [(0, 1), (1, 2)], [4.0 / 3.0, 8.0 / 3.0], [5 * 2.0, 4 * 4.0, 5 * 8.0])
    for shape in ((1, 1, 3), (1, 3, 1), (3, 1, 1)):  # (nz, ny, nx)
        nz, ny, nx = shape
        D = _dense(f3(nx, ny, nz, line.reshape(shape)))
        assert np.all(np.abs(D - E) <= 4 * U * np.abs(E)), shape
    # G4: 2D, cell 0 with kappa 3 on 2x2, and a line of three cells
    k = np.ones((2, 2))
    k[0, 0] = 3.0
    face = [1.5 if 0 in p else 1.0 for p in PAIRS_22]
    bnd = [2 * 2 * 3.0] + [2 * 2 * 1.0] * 3
    assert np.array_equal(_dense(f2(2, 2, k)), _expected(4, PAIRS_22, face, bnd))
    E = _expected(3, [(0, 1), (1, 2)], [4.0 / 3.0, 8.0 / 3.0], [3 * 2.0, 2 * 4.0, 3 * 8.0])
    for shape in ((1, 3), (3, 1)):  # (ny, nx)
        ny, nx = shape
        D = _dense(f2(nx, ny, line.reshape(shape)))
        assert np.all(np.abs(D - E) <= 4 * U * np.abs(E)), shape


def test_fv_generator_pins():
    pin_fv()


FV_MUTATIONS = {
    # boundary faces at full-cell distance (k instead of 2k)
    "fv3d_boundary_k": ("fv3d_7pt", "bnd = 2.0 * k", "bnd = 1.0 * k"),
    # arithmetic instead of harmonic mean
    "fv3d_arith_mean": ("fv3d_7pt", "return 2.0 * a * b / (a + b)", "return 0.5 * (a + b)"),
    # y- face coefficients shifted onto the wrong cells
    "fv3d_y_shift": ("fv3d_7pt", "tym[:, 1:, :] = fy", "tym[:, :-1, :] = fy"),
    # z faces from one side only
    "fv3d_z_one_sided": ("fv3d_7pt", "fz = harm(k[:-1, :, :], k[1:, :, :])", "fz = harm(k[:-1, :, :], k[:-1, :, :])"),
    "fv2d_boundary_k": ("fv2d_5pt", "bnd = 2.0 * k", "bnd = 1.0 * k"),
    "fv2d_x_shift": ("fv2d_5pt", "txm[:, 1:] = fx", "txm[:, :-1] = fx"),
}


@pytest.mark.parametrize("name", sorted(FV_MUTATIONS))
def test_fv_planted_mistake_is_caught(name):
    fname, old, new = FV_MUTATIONS[name]
    src = inspect.getsource(getattr(problems, fname))
    assert src.count(old) == 1, name
    ns = dict(vars(problems))
    exec(src.replace(old, new), ns)
    fns = {"f3": fv3d_7pt, "f2": fv2d_5pt}
    fns["f3" if fname == "fv3d_7pt" else "f2"] = ns[fname]
    with pytest.raises(AssertionError):
        pin_fv(**fns)


# ---------------------------------------------------------------- mixed inner iteration counts
# 2x2 blocks [[a, b], [b, a]]: eigenvalues a - b and a + b
COUNT_CASES = [
    ("d4_kappa27", [(14.0, 13.0), (6.0, 3.0)], 4),   # 1, 27, 3, 9
    ("d3_kappa16", [(2.5, 1.5), (10.0, 6.0)], 3),     # 1, 4, 4, 16
    ("d2_kappa4", [(5.0, 3.0)], 2),                   # 2, 8
]


def count_case(blocks, seed, nrep=25, P=5):
    rng = np.random.default_rng(seed)
    A = pair_blocks(blocks, nrep)
    b = rng.uniform(-1, 1, A.n)
    part = rng.integers(0, P, A.n).astype(np.int32)
    return A, b, part, P


@pytest.mark.parametrize("case", COUNT_CASES, ids=[c[0] for c in COUNT_CASES])
def test_mixed_inner_counts_finite_termination(case):
    _, blocks, d = case
    for seed in range(4):
        A, b, part, P = count_case(blocks, seed)
        Pt = oracle.Partition(A, part, P)
        assert Pt.maps.ngamma > 0  # the pairs are split across subdomains
        r = Pt.cg_mixed(b, 1e-13, 1000, 1e-4, 2)
        assert r.status in (oracle.OK, oracle.NOT_CONVERGED)
        assert r.outer == 2 and r.iters == 2 * d, (seed, r.iters, r.outer)
        assert np.linalg.norm(b - oracle.spmv(A, r.x)) <= 1e-9 * np.linalg.norm(b)
