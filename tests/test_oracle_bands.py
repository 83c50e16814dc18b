"""Pins of the oracle's band-row and band-column splittings (Sections 2.1 and
2.2, Algorithms 1 and 2) and of the products through them.

What fixes the expected values:
  * the 10x10 pattern drawn in the paper's splitting tables, with per-band
    sizes and arrays derived by hand (tests/golden/band_pattern_10x10.txt);
  * invariants: the bands of either splitting hold every stored entry of A
    exactly once, in A's order, and put back together give A bit for bit;
  * special cases: the band-row product is the textbook CSR product row for
    row, so it equals or_spmv bit for bit; one column band is the whole
    matrix; on integer data every summation order is exact, so the
    band-column product equals A x computed in integer arithmetic;
  * a rounding bound against the exact row sums (math.fsum) on real data.
Planted mistakes in the oracle's band code (each keeping every memory access
in bounds, since the variants run in this process) each fail one of these.
"""

import math
import os

import numpy as np
import pytest

import oracle
from synth import CSR, poisson2d_5pt, random_spd

GOLD = os.path.join(os.path.dirname(__file__), "golden", "band_pattern_10x10.txt")
U = 2.0**-53


def _read_gold():
    pairs, fields, mode = [], {}, None
    for line in open(GOLD):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line == "pairs":
            mode = "pairs"
            continue
        if line == "end":
            mode = None
            continue
        t = line.split()
        if mode == "pairs":
            pairs += [(int(t[i]), int(t[i + 1])) for i in range(0, len(t), 2)]
        else:
            fields[t[0]] = [int(v) for v in t[1:]]
    return pairs, fields


def _pattern_matrix():
    """The paper's 10x10 pattern with value 10*row + col (1-based), CSR 0-based."""
    pairs, f = _read_gold()
    n = 10
    rows = [[] for _ in range(n)]
    for i, j in pairs:
        rows[i - 1].append(j - 1)
    rowptr = [0]
    col, val = [], []
    for i in range(n):
        for j in sorted(rows[i]):
            col.append(j)
            val.append(10.0 * (i + 1) + (j + 1))
        rowptr.append(len(col))
    return CSR(n, np.array(rowptr, np.int32), np.array(col, np.int32), np.array(val)), f


def pin_pattern_counts():
    A, f = _pattern_matrix()
    assert np.diff(A.rowptr).tolist() == f["row_nnz"]
    for nb in (3, 4):
        for kind in ("row", "col"):
            bands = [oracle.band(A, kind, nb, p) for p in range(nb)]
            assert [b.np for b in bands] == f["nb%d_np" % nb]
            assert [b.displ for b in bands] == f["nb%d_displ" % nb]
            assert [b.colidx.size for b in bands] == f["nb%d_%s_nnz" % (nb, kind)]
    for kind in ("row", "col"):
        b = oracle.band(A, kind, 3, 1)
        assert b.rowptr.tolist() == f["nb3_%s_p1_rowptr" % kind]
        assert b.colidx.tolist() == f["nb3_%s_p1_colidx" % kind]


def _cases():
    rng = np.random.default_rng(2101)
    out = [poisson2d_5pt(9, 7), random_spd(157, 6.0, rng)]
    # a nonsymmetric pattern with empty rows: the splittings need neither symmetry nor full rows
    n = 41
    rp, ci, va = [0], [], []
    for i in range(n):
        cols = sorted(rng.choice(n, size=int(rng.integers(0, 6)), replace=False)) if i % 5 else []
        ci += cols
        va += list(rng.uniform(-2, 2, len(cols)))
        rp.append(len(ci))
    out.append(CSR(n, np.array(rp, np.int32), np.array(ci, np.int32), np.array(va)))
    return out


CASES = _cases()


def pin_band_row_reassembly(A, nb):
    rp, ci, va = [0], [], []
    start = 0
    for p in range(nb):
        b = oracle.band(A, "row", nb, p)
        assert b.displ == start and b.rowptr[0] == 0 and b.rowptr.size == b.np + 1
        rp += (b.rowptr[1:] + rp[-1]).tolist()
        ci += b.colidx.tolist()
        va += b.val.tolist()
        start += b.np
    assert start == A.n
    assert np.array_equal(np.array(rp), A.rowptr)
    assert np.array_equal(np.array(ci), A.colidx)
    assert np.array_equal(np.array(va), A.val)


def pin_band_col_reassembly(A, nb):
    bands = [oracle.band(A, "col", nb, p) for p in range(nb)]
    assert sum(b.np for b in bands) == A.n
    assert [b.displ for b in bands] == list(np.cumsum([0] + [b.np for b in bands[:-1]]))
    for i in range(A.n):
        cols, vals = [], []
        for b in bands:
            assert b.rowptr.size == A.n + 1
            seg = slice(b.rowptr[i], b.rowptr[i + 1])
            assert np.all((b.colidx[seg] >= 0) & (b.colidx[seg] < b.np))
            cols += (b.colidx[seg] + b.displ).tolist()
            vals += b.val[seg].tolist()
        row = slice(A.rowptr[i], A.rowptr[i + 1])
        assert cols == A.colidx[row].tolist()
        assert np.array_equal(np.array(vals), A.val[row])


def pin_products(A, nb):
    x = np.random.default_rng(nb).uniform(-1, 1, A.n)
    y = oracle.spmv(A, x)
    assert np.array_equal(oracle.band_spmv(A, "row", nb, x), y)
    assert np.array_equal(oracle.band_spmv(A, "col", 1, x), y)
    yc = oracle.band_spmv(A, "col", nb, x)
    for i in range(A.n):
        terms = [A.val[k] * x[A.colidx[k]] for k in range(A.rowptr[i], A.rowptr[i + 1])]
        L = len(terms)
        assert abs(yc[i] - math.fsum(terms)) <= 2 * (L + nb) * U * sum(abs(t) for t in terms)
    # integer data: every partial sum is exact, so the order of the bands cannot matter
    rng = np.random.default_rng(7 + nb)
    Ai = CSR(A.n, A.rowptr, A.colidx, rng.integers(-9, 10, A.colidx.size).astype(np.float64))
    xi = rng.integers(-9, 10, A.n)
    ye = np.zeros(A.n, np.int64)
    for i in range(A.n):
        for k in range(A.rowptr[i], A.rowptr[i + 1]):
            ye[i] += int(Ai.val[k]) * int(xi[A.colidx[k]])
    for kind in ("row", "col"):
        assert np.array_equal(oracle.band_spmv(Ai, kind, nb, xi.astype(np.float64)), ye.astype(np.float64))


def test_paper_pattern_counts():
    pin_pattern_counts()


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("nb", [1, 2, 3, 7])
def test_band_row_reassembly(case, nb):
    pin_band_row_reassembly(CASES[case], nb)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("nb", [1, 2, 3, 7])
def test_band_col_reassembly(case, nb):
    pin_band_col_reassembly(CASES[case], nb)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("nb", [1, 3, 7])
def test_band_products(case, nb):
    pin_products(CASES[case], nb)


def test_one_band_per_row_and_bad_counts():
    A = poisson2d_5pt(4, 3)
    pin_band_row_reassembly(A, A.n)
    pin_band_col_reassembly(A, A.n)
    pin_products(A, A.n)
    for nb, p in ((0, 0), (A.n + 1, 0), (3, 3), (3, -1)):
        with pytest.raises(ValueError):
            oracle.band(A, "row", nb, p)
        with pytest.raises(ValueError):
            oracle.band(A, "col", nb, p)
    with pytest.raises(ValueError):
        oracle.band_spmv(A, "col", A.n + 1, np.zeros(A.n))


BAND_MUTATIONS = {
    # the last band keeps q rows instead of the rest
    "no_remainder": ("*np = (p == nb - 1) ? n - p * q : q;", "*np = q;"),
    # band-column filter includes the first column of the next band
    "col_filter_inclusive": ("if (displ <= colidx[k] && colidx[k] < displ + np) {",
                             "if (displ <= colidx[k] && colidx[k] <= displ + np) {"),
    # band-column column ids shifted one too far (kept in range, so every access stays in bounds)
    "col_shift_off_by_one": ("bcol[c] = colidx[k] - displ;", "bcol[c] = colidx[k] - displ - (colidx[k] > displ);"),
    # band-row values copied from the start of A instead of the band's first entry
    "row_values_unshifted": ("bval[k] = val[nnz_displ + k];", "bval[k] = val[k];"),
    # band-column partials overwrite instead of summing
    "col_overwrite": ("for (int32_t i = 0; i < n; ++i) y[i] += yp[i];", "for (int32_t i = 0; i < n; ++i) y[i] = yp[i];"),
    # every band writes its block at the start of y
    "row_block_offset": ("or_spmv((int32_t)sz[0], br, bc, bv, x, y + sz[1]);", "or_spmv((int32_t)sz[0], br, bc, bv, x, y);"),
}


def _all_band_pins():
    failures = []
    checks = [
        ("pattern", pin_pattern_counts),
        ("row_reassembly", lambda: [pin_band_row_reassembly(A, nb) for A in CASES[:2] for nb in (3, 7)]),
        ("col_reassembly", lambda: [pin_band_col_reassembly(A, nb) for A in CASES[:2] for nb in (3, 7)]),
        ("products", lambda: [pin_products(A, nb) for A in CASES[:2] for nb in (3, 7)]),
    ]
    for name, fn in checks:
        try:
            fn()
        except (AssertionError, ValueError, IndexError):
            failures.append(name)
    return failures


@pytest.mark.parametrize("name", sorted(BAND_MUTATIONS))
def test_band_planted_mistake_is_caught(name):
    old, new = BAND_MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, name
    path = oracle.compile_variant(src.replace(old, new), name)
    try:
        with oracle.use_library(path):
            failures = _all_band_pins()
    finally:
        os.remove(path)
    assert failures, "planted mistake %s passed every band pin" % name


def test_unmutated_oracle_passes_band_pins():
    assert _all_band_pins() == []
