"""GPU band-row and band-column splittings (Sections 2.1, 2.2; Algorithms 1, 2)
against the oracle's or_band_row / or_band_col and their products, through
the C ABI.

Readings: the band arrays (row pointers, column ids, values) are bit-exact;
the products are within 2 (L_i + nb) u sum_j |A_ij x_j| of the oracle's (both
sides sum each band's row left to right, the GPU with fused multiply-adds,
the lane variants in a strided order), exact on integer data for every
variant (every partial sum is an integer), and the staged kernel gives the
same bits as one thread per row (same order, same operations).
"""

import numpy as np
import pytest

import oracle
from synth import CSR, config_problem, poisson2d_5pt, random_spd

pytestmark = pytest.mark.gpu

U = 2.0**-53
ROW_VARIANTS = [-1, 1, 2, 4, 8, 16, 32]
COL_VARIANTS = [-1, 1]


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2108_13162_gb300 import build as ssg_build
    from paper_2108_13162_gb300.ssg import Context

    ssg_build.build()
    c = Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _nonsym(n, seed, long_rows=()):
    """Nonsymmetric pattern with empty rows; rows in long_rows get that many entries."""
    rng = np.random.default_rng(seed)
    rp, ci, va = [0], [], []
    for i in range(n):
        k = dict(long_rows).get(i, int(rng.integers(0, 9)) if i % 7 else 0)
        cols = np.sort(rng.choice(n, size=min(k, n), replace=False))
        ci += cols.tolist()
        va += rng.uniform(-2, 2, cols.size).tolist()
        rp.append(len(ci))
    return CSR(n, np.array(rp, np.int32), np.array(ci, np.int32), np.array(va))


def _cases():
    rng = np.random.default_rng(77)
    return [
        ("poisson2d_33x29", poisson2d_5pt(33, 29)),
        ("random_spd_3001", random_spd(3001, 9.0, rng)),
        ("nonsym_2111", _nonsym(2111, 5)),
        # rows longer than a staged tile (2048 entries) and one exactly at it
        ("long_rows_6000", _nonsym(6000, 6, long_rows=((17, 5000), (3000, 2048), (5999, 2049)))),
    ]


CASES = _cases()


def _bound(A, x, nb):
    ax = np.abs(A.val * x[A.colidx])
    s = np.add.reduceat(np.append(ax, 0.0), A.rowptr[:-1]) * (np.diff(A.rowptr) > 0)
    L = np.diff(A.rowptr)
    return 2.0 * (L + nb) * U * s


@pytest.mark.parametrize("name,A", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kind", ["row", "col"])
def test_band_arrays_bit_exact(ctx, name, A, kind):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Band

    for nb in (1, 3, 7, 64):
        B = Band(ctx, A, ssg.SSG_BAND_ROW if kind == "row" else ssg.SSG_BAND_COL, nb)
        for p in sorted({0, 1 % nb, nb // 2, nb - 1}):
            npr, displ, rp, ci, va = B.band(p)
            ref = oracle.band(A, kind, nb, p)
            assert (npr, displ) == (ref.np, ref.displ)
            assert np.array_equal(rp, ref.rowptr)
            assert np.array_equal(ci, ref.colidx)
            assert np.array_equal(va, ref.val)
        B.close()


@pytest.mark.parametrize("name,A", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kind", ["row", "col"])
def test_band_products(ctx, name, A, kind):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Band

    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, A.n)
    Ai = CSR(A.n, A.rowptr, A.colidx, rng.integers(-9, 10, A.colidx.size).astype(np.float64))
    xi = rng.integers(-9, 10, A.n).astype(np.float64)
    for nb in (1, 5, 64):
        y_ref = oracle.band_spmv(A, kind, nb, x)
        yi_ref = oracle.band_spmv(Ai, kind, nb, xi)
        bound = _bound(A, x, nb)
        code = ssg.SSG_BAND_ROW if kind == "row" else ssg.SSG_BAND_COL
        B = Band(ctx, A, code, nb)
        Bi = Band(ctx, Ai, code, nb)
        outs = {}
        for v in (ROW_VARIANTS if kind == "row" else COL_VARIANTS):
            B.set_variant(v)
            Bi.set_variant(v)
            y = B.spmv(_t(x)).cpu().numpy()
            assert np.all(np.abs(y - y_ref) <= bound), (nb, v)
            assert np.array_equal(Bi.spmv(_t(xi)).cpu().numpy(), yi_ref), (nb, v)
            outs[v] = y
        assert np.array_equal(outs[-1], outs[1])  # staged = one thread per row, bit for bit
        B.close()
        Bi.close()


def test_band_autotune_and_rule(ctx):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Band

    def rule(A, code):
        # one thread per row while the mean row length is at most 8, else
        # lanes = the power of two >= mean / 2 in [2, 32]; band-column
        # products always one thread per row
        mean = A.nnz / A.n
        if code == ssg.SSG_BAND_COL or mean <= 8:
            return 1
        v = 2
        while v < 32 and v < mean / 2:
            v *= 2
        return v

    x = _t(np.random.default_rng(4).uniform(-1, 1, CASES[1][1].n))
    for A in (CASES[0][1], CASES[1][1]):
        for code in (ssg.SSG_BAND_ROW, ssg.SSG_BAND_COL):
            B = Band(ctx, A, code, 7)
            assert B.autotune(reps=1)["rule_variant"] == rule(A, code)
            B.close()
    assert rule(CASES[0][1], ssg.SSG_BAND_ROW) == 1 and rule(CASES[1][1], ssg.SSG_BAND_ROW) > 1
    A = CASES[1][1]
    for code, valid in ((ssg.SSG_BAND_ROW, ROW_VARIANTS), (ssg.SSG_BAND_COL, COL_VARIANTS)):
        B = Band(ctx, A, code, 7)
        t = B.autotune(reps=3)
        assert t["variant"] in valid and sorted(t["us"]) == sorted(valid)
        y = B.spmv(x)
        B.set_variant(t["variant"])
        assert np.array_equal(B.spmv(x).cpu().numpy(), y.cpu().numpy())
        B.close()
    # long rows: the rule takes lanes per row
    n = 512
    rp = np.arange(n + 1, dtype=np.int32) * 40
    ci = np.concatenate([np.sort(np.random.default_rng(i).choice(n, 40, replace=False)) for i in range(n)])
    Bl = Band(ctx, CSR(n, rp, ci.astype(np.int32), np.ones(n * 40)), ssg.SSG_BAND_ROW, 4)
    assert Bl.autotune(reps=2)["rule_variant"] == 32
    Bl.close()


def test_band_rejects_bad_input(ctx):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Band

    A = poisson2d_5pt(6, 5)
    for nb in (0, A.n + 1):
        with pytest.raises(ssg.SSGError):
            Band(ctx, A, ssg.SSG_BAND_ROW, nb)
    bad = CSR(A.n, A.rowptr, A.colidx.copy(), A.val)
    bad.colidx[[0, 1]] = bad.colidx[[1, 0]]  # unsorted row 0
    with pytest.raises(ssg.SSGError):
        Band(ctx, bad, ssg.SSG_BAND_COL, 2)
    with pytest.raises(ssg.SSGError):
        Band(ctx, A, 2, 2)
    B = Band(ctx, A, ssg.SSG_BAND_COL, 3)
    for v in (2, 4, 32, 3, 64):
        with pytest.raises(ssg.SSGError):
            B.set_variant(v)
    with pytest.raises(ssg.SSGError):
        ssg.ssg_band_get(B.h, 3, A.n)
    B.close()


@pytest.mark.parametrize("kind", ["row", "col"])
def test_band_full_size_128cube(ctx, kind):
    """The 128^3 finite-volume matrix in 64 bands, in the launch configuration
    the benchmark times: every entry against the oracle's product."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Band

    p = config_problem(2)
    A = p.A
    x = np.random.default_rng(9).uniform(-1, 1, A.n)
    B = Band(ctx, A, ssg.SSG_BAND_ROW if kind == "row" else ssg.SSG_BAND_COL, 64)
    y = B.spmv(_t(x)).cpu().numpy()
    y_ref = oracle.band_spmv(A, kind, 64, x)
    assert np.all(np.abs(y - y_ref) <= _bound(A, x, 64))
    B.set_variant(1)
    assert np.array_equal(B.spmv(_t(x)).cpu().numpy(), y)
    npr, displ, rp, ci, va = B.band(63)
    ref = oracle.band(A, kind, 64, 63)
    assert np.array_equal(rp, ref.rowptr) and np.array_equal(ci, ref.colidx) and np.array_equal(va, ref.val)
    B.close()


@pytest.mark.parametrize("kind", ["row", "col"])
def test_band_degenerate_matrices(ctx, kind):
    """One row (n = 1, one band) and a matrix without stored entries (every
    row empty): y = A x exactly for every kernel variant."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Band

    code = ssg.SSG_BAND_ROW if kind == "row" else ssg.SSG_BAND_COL
    one = CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.5]))
    empty = CSR(5, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0))
    for A, nb in ((one, 1), (empty, 1), (empty, 5)):
        B = Band(ctx, A, code, nb)
        x = np.arange(1.0, A.n + 1.0)
        y_ref = oracle.band_spmv(A, kind, nb, x)
        for v in (ROW_VARIANTS if kind == "row" else COL_VARIANTS):
            B.set_variant(v)
            assert np.array_equal(B.spmv(_t(x)).cpu().numpy(), y_ref), (A.n, nb, v)
        npr, displ, rp, ci, va = B.band(nb - 1)
        ref = oracle.band(A, kind, nb, nb - 1)
        assert np.array_equal(rp, ref.rowptr) and ci.size == ref.colidx.size
        B.close()


def test_band_bounded_wait_times_out(ctx):
    """The staged kernel's mbarrier wait is bounded: on a phase that nothing
    completes it gives up after about a second and reports SSG_E_TIMEOUT; the
    operator (and the context) keep working afterwards."""
    import time

    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Band

    A = poisson2d_5pt(20, 20)
    B = Band(ctx, A, ssg.SSG_BAND_ROW, 4)
    t0 = time.perf_counter()
    rc = ssg.ssg_band_check_timeout(B.h)
    dt = time.perf_counter() - t0
    assert rc == ssg.SSG_E_TIMEOUT, rc
    assert 0.5 <= dt <= 30.0, dt
    x = np.random.default_rng(2).uniform(-1, 1, A.n)
    B.set_variant(ssg.SSG_BAND_STAGED)
    y = B.spmv(_t(x)).cpu().numpy()
    assert np.all(np.abs(y - oracle.band_spmv(A, "row", 4, x)) <= _bound(A, x, 4))
    B.close()
