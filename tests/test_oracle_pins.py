"""Pins for the CPU oracle: facts the paper and the mathematics fix, checked
without reference to the oracle's own formulas.

P1  sum_s R_s^T A^(s) R_s == A, same structure, bit-identical values
    (Eq. interface_summation: the interface blocks of the local matrices add
    up to the global one).
P2  every stored nonzero owned exactly once; hand-derived interface counts
    for the 2x2 split of the 64x64 grid and the closed form for box splits of
    a 3D grid.
P3  assembled local SpMV == global SpMV within a rounding bound (Section 3.4.1).
P4  weighted dot == global dot on consistent vectors (Section 3.4.2).
P5  one subdomain: sub-structured CG == textbook CG bit for bit (Algorithm 3).
P6  tiny SPD systems: CG to 1e-12 matches a dense Cholesky solve (oracle's own
    and LAPACK's) to 1e-10.
P7  finite termination: A = I in one step, d distinct eigenvalues in <= d
    steps, the 1D Laplacian of size n in <= n steps.
P8  manufactured solution recovered within 2*kappa*rtol.
P9  the worked 5x5 CSR example of Section 1.2.
P10 Algorithm 3 with the diagonal preconditioner M = diag(S): a diagonal S is
    solved in one iteration; one subdomain equals the global PCG bit for bit;
    k iterations equal k iterations of plain CG on D^-1/2 S D^-1/2 mapped
    back by D^-1/2 (global and sub-structured); agreement with Cholesky.
Planted mistakes: textual mutations of the oracle's C source must each break
at least one pin.
"""

import os

import numpy as np
import pytest

import oracle
from synth import (
    CSR,
    box_partition_2d,
    box_partition_3d,
    config_problem,
    fe2d_p1_jittered,
    fv3d_7pt,
    laplace1d,
    manufactured_rhs,
    poisson2d_5pt,
    random_spd,
    rcb_partition,
)

U = 2.0**-53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- fixtures
def _small_cases():
    """(name, A, part, P) tuples covering regular, irregular and odd partitions."""
    rng = np.random.default_rng(7)
    cases = []
    A = poisson2d_5pt(12, 9)
    cases.append(("p2d_12x9_3x2", A, box_partition_2d(12, 9, 3, 2), 6))
    kap = np.exp(rng.standard_normal((6, 5, 7)))
    A = fv3d_7pt(7, 5, 6, kap)
    cases.append(("fv3d_7x5x6_2x2x3", A, box_partition_3d(7, 5, 6, 2, 2, 3), 12))
    A, coords, _ = fe2d_p1_jittered(14, rng)
    cases.append(("fe_14_rcb8", A, rcb_partition(coords, 3, rng), 8))
    A = random_spd(150, 6.0, rng)
    cases.append(("rand150_P5", A, rng.integers(0, 5, 150).astype(np.int32), 5))
    # a subdomain id with no node at all (empty V_s) and an unused top id
    part = rng.integers(0, 4, 150).astype(np.int32)
    part[part == 2] = 1
    cases.append(("rand150_empty", A, part, 5))
    A = laplace1d(40)
    cases.append(("lap1d_40_P1", A, np.zeros(40, np.int32), 1))
    return cases


SMALL = _small_cases()


def _dense(A: CSR):
    D = np.zeros((A.n, A.n))
    for i in range(A.n):
        for k in range(A.rowptr[i], A.rowptr[i + 1]):
            D[i, A.colidx[k]] = A.val[k]
    return D


# ---------------------------------------------------------------- pins as functions
def pin_reassembly(A, part, P):
    """P1 + P2: rebuild A from the local matrices via the l2g maps."""
    m = oracle.Partition(A, part, P).maps
    assert m.nnz == A.nnz
    sub = np.searchsorted(m.off, np.arange(m.nloc), side="right") - 1
    row_g = np.repeat(m.l2g, np.diff(m.lrowptr))
    row_s = np.repeat(sub, np.diff(m.lrowptr))
    col_g = m.l2g[m.off[row_s] + m.lcol]
    key = row_g.astype(np.int64) * A.n + col_g
    order = np.argsort(key, kind="stable")
    ref_key = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.rowptr)) * A.n + A.colidx
    # every stored entry appears exactly once (ownership is a partition of the entries)
    assert np.array_equal(key[order], ref_key)
    # and carries the global value unchanged, bit for bit
    assert np.array_equal(m.lval[order].view(np.int64), A.val.view(np.int64))
    # every node has at least one copy, and its copy count equals m
    assert np.array_equal(np.bincount(m.l2g, minlength=A.n), m.mult)
    assert m.mult.min() >= 1
    return m


def pin_sub_spmv(A, part, P, seed=3):
    """P3: assembled SpMV equals the global SpMV within a rounding bound."""
    Pt = oracle.Partition(A, part, P)
    m = Pt.maps
    x = np.random.default_rng(seed).uniform(-1, 1, A.n)
    y_ref = A.to_scipy() @ x
    yl = Pt.spmv(Pt.scatter(x))
    absAx = abs(A.to_scipy()) @ np.abs(x)
    L = np.diff(A.rowptr)
    bound = 2.0 * (L + m.mult) * U * absAx + 1e-300
    y_own = yl[m.own]
    assert np.all(np.abs(y_own - y_ref) <= bound)
    # consistency: every copy of a node carries the same value (fixed order)
    assert np.array_equal(yl, y_own[m.l2g])
    return yl


def pin_wdot(A, part, P, seed=4):
    """P4: weighted dot of consistent vectors equals the global dot."""
    Pt = oracle.Partition(A, part, P)
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1, 1, A.n)
    v = rng.uniform(-1, 1, A.n)
    got = Pt.wdot(Pt.scatter(u), Pt.scatter(v))
    ref = float(np.dot(u, v))
    scale = float(np.dot(np.abs(u), np.abs(v)))
    assert abs(got - ref) <= 1e-14 * scale
    # and a vector of ones has squared weighted norm n
    one = Pt.scatter(np.ones(A.n))
    assert abs(Pt.wdot(one, one) - A.n) <= 1e-12 * A.n


def pin_cholesky(A, part, P, seed=5):
    """P6: CG on a tiny SPD system agrees with dense Cholesky (two of them)."""
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1, 1, A.n)
    D = _dense(A)
    x_chol = oracle.cholesky_solve(D, b)
    x_lapack = np.linalg.solve(D, b)
    assert np.linalg.norm(x_chol - x_lapack) <= 1e-12 * np.linalg.norm(x_lapack)
    r = oracle.Partition(A, part, P).cg(b, 1e-12, 20 * A.n)
    assert r.status == oracle.OK
    assert np.linalg.norm(r.x - x_chol) <= 1e-10 * np.linalg.norm(x_chol)


def pin_config1_counts():
    """P2 hand-derived: 64x64 grid, 2x2 boxes.

    V_0 gains the column ix=32 (iy<32) and the row iy=32 (ix<32): 1024+64;
    V_1 gains the row iy=32 (ix>=32): 1056; V_2 the column ix=32 (iy>=32): 1056;
    V_3: 1024.  Interface = the 127 distinct borrowed nodes, node (32,32) shared
    by three subdomains, 126*2 + 3 = 255 copies.
    """
    p = config_problem(1)
    m = oracle.Partition(p.A, p.part, p.P).maps
    assert list(np.diff(m.off)) == [1088, 1056, 1056, 1024]
    assert m.nloc == 4224
    assert m.ngamma == 127
    assert m.ncopies == 255
    assert np.count_nonzero(m.mult == 3) == 1 and m.mult[32 + 64 * 32] == 3
    assert np.count_nonzero(m.mult == 2) == 126
    assert list(m.nint) == [1024, 992, 992, 961]


def pin_box3d_closed_form(s, p):
    """P2 closed form for a 7-point s^3 grid split into p^3 boxes.

    A node is borrowed once per low face of its box that touches another box
    (3(p-1) planes of s^2 nodes); the interface is the union of those planes:
    3(p-1)s^2 - 3(p-1)^2 s + (p-1)^3 nodes (inclusion-exclusion over plane
    pairs and triples); copies = interface + borrowed.
    """
    kap = np.ones((s, s, s))
    A = fv3d_7pt(s, s, s, kap)
    m = oracle.Partition(A, box_partition_3d(s, s, s, p, p, p), p**3).maps
    borrowed = 3 * (p - 1) * s * s
    gam = 3 * (p - 1) * s * s - 3 * (p - 1) ** 2 * s + (p - 1) ** 3
    assert m.nloc == s**3 + borrowed
    assert m.ngamma == gam
    assert m.ncopies == gam + borrowed


def pin_p1_bitwise(A, b):
    """P5: with one subdomain the sub-structured CG is textbook CG, bitwise."""
    Pt = oracle.Partition(A, np.zeros(A.n, np.int32), 1)
    r1 = Pt.cg(b, 1e-10, 5 * A.n)
    r0 = oracle.cg(A, b, 1e-10, 5 * A.n)
    assert r1.iters == r0.iters and r1.status == r0.status == oracle.OK
    assert np.array_equal(r1.x, r0.x)
    assert np.array_equal(r1.alpha, r0.alpha)


def pin_termination():
    """P7: finite termination counts."""
    rng = np.random.default_rng(11)
    n = 60
    eye = CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    part = rng.integers(0, 3, n).astype(np.int32)
    r = oracle.Partition(eye, part, 3).cg(rng.uniform(-1, 1, n), 1e-12, 10)
    assert r.status == oracle.OK and r.iters == 1
    d = 5
    dv = np.repeat(np.arange(1.0, d + 1), n // d)
    Dg = CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), dv)
    r = oracle.Partition(Dg, part, 3).cg(rng.uniform(-1, 1, n), 1e-10, 50)
    assert r.status == oracle.OK and r.iters <= d
    for nn in (16, 32, 64):
        A = laplace1d(nn)
        pp = (np.arange(nn) * 4 // nn).astype(np.int32)
        r = oracle.Partition(A, pp, 4).cg(rng.uniform(-1, 1, nn), 1e-10, 10 * nn)
        assert r.status == oracle.OK and r.iters <= nn


def pin_manufactured(A, part, P, xs, b, rtol):
    """P8: ||x - x*|| / ||x*|| <= 2 * kappa_est * rtol (kappa from Lanczos)."""
    r = oracle.Partition(A, part, P).cg(b, rtol, 50 * A.n)
    assert r.status == oracle.OK
    kap = oracle.cond_from_lanczos(r.alpha, r.beta)
    err = np.linalg.norm(r.x - xs) / np.linalg.norm(xs)
    assert err <= 2.0 * kap * rtol
    # true residual agrees with the recursive one to the same order
    tr = np.linalg.norm(b - A.to_scipy() @ r.x) / np.linalg.norm(b)
    assert tr <= 10 * rtol
    return r


# ---------------------------------------------------------------- tests
def test_csr_example_5x5():
    """P9: the 5x5 example of Section 1.2, encoded and multiplied."""
    lines = [l.split() for l in open(os.path.join(GOLDEN, "csr_example_5x5.txt")) if l.strip() and l[0] != "#"]
    i = lines.index(["dense"])
    dense = np.array([[float(v) for v in lines[i + 1 + r]] for r in range(5)])
    kv = {}
    xs, ys = [], []
    for l in lines[i + 6 :]:
        if l[0] == "x":
            xs.append(np.array(l[1:], float))
        elif l[0] == "y":
            ys.append(np.array(l[1:], float))
        else:
            kv[l[0]] = np.array(l[1:], float)
    # encode the dense matrix row by row, as the CSR definition says
    rp, ci, va = [0], [], []
    for r in range(5):
        for c in range(5):
            if dense[r, c] != 0:
                ci.append(c)
                va.append(dense[r, c])
        rp.append(len(ci))
    assert rp == list(kv["rowptr"].astype(int))
    assert ci == list(kv["colidx"].astype(int))
    assert va == list(kv["val"])
    A = CSR(5, np.array(rp, np.int32), np.array(ci, np.int32), np.array(va))
    for x, y in zip(xs, ys):
        assert np.array_equal(oracle.spmv(A, x), y)
    # the example is not symmetric: the partitioner must refuse it
    with pytest.raises(ValueError):
        oracle.Partition(A, np.zeros(5, np.int32), 1)


@pytest.mark.parametrize("case", SMALL, ids=[c[0] for c in SMALL])
def test_reassembly_exact(case):
    _, A, part, P = case
    pin_reassembly(A, part, P)


@pytest.mark.parametrize("case", SMALL, ids=[c[0] for c in SMALL])
def test_sub_spmv_matches_global(case):
    _, A, part, P = case
    pin_sub_spmv(A, part, P)


@pytest.mark.parametrize("case", SMALL, ids=[c[0] for c in SMALL])
def test_wdot_matches_global(case):
    _, A, part, P = case
    pin_wdot(A, part, P)


@pytest.mark.parametrize("case", SMALL, ids=[c[0] for c in SMALL])
def test_cg_matches_cholesky(case):
    _, A, part, P = case
    pin_cholesky(A, part, P)


def test_config1_counts():
    pin_config1_counts()


@pytest.mark.parametrize("s,p", [(8, 2), (12, 3), (16, 4)])
def test_box3d_counts(s, p):
    pin_box3d_closed_form(s, p)


def test_single_subdomain_is_textbook_cg():
    A = poisson2d_5pt(20, 17)
    b = np.random.default_rng(2).uniform(-1, 1, A.n)
    pin_p1_bitwise(A, b)


def test_finite_termination():
    pin_termination()


def test_manufactured_config1():
    p = config_problem(1)
    r = pin_manufactured(p.A, p.part, p.P, p.xstar[:, 0], p.b[:, 0], 1e-10)
    assert 100 < r.iters < 400


def test_manufactured_fv3d_small():
    p = config_problem(2, scale=16)
    pin_manufactured(p.A, p.part, p.P, p.xstar[:, 0], p.b[:, 0], 1e-8)


def test_local_numbering_and_lists():
    """Interior-first numbering, ascending ids, copies in ascending s, w = 1/m."""
    _, A, part, P = SMALL[2]
    m = oracle.Partition(A, part, P).maps
    for s in range(P):
        g = m.l2g[m.off[s] : m.off[s + 1]]
        ni = m.nint[s]
        assert np.all(m.mult[g[:ni]] == 1) and np.all(m.mult[g[ni:]] >= 2)
        assert np.all(np.diff(g[:ni]) > 0) and np.all(np.diff(g[ni:]) > 0)
        assert np.all(part[g[:ni]] == s)
    assert np.all(np.diff(m.gamma) > 0)
    for gi in range(m.ngamma):
        c = m.icopy[m.iptr[gi] : m.iptr[gi + 1]]
        assert np.all(np.diff(c) > 0)  # ascending s <=> ascending concatenated index
        assert np.all(m.l2g[c] == m.gamma[gi])
    assert np.array_equal(m.w, 1.0 / m.mult[m.l2g])
    assert np.all(m.l2g[m.own] == np.arange(A.n))


def test_invalid_inputs_rejected():
    A = poisson2d_5pt(5, 5)
    bad = np.zeros(A.n, np.int32)
    bad[3] = 4
    with pytest.raises(ValueError):
        oracle.Partition(A, bad, 4)
    # value asymmetry
    v = A.val.copy()
    v[1] += 0.5
    with pytest.raises(ValueError):
        oracle.Partition(CSR(A.n, A.rowptr, A.colidx, v), np.zeros(A.n, np.int32), 1)
    # unsorted columns
    c = A.colidx.copy()
    c[0], c[1] = c[1], c[0]
    with pytest.raises(ValueError):
        oracle.Partition(CSR(A.n, A.rowptr, c, A.val), np.zeros(A.n, np.int32), 1)


def test_breakdown_on_indefinite():
    """(p, Sp) <= 0 must stop the iteration with a breakdown status."""
    A = laplace1d(10)
    An = CSR(A.n, A.rowptr, A.colidx, -A.val)  # negative definite
    r = oracle.Partition(An, np.zeros(10, np.int32), 1).cg(np.ones(10), 1e-10, 100)
    assert r.status == oracle.BREAKDOWN


# ---------------------------------------------------------------- planted mistakes
MUTATIONS = {
    # interface assembly keeps only the last copy instead of the sum
    "no_assembly_sum": ("double S = 0.0;\n        for (int32_t c = h->iptr[g]; c < h->iptr[g + 1]; ++c) S += yl[h->icopy[c]];",
                        "double S = 0.0;\n        for (int32_t c = h->iptr[g]; c < h->iptr[g + 1]; ++c) S = yl[h->icopy[c]];"),
    # unweighted dot (w = 1 on every copy)
    "unit_weights": ("    if (!h->w) { free(memloc); goto oom; }\n    for (int64_t k = 0; k < h->nloc; ++k) h->w[k] = 1.0 / (double)h->mult[h->l2g[k]];",
                     "    if (!h->w) { free(memloc); goto oom; }\n    for (int64_t k = 0; k < h->nloc; ++k) h->w[k] = 1.0;"),
    # off-diagonal entries owned by the higher subdomain, interface entries counted twice
    "double_owner": ("return part[i] < part[j] ? part[i] : part[j];", "return part[i];"),
    # wrong sign in the residual update
    "residual_sign": ("for (int64_t k = 0; k < L; ++k) r[k] = r[k] - alpha * q[k];\n        double rho_new",
                      "for (int64_t k = 0; k < L; ++k) r[k] = r[k] + alpha * q[k];\n        double rho_new"),
    # row index used where the column index belongs in the local product
    "wrong_index": ("acc += h->lval[k] * xl[o + h->lcol[k]];", "acc += h->lval[k] * xl[o + li];"),
    # inverted ratio for the new direction
    "beta_inverted": ("double beta = rho_new / rho;\n        for (int64_t k",
                      "double beta = rho / rho_new;\n        for (int64_t k"),
}


def _run_all_pins():
    failures = []
    checks = [
        ("config1_counts", pin_config1_counts),
        ("reassembly", lambda: [pin_reassembly(*c[1:]) for c in SMALL[:4]]),
        ("sub_spmv", lambda: [pin_sub_spmv(*c[1:]) for c in SMALL[:4]]),
        ("wdot", lambda: [pin_wdot(*c[1:]) for c in SMALL[:4]]),
        ("cholesky", lambda: [pin_cholesky(*c[1:]) for c in SMALL[:4]]),
        ("termination", pin_termination),
    ]
    for name, fn in checks:
        try:
            fn()
        except Exception as e:  # noqa: BLE001 - any failure counts as caught
            failures.append((name, type(e).__name__))
    return failures


def test_pins_pass_on_oracle():
    assert _run_all_pins() == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, "mutation anchor not found: %s" % name
    path = oracle.compile_variant(src.replace(old, new), name)
    try:
        with oracle.use_library(path):
            failures = _run_all_pins()
    finally:
        os.remove(path)
    assert failures, "planted mistake %s slipped through every pin" % name


# ---------------------------------------------------------------- P10: diagonal preconditioner
def _diag(A):
    return np.array([A.val[A.rowptr[i]:A.rowptr[i + 1]][A.colidx[A.rowptr[i]:A.rowptr[i + 1]] == i][0]
                     for i in range(A.n)])


def _sym_scaled(A):
    """D^-1/2 A D^-1/2 with D = diag(A), entry by entry."""
    s = 1.0 / np.sqrt(_diag(A))
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    return CSR(A.n, A.rowptr, A.colidx, A.val * (s[rows] * s[A.colidx])), s


def pin_pcg_diagonal():
    """M = S for a diagonal S: z_1 = S^-1 b, so one iteration solves it."""
    rng = np.random.default_rng(21)
    n = 90
    d = rng.uniform(0.5, 50.0, n)
    Dg = CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    b = rng.uniform(-1, 1, n)
    part = rng.integers(0, 4, n).astype(np.int32)
    for r in (oracle.pcg(Dg, b, 1e-12, 10), oracle.Partition(Dg, part, 4).pcg(b, 1e-12, 10)):
        assert r.status == oracle.OK and r.iters == 1
        assert np.all(np.abs(r.x - b / d) <= 4 * U * np.abs(b / d))


def pin_pcg_p1_bitwise(A, b):
    Pt = oracle.Partition(A, np.zeros(A.n, np.int32), 1)
    r1 = Pt.pcg(b, 1e-10, 5 * A.n)
    r0 = oracle.pcg(A, b, 1e-10, 5 * A.n)
    assert r1.status == r0.status == oracle.OK and r1.iters == r0.iters
    assert np.array_equal(r1.x, r0.x)


def pin_pcg_scaled_equivalence(A, part, P, k=6, seed=8):
    """Jacobi-preconditioned CG on S is plain CG on D^-1/2 S D^-1/2 in the
    variable D^1/2 x: after k iterations both give the same x up to rounding."""
    b = np.random.default_rng(seed).uniform(-1, 1, A.n)
    Ah, s = _sym_scaled(A)
    xh = oracle.cg(Ah, s * b, 0.0, k).x
    x_ref = s * xh
    scale = np.linalg.norm(x_ref)
    xg = oracle.pcg(A, b, 0.0, k).x
    assert np.linalg.norm(xg - x_ref) <= 1e-10 * scale
    Pt = oracle.Partition(A, part, P)
    xs = Pt.pcg(b, 0.0, k).x
    assert np.linalg.norm(xs - x_ref) <= 1e-10 * scale
    xsh = oracle.Partition(Ah, part, P).cg(s * b, 0.0, k).x
    assert np.linalg.norm(xs - s * xsh) <= 1e-10 * scale


def pin_pcg_cholesky(A, part, P, seed=5):
    b = np.random.default_rng(seed).uniform(-1, 1, A.n)
    x_chol = oracle.cholesky_solve(_dense(A), b)
    r = oracle.Partition(A, part, P).pcg(b, 1e-12, 20 * A.n)
    assert r.status == oracle.OK
    assert np.linalg.norm(r.x - x_chol) <= 1e-10 * np.linalg.norm(x_chol)


def _run_pcg_pins():
    failures = []
    checks = [
        ("pcg_diagonal", pin_pcg_diagonal),
        ("pcg_scaled", lambda: [pin_pcg_scaled_equivalence(*c[1:]) for c in SMALL[:4]]),
        ("pcg_cholesky", lambda: [pin_pcg_cholesky(*c[1:]) for c in SMALL[:4]]),
    ]
    for name, fn in checks:
        try:
            fn()
        except Exception as e:  # noqa: BLE001 - any failure counts as caught
            failures.append((name, type(e).__name__))
    return failures


def test_pcg_diagonal_one_step():
    pin_pcg_diagonal()


def test_pcg_single_subdomain_is_global_pcg():
    A = fv3d_7pt(6, 5, 7, np.exp(np.random.default_rng(4).standard_normal((7, 5, 6))))
    pin_pcg_p1_bitwise(A, np.random.default_rng(2).uniform(-1, 1, A.n))


@pytest.mark.parametrize("case", SMALL, ids=[c[0] for c in SMALL])
def test_pcg_scaled_equivalence(case):
    _, A, part, P = case
    pin_pcg_scaled_equivalence(A, part, P)


@pytest.mark.parametrize("case", SMALL, ids=[c[0] for c in SMALL])
def test_pcg_matches_cholesky(case):
    _, A, part, P = case
    pin_pcg_cholesky(A, part, P)


def test_pcg_manufactured_and_fewer_iterations():
    """On the heterogeneous FV problem the diagonal preconditioner removes the
    kappa scaling: it converges in fewer iterations, the true residual is
    <= rtol (to rounding), and ||x - x*|| / ||x*|| <= cond(S) ||r|| / ||b||."""
    p = config_problem(2, scale=24)
    b = p.b[:, 0]
    Pt = oracle.Partition(p.A, p.part, p.P)
    r = Pt.pcg(b, 1e-8, 100000)
    r0 = Pt.cg(b, 1e-8, 100000)
    assert r.status == oracle.OK and r.iters < 0.7 * r0.iters
    tr = np.linalg.norm(b - oracle.spmv(p.A, r.x)) / np.linalg.norm(b)
    assert tr <= 1.01e-8
    kap = oracle.cond_from_lanczos(r0.alpha, r0.beta)
    assert np.linalg.norm(r.x - p.xstar[:, 0]) / np.linalg.norm(p.xstar[:, 0]) <= 1.1 * kap * tr


def test_pcg_rejects_missing_diagonal():
    n = 6
    # a symmetric matrix whose row 2 stores no diagonal entry
    rows, cols, vals = [], [], []
    for i in range(n):
        if i != 2:
            rows.append(i), cols.append(i), vals.append(4.0)
        if i + 1 < n:
            rows += [i, i + 1]
            cols += [i + 1, i]
            vals += [-1.0, -1.0]
    import scipy.sparse as sp

    M = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    M.sort_indices()
    A = CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
    assert oracle.pcg(A, np.ones(n), 1e-10, 10).status == oracle.INVALID


PCG_MUTATIONS = {
    # z = M r instead of M^-1 r
    "pcg_times_diag": ("        for (int64_t k = 0; k < L; ++k) z[k] = r[k] / dl[k];\n        const double rz_new",
                       "        for (int64_t k = 0; k < L; ++k) z[k] = r[k] * dl[k];\n        const double rz_new"),
    # the new direction built from r instead of z
    "pcg_direction_from_r": ("for (int64_t k = 0; k < L; ++k) p[k] = z[k] + beta * p[k];",
                             "for (int64_t k = 0; k < L; ++k) p[k] = r[k] + beta * p[k];"),
    # beta from the unpreconditioned residual norms
    "pcg_beta_from_rr": ("        const double rz_new = or_wdot(h, r, z);\n        rr = or_wdot(h, r, r);",
                         "        rr = or_wdot(h, r, r);\n        const double rz_new = rr;"),
    # the diagonal taken from the local copy, which lacks the other copies' share
    "pcg_local_diagonal": ("for (int64_t k = 0; k < h->nloc; ++k) dl[k] = dg[h->l2g[k]];",
                           "for (int64_t k = 0; k < h->nloc; ++k) dl[k] = h->lrowptr[k + 1] > h->lrowptr[k] ? dg[h->l2g[k]] * (h->own[h->l2g[k]] == k ? 1.0 : 0.5) : 1.0;"),
}


@pytest.mark.parametrize("name", sorted(PCG_MUTATIONS))
def test_pcg_planted_mistake_is_caught(name):
    old, new = PCG_MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, "mutation anchor not found: %s" % name
    path = oracle.compile_variant(src.replace(old, new), name)
    try:
        with oracle.use_library(path):
            failures = _run_pcg_pins()
    finally:
        os.remove(path)
    assert failures, "planted mistake %s slipped through every pin" % name


def test_pcg_pins_pass_on_oracle():
    assert _run_pcg_pins() == []


# ---------------------------------------------------------------- mixed precision (library mode SSG_MIXED)
def test_mixed_identity_one_step():
    """A = I with b exactly representable in FP32: one inner iteration gives
    d = b exactly, so one refinement reaches a zero residual."""
    n = 64
    eye = CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    b = np.float32(np.random.default_rng(3).uniform(-1, 1, n)).astype(np.float64)
    r = oracle.Partition(eye, (np.arange(n) % 3).astype(np.int32), 3).cg_mixed(b, 1e-12, 100, 1e-4, 10)
    assert r.status == oracle.OK and r.outer == 1 and r.iters == 1
    assert np.array_equal(r.x, b)


@pytest.mark.parametrize("scale", [16, 24])
def test_mixed_true_residual_and_manufactured(scale):
    """The refinement stops on the FP64 true residual: recomputed with the
    global FP64 product it is <= rtol, and x* is recovered within 2 kappa rtol."""
    p = config_problem(2, scale=scale)
    b = p.b[:, 0]
    Pt = oracle.Partition(p.A, p.part, p.P)
    r = Pt.cg_mixed(b, 1e-8, 100000, 1e-4, 30)
    assert r.status == oracle.OK and r.outer >= 2
    tr = np.linalg.norm(b - oracle.spmv(p.A, r.x)) / np.linalg.norm(b)
    assert tr <= 1.0001e-8
    r64 = Pt.cg(b, 1e-8, 100000)
    kap = oracle.cond_from_lanczos(r64.alpha, r64.beta)
    assert np.linalg.norm(r.x - p.xstar[:, 0]) / np.linalg.norm(p.xstar[:, 0]) <= 2 * kap * 1e-8
    # FP32 inner solves cost only a few more iterations than one FP64 solve
    assert r.iters <= 1.5 * r64.iters


MIXED_MUTATIONS = {
    # the outer residual is not recomputed after the correction
    "stale_outer_residual": ("(double)d32[k];\n        or_sub_spmv(h, xl, q);\n        for (int64_t k = 0; k < L; ++k) r[k] = bl[k] - q[k];\n        rho = or_wdot(h, r, r);\n        ++outer;\n        if (sqrt(rho) <= rtol * bnorm) status = OR_OK;\n        else if (broke) status = OR_BREAKDOWN;\n    }\n    or_gather(h, xl, x);\n    *iters_out = total;\n    *outer_out = outer;\n    *relres_out = bnorm > 0.0 ? sqrt(rho) / bnorm : 0.0;\n    free(bl); free(xl); free(r); free(q); free(val32);",
                             "(double)d32[k];\n        ++outer;\n        if (sqrt(rho) <= rtol * bnorm) status = OR_OK;\n        else if (broke) status = OR_BREAKDOWN;\n    }\n    or_gather(h, xl, x);\n    *iters_out = total;\n    *outer_out = outer;\n    *relres_out = bnorm > 0.0 ? sqrt(rho) / bnorm : 0.0;\n    free(bl); free(xl); free(r); free(q); free(val32);"),
    # the correction is dropped
    "no_correction": ("            rho32 = rho_new;\n            ++total;\n        }\n        for (int64_t k = 0; k < L; ++k) xl[k] = xl[k] + (double)d32[k];",
                      "            rho32 = rho_new;\n            ++total;\n        }\n"),
}


@pytest.mark.parametrize("name", sorted(MIXED_MUTATIONS))
def test_mixed_planted_mistake_is_caught(name):
    old, new = MIXED_MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, name
    path = oracle.compile_variant(src.replace(old, new), name)
    caught = False
    try:
        with oracle.use_library(path):
            try:
                test_mixed_true_residual_and_manufactured(16)
            except AssertionError:
                caught = True
    finally:
        os.remove(path)
    assert caught, "planted mistake %s slipped through" % name


# ---------------------------------------------------------------- mixed precision with the diagonal preconditioner
def pin_pcg_mixed():
    """Diagonal S with b exactly in FP32: every inner solve ends after one
    iteration; on the heterogeneous FV problem the refinement reaches the FP64
    true residual <= rtol, recovers x* within 2 kappa rtol, and its inner
    solves need fewer iterations than the unpreconditioned ones."""
    rng = np.random.default_rng(8)
    n = 80
    d = rng.uniform(0.5, 20.0, n)
    Dg = CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    b = np.float32(rng.uniform(-1, 1, n)).astype(np.float64)
    r = oracle.Partition(Dg, (np.arange(n) % 4).astype(np.int32), 4).pcg_mixed(b, 1e-12, 100, 1e-4, 10)
    assert r.status == oracle.OK and r.outer <= 3 and r.iters == r.outer
    p = config_problem(2, scale=20)
    b = p.b[:, 0]
    Pt = oracle.Partition(p.A, p.part, p.P)
    rm = Pt.pcg_mixed(b, 1e-8, 100000, 1e-4, 30)
    assert rm.status == oracle.OK
    tr = np.linalg.norm(b - oracle.spmv(p.A, rm.x)) / np.linalg.norm(b)
    assert tr <= 1.0001e-8
    r64 = Pt.cg(b, 1e-8, 100000)
    kap = oracle.cond_from_lanczos(r64.alpha, r64.beta)
    assert np.linalg.norm(rm.x - p.xstar[:, 0]) / np.linalg.norm(p.xstar[:, 0]) <= 2 * kap * 1e-8
    assert rm.iters < 0.7 * Pt.cg_mixed(b, 1e-8, 100000, 1e-4, 30).iters


def test_pcg_mixed_pins():
    pin_pcg_mixed()


PCG_MIXED_MUTATIONS = {
    # z = M r instead of M^-1 r in the inner solves
    "inner_times_diag": ("            for (int64_t k = 0; k < L; ++k) z32[k] = r32[k] / g32[k];\n            const double rz_new",
                         "            for (int64_t k = 0; k < L; ++k) z32[k] = r32[k] * g32[k];\n            const double rz_new"),
    # the inner direction built from r instead of z
    "inner_direction_from_r": ("for (int64_t k = 0; k < L; ++k) p32[k] = z32[k] + beta * p32[k];",
                               "for (int64_t k = 0; k < L; ++k) p32[k] = r32[k] + beta * p32[k];"),
}


@pytest.mark.parametrize("name", sorted(PCG_MIXED_MUTATIONS))
def test_pcg_mixed_planted_mistake_is_caught(name):
    old, new = PCG_MIXED_MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, name
    path = oracle.compile_variant(src.replace(old, new), name)
    caught = False
    try:
        with oracle.use_library(path):
            try:
                pin_pcg_mixed()
            except AssertionError:
                caught = True
    finally:
        os.remove(path)
    assert caught, "planted mistake %s slipped through" % name
