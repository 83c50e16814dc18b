"""GPU solves with the diagonal preconditioner (SSG_FP64_JACOBI, Algorithm 3
with M = diag(S), and SSG_MIXED_JACOBI) against the oracle's or_sub_pcg and
or_sub_pcg_mixed, through the C ABI, one right-hand side at a time and
several together (the K-column kernels).

The readings are those of the unpreconditioned parity tests: early iterates
(k <= 6) within 1e-10, solutions converged to 1e-12 within 1e-10, iteration
counts at 1e-8 within max(2, 3 %); the 128^3 workload against the stored
oracle run.  The GPU stores 1 / S_ii and multiplies, the oracle divides by
S_ii: one more rounding per entry of z, inside those tolerances.
"""

import json
import os

import numpy as np
import pytest

import oracle
from synth import CSR, config_problem, random_spd

pytestmark = pytest.mark.gpu


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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _cases():
    rng = np.random.default_rng(31)
    out = [("config1", config_problem(1)), ("fv3d_24", config_problem(2, scale=24)),
           ("fe2d_64", config_problem(3, scale=64))]
    A = random_spd(2000, 8.0, rng)
    out.append(("rand2000_P7", (A, rng.integers(0, 7, A.n).astype(np.int32), 7, rng.uniform(-1, 1, A.n))))
    return out


CASES = _cases()


def _unpack(case):
    if isinstance(case, tuple):
        return case
    return case.A, case.part, case.P, case.b[:, 0]


@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
def test_jacobi_matches_oracle(ctx, name, case):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    A, part, P, b = _unpack(case)
    S = System(ctx, A, part, P)
    ref = oracle.Partition(A, part, P)
    x, rc, st = S.solve(_t(b), rtol=0.0, max_iter=6, mode=ssg.SSG_FP64_JACOBI)
    assert rc == ssg.SSG_E_NOT_CONVERGED and st[0]["iters"] == 6
    assert _rel(x.cpu().numpy(), ref.pcg(b, 0.0, 6).x) <= 1e-10
    x, rc, st = S.solve(_t(b), rtol=1e-12, max_iter=100000, mode=ssg.SSG_FP64_JACOBI)
    assert rc == ssg.SSG_OK
    assert _rel(x.cpu().numpy(), ref.pcg(b, 1e-12, 100000).x) <= 1e-10
    x, rc, st = S.solve(_t(b), rtol=1e-8, max_iter=100000, mode=ssg.SSG_FP64_JACOBI)
    r = ref.pcg(b, 1e-8, 100000)
    assert rc == ssg.SSG_OK and abs(st[0]["iters"] - r.iters) <= max(2, 0.03 * r.iters)
    assert st[0]["true_relres"] <= 1.01e-8


def test_jacobi_fewer_iterations_and_drivers_agree(ctx):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p = config_problem(2, scale=32)
    S = System(ctx, p.A, p.part, p.P)
    b = _t(p.b[:, 0])
    _, _, s0 = S.solve(b, rtol=1e-8)
    x1, rc1, s1 = S.solve(b, rtol=1e-8, mode=ssg.SSG_FP64_JACOBI)
    assert rc1 == ssg.SSG_OK and s1[0]["iters"] < 0.7 * s0[0]["iters"]
    # the graph-driven and the host-driven loop (the one-cluster solve off):
    # the same kernels, the same bits
    limit = ctx.cluster_solve()[0]
    ctx.set_cluster_solve(0)
    try:
        x1, rc1, s1 = S.solve(b, rtol=1e-8, mode=ssg.SSG_FP64_JACOBI)
        ctx.set_driver(ssg.SSG_DRIVER_HOST)
        x2, rc2, s2 = S.solve(b, rtol=1e-8, mode=ssg.SSG_FP64_JACOBI)
    finally:
        ctx.set_driver(ssg.SSG_DRIVER_GRAPH)
        ctx.set_cluster_solve(limit)
    assert s2[0]["iters"] == s1[0]["iters"]
    assert np.array_equal(x1.cpu().numpy(), x2.cpu().numpy())
    # several right-hand sides iterate together (K = 2), each column against the oracle
    B = np.stack([p.b[:, 0], 2.0 * p.b[:, 0]])
    X, rc, st = S.solve(_t(B), rtol=1e-8, mode=ssg.SSG_FP64_JACOBI)
    assert rc == ssg.SSG_OK and [s["block"] for s in st] == [2, 2]
    ref = oracle.Partition(p.A, p.part, p.P)
    for j in range(2):
        r = ref.pcg(B[j], 1e-8, 100000)
        assert abs(st[j]["iters"] - r.iters) <= max(2, 0.03 * r.iters)
        assert st[j]["true_relres"] <= 1.01e-8
    ctx.set_driver(ssg.SSG_DRIVER_HOST)
    try:
        X2, rc2, st2 = S.solve(_t(B), rtol=1e-8, mode=ssg.SSG_FP64_JACOBI)
    finally:
        ctx.set_driver(ssg.SSG_DRIVER_GRAPH)
    assert rc2 == ssg.SSG_OK and [a["iters"] for a in st2] == [a["iters"] for a in st]
    assert np.array_equal(X2.cpu().numpy(), X.cpu().numpy())


@pytest.mark.parametrize("name,case", CASES[1:], ids=[c[0] for c in CASES[1:]])
@pytest.mark.parametrize("k", [3, 16])
def test_jacobi_block_matches_oracle(ctx, name, case, k):
    """k right-hand sides through the K-column kernels (K = 4, 16) with the
    diagonal preconditioner: per column the single-solve readings (early
    iterates within 1e-10, converged to 1e-12 within 1e-10; mixed: refinements
    within +-1, inner iterations within max(3 per refinement, 10 %), FP64 true
    residual <= rtol)."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    A, part, P, b = _unpack(case)
    rng = np.random.default_rng(k)
    B = np.stack([b] + [rng.uniform(-1, 1, A.n) for _ in range(k - 1)])
    S = System(ctx, A, part, P)
    ref = oracle.Partition(A, part, P)
    X, rc, st = S.solve(_t(B), rtol=0.0, max_iter=6, mode=ssg.SSG_FP64_JACOBI)
    assert rc == ssg.SSG_E_NOT_CONVERGED and all(t["iters"] == 6 and t["block"] == (4 if k == 3 else 16) for t in st)
    X = X.cpu().numpy()
    for j in range(k):
        assert _rel(X[j], ref.pcg(B[j], 0.0, 6).x) <= 1e-10
    X, rc, st = S.solve(_t(B), rtol=1e-12, max_iter=100000, mode=ssg.SSG_FP64_JACOBI)
    assert rc == ssg.SSG_OK
    X = X.cpu().numpy()
    for j in range(k):
        assert _rel(X[j], ref.pcg(B[j], 1e-12, 100000).x) <= 1e-10
    X, rc, st = S.solve(_t(B), rtol=1e-8, max_iter=100000, mode=ssg.SSG_MIXED_JACOBI)
    assert rc == ssg.SSG_OK
    X = X.cpu().numpy()
    for j in range(k):
        rm = ref.pcg_mixed(B[j], 1e-8, 100000, 1e-4, 30)
        tr = np.linalg.norm(B[j] - oracle.spmv(A, X[j])) / np.linalg.norm(B[j])
        assert tr <= 1.0001e-8
        assert abs(st[j]["outer"] - rm.outer) <= 1
        assert abs(st[j]["iters"] - rm.iters) <= max(3 * rm.outer, 0.10 * rm.iters)


def test_jacobi_rejects_bad_diagonal(ctx):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    # a symmetric positive definite tridiagonal matrix whose row 3 stores no diagonal
    n = 8
    rows, cols, vals = [], [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n and not (i == j == 3):
                rows.append(i)
                cols.append(j)
                vals.append(4.0 if i == j else -1.0)
    import scipy.sparse as sp

    M = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    M.sort_indices()
    A = CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
    S = System(ctx, A, (np.arange(n) % 2).astype(np.int32), 2)
    with pytest.raises(ssg.SSGError):
        S.solve(_t(np.ones(n)), rtol=1e-8, mode=ssg.SSG_FP64_JACOBI)
    # new values with a negative diagonal entry are refused too; valid ones accepted again
    p = config_problem(1)
    S2 = System(ctx, p.A, p.part, p.P)
    v = p.A.val.copy()
    row = slice(p.A.rowptr[5], p.A.rowptr[6])
    v[p.A.rowptr[5] + int(np.nonzero(p.A.colidx[row] == 5)[0][0])] = -1.0  # the diagonal of row 5
    ssg.ssg_set_values(S2.h, _t(v))
    with pytest.raises(ssg.SSGError):
        S2.solve(_t(p.b[:, 0]), rtol=1e-8, mode=ssg.SSG_FP64_JACOBI)
    ssg.ssg_set_values(S2.h, _t(p.A.val))
    x, rc, st = S2.solve(_t(p.b[:, 0]), rtol=1e-10, mode=ssg.SSG_FP64_JACOBI)
    assert rc == ssg.SSG_OK


def test_jacobi_full_size_128cube(ctx):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_fv3d_128_4x4x4.json")) as f:
        g = json.load(f)
    gj = g["jacobi"]
    kap = [s for s in g["solves"] if s["rtol"] == 1e-8][0]["kappa_lanczos"]
    p = config_problem(2)
    S = System(ctx, p.A, p.part, p.P)
    x, rc, st = S.solve(_t(p.b[:, 0]), rtol=1e-8, max_iter=100000, mode=ssg.SSG_FP64_JACOBI)
    assert rc == ssg.SSG_OK
    print("jacobi 128^3: %d iterations (oracle %d)" % (st[0]["iters"], gj["iters"]))
    assert abs(st[0]["iters"] - gj["iters"]) <= max(2, 0.03 * gj["iters"])
    xg = x.cpu().numpy()
    idx = np.array(g["sample_idx"])
    assert _rel(xg[idx], np.array(gj["sample_x"])) <= 2 * kap * 1e-8
    assert st[0]["true_relres"] <= 1.01e-8


@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
def test_mixed_jacobi_matches_oracle(ctx, name, case):
    """SSG_MIXED_JACOBI against or_sub_pcg_mixed: refinements within +-1, inner
    iterations within max(3 per refinement, 10 %), FP64 true residual <= rtol."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    A, part, P, b = _unpack(case)
    S = System(ctx, A, part, P)
    ref = oracle.Partition(A, part, P)
    rm = ref.pcg_mixed(b, 1e-8, 100000, 1e-4, 30)
    x, rc, st = S.solve(_t(b), rtol=1e-8, max_iter=100000, mode=ssg.SSG_MIXED_JACOBI)
    assert rc == ssg.SSG_OK and rm.status == oracle.OK
    tr = np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert tr <= 1.0001e-8
    assert abs(st[0]["outer"] - rm.outer) <= 1
    assert abs(st[0]["iters"] - rm.iters) <= max(3 * rm.outer, 0.10 * rm.iters)


def test_mixed_jacobi_full_size_128cube(ctx):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_fv3d_128_4x4x4.json")) as f:
        g = json.load(f)
    gm = g["mixed_jacobi"]
    kap = [s for s in g["solves"] if s["rtol"] == 1e-8][0]["kappa_lanczos"]
    p = config_problem(2)
    S = System(ctx, p.A, p.part, p.P)
    x, rc, st = S.solve(_t(p.b[:, 0]), rtol=1e-8, max_iter=100000, mode=ssg.SSG_MIXED_JACOBI)
    assert rc == ssg.SSG_OK
    print("mixed jacobi 128^3: %d inner (oracle %d), %d refinements (oracle %d)" % (
        st[0]["iters"], gm["iters"], st[0]["outer"], gm["outer"]))
    assert abs(st[0]["outer"] - gm["outer"]) <= 1
    assert abs(st[0]["iters"] - gm["iters"]) <= max(3 * gm["outer"], 0.10 * gm["iters"])
    idx = np.array(g["sample_idx"])
    assert _rel(x.cpu().numpy()[idx], np.array(gm["sample_x"])) <= 2 * kap * 1e-8
    assert st[0]["true_relres"] <= 1.0001e-8
