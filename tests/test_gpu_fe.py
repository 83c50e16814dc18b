"""GPU solves on sub-structures built from finite elements (ssg_partition_fe,
Section 2.4: each local matrix sums its own element matrices) against the
oracle's or_partition_fe, through the C ABI.

The local values are bit-identical on both sides (same element order), so the
readings of the assembled-matrix parity tests apply unchanged: SpMV entries
within 4 (L_i + m_i) u (|A||x|)_i, early iterates (k <= 6) within 1e-10,
solutions converged to 1e-12 within 1e-10, iteration counts at 1e-8 within
max(2, 3 %), for plain CG and for the diagonal preconditioner (assembled
diagonal).  The element and the entry-ownership sub-structures of the same
mesh solve the same system: solutions within 2 kappa rtol.
"""

import numpy as np
import pytest

import oracle
from synth import fe_element_problem

pytestmark = pytest.mark.gpu

U = 2.0**-53


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


CASES = [(40, 3), (96, 6)]


@pytest.mark.parametrize("N,levels", CASES)
def test_fe_spmv_parity(ctx, N, levels):
    from paper_2108_13162_gb300.ssg import System

    ids, Ke, epart, P, A, xs, b = fe_element_problem(N, levels)
    S = System.from_elements(ctx, A.n, ids, Ke, epart, P)
    ref = oracle.Partition.from_elements(A.n, ids, Ke, epart, P)
    m = ref.maps
    x = np.random.default_rng(5).uniform(-1, 1, A.n)
    xl = ref.scatter(x)
    y = S.spmv(_t(xl)).cpu().numpy()
    y_ref = ref.spmv(xl)
    absAx = abs(A.to_scipy()) @ np.abs(x)
    lens = np.diff(m.lrowptr)
    L = np.zeros(A.n)
    np.maximum.at(L, m.l2g, lens)
    bound = 4.0 * (L[m.l2g] + m.mult[m.l2g]) * U * absAx[m.l2g] * 2
    assert np.all(np.abs(y - y_ref) <= bound)
    assert np.array_equal(y, y[m.own][m.l2g])


@pytest.mark.parametrize("N,levels", CASES)
@pytest.mark.parametrize("jacobi", [False, True])
def test_fe_solve_parity(ctx, N, levels, jacobi):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    ids, Ke, epart, P, A, xs, b = fe_element_problem(N, levels)
    S = System.from_elements(ctx, A.n, ids, Ke, epart, P)
    ref = oracle.Partition.from_elements(A.n, ids, Ke, epart, P)
    mode = ssg.SSG_FP64_JACOBI if jacobi else ssg.SSG_FP64
    solve = ref.pcg if jacobi else ref.cg
    x, rc, st = S.solve(_t(b), rtol=0.0, max_iter=6, mode=mode)
    assert _rel(x.cpu().numpy(), solve(b, 0.0, 6).x) <= 1e-10
    x, rc, st = S.solve(_t(b), rtol=1e-12, max_iter=100000, mode=mode)
    assert rc == ssg.SSG_OK
    assert _rel(x.cpu().numpy(), solve(b, 1e-12, 100000).x) <= 1e-10
    x, rc, st = S.solve(_t(b), rtol=1e-8, max_iter=100000, mode=mode)
    r = solve(b, 1e-8, 100000)
    assert rc == ssg.SSG_OK and abs(st[0]["iters"] - r.iters) <= max(2, 0.03 * r.iters)


def test_fe_and_entry_ownership_agree(ctx):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    ids, Ke, epart, P, A, xs, b = fe_element_problem(64, 4)
    S_fe = System.from_elements(ctx, A.n, ids, Ke, epart, P)
    # node partition: each node in the subdomain of its owner copy
    own_sub = np.searchsorted(oracle.Partition.from_elements(A.n, ids, Ke, epart, P).maps.off,
                              oracle.Partition.from_elements(A.n, ids, Ke, epart, P).maps.own, side="right") - 1
    S_as = System(ctx, A, own_sub.astype(np.int32), P)
    x1, rc1, s1 = S_fe.solve(_t(b), rtol=1e-10)
    x2, rc2, s2 = S_as.solve(_t(b), rtol=1e-10)
    r = oracle.Partition(A, own_sub.astype(np.int32), P).cg(b, 1e-10, 100000)
    kap = oracle.cond_from_lanczos(r.alpha, r.beta)
    assert rc1 == rc2 == ssg.SSG_OK
    assert _rel(x1.cpu().numpy(), xs) <= 2 * kap * 1e-10
    assert _rel(x1.cpu().numpy(), x2.cpu().numpy()) <= 4 * kap * 1e-10
    with pytest.raises(ssg.SSGError):
        ssg.ssg_set_values(S_fe.h, _t(A.val))


def test_fe_several_rhs_jacobi(ctx):
    """Three right-hand sides together (K = 4) with the diagonal preconditioner
    on element sub-structures (the assembled diagonal sums the copies' local
    diagonals): each column converged to 1e-12 within 1e-10 of or_sub_pcg."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    ids, Ke, epart, P, A, xs, b = fe_element_problem(40, 3)
    S = System.from_elements(ctx, A.n, ids, Ke, epart, P)
    ref = oracle.Partition.from_elements(A.n, ids, Ke, epart, P)
    rng = np.random.default_rng(41)
    B = np.stack([b, rng.uniform(-1, 1, A.n), rng.uniform(-1, 1, A.n)])
    X, rc, st = S.solve(_t(B), rtol=1e-12, max_iter=100000, mode=ssg.SSG_FP64_JACOBI)
    assert rc == ssg.SSG_OK and [t["block"] for t in st] == [4, 4, 4]
    X = X.cpu().numpy()
    for j in range(3):
        assert _rel(X[j], ref.pcg(B[j], 1e-12, 100000).x) <= 1e-10
