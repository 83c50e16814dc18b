"""GPU parity of the sub-structured SpMV, weighted dot and scatter/gather
against the FP64 oracle, element by element, through the C ABI.

Tolerances (both sides FP64, different summation order and FMA use):
  SpMV entry i:  |y_gpu - y_oracle| <= 4 (L_i + m_i) u (|A| |x|)_i,
                 u = 2^-53, L_i the row length, m_i the node multiplicity
                 (each side is within gamma_{L+m} (|A||x|)_i of the exact value).
  weighted dot:  |d_gpu - d_oracle| <= 4 N u sum_k w_k |u_k v_k|.
  scatter / gather: bit-exact (pure data movement).
"""

import numpy as np
import pytest

import oracle
from synth import config_problem, fv3d_7pt, box_partition_3d, random_spd, poisson2d_5pt

pytestmark = pytest.mark.gpu

U = 2.0**-53


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2108_13162_gb300 import build as ssg_build
    from paper_2108_13162_gb300.ssg import Context

    ssg_build.build()
    assert torch.cuda.is_available()
    c = Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()


def _cases():
    rng = np.random.default_rng(99)
    out = []
    p = config_problem(1)
    out.append(("config1_64x64_2x2", p.A, p.part, p.P))
    p = config_problem(2, scale=40)  # 40^3: several tiles per subdomain, ragged 10^3 boxes
    out.append(("fv3d_40_4x4x4", p.A, p.part, p.P))
    p = config_problem(3, scale=96)
    out.append(("fe2d_96_rcb", p.A, p.part, p.P))
    A = random_spd(3001, 9.0, rng)  # irregular rows, random partition, high multiplicities
    out.append(("rand3001_P13", A, rng.integers(0, 13, A.n).astype(np.int32), 13))
    # a long dense-ish row: hub node connected to many others (tile of its own)
    n = 5000
    import scipy.sparse as sp

    i = np.concatenate([np.zeros(4500, np.int64), np.arange(1, n)])
    j = np.concatenate([np.arange(1, 4501), np.arange(0, n - 1)])
    W = sp.coo_matrix((np.full(i.size, 0.01), (i, j)), shape=(n, n)).tocsr()
    W.data[:] = 0.01
    W = (W + W.T).tocsr()
    W.data[:] = -0.01
    Dg = sp.diags(np.asarray(abs(W).sum(axis=1)).ravel() + 1.0)
    M = (Dg + W).tocsr()
    M.sort_indices()
    U_ = sp.triu(M, 0, format="csr")
    M = (U_ + sp.triu(U_, 1, format="csr").T).tocsr()
    M.sort_indices()
    from synth import CSR

    A = CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
    out.append(("hub5000_P2", A, (np.arange(n) * 2 // n).astype(np.int32), 2))
    A = poisson2d_5pt(3, 1)  # tiny, fewer rows than one warp
    out.append(("tiny3", A, np.array([0, 1, 1], np.int32), 2))
    return out


CASES = _cases()


def _torch(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check_spmv(ctx, A, part, P, seed=0):
    import torch

    from paper_2108_13162_gb300.ssg import System

    S = System(ctx, A, part, P)
    ref = oracle.Partition(A, part, P)
    m = ref.maps
    x = np.random.default_rng(seed).uniform(-1, 1, A.n)
    xl_ref = ref.scatter(x)
    y_ref = ref.spmv(xl_ref)
    xg = _torch(x)
    xl = S.scatter(xg)
    torch.cuda.synchronize()
    assert np.array_equal(xl.cpu().numpy(), xl_ref)  # scatter bit-exact
    xSx = torch.zeros(1, dtype=torch.float64, device="cuda")
    y = S.spmv(xl, xSx=xSx).cpu().numpy()
    absAx = abs(A.to_scipy()) @ np.abs(x)
    L = np.diff(A.rowptr)
    bound = 4.0 * (L[m.l2g] + m.mult[m.l2g]) * U * absAx[m.l2g]
    err = np.abs(y - y_ref)
    assert np.all(err <= bound), "max err %g at %d" % (err.max(), int(np.argmax(err - bound)))
    # consistency: all copies of an interface node are bitwise equal
    own_vals = y[m.own]
    assert np.array_equal(y, own_vals[m.l2g])
    # (x, Sx)_w from the SpMV epilogue matches the oracle's weighted dot
    d_ref = ref.wdot(xl_ref, y_ref)
    scale = float(np.sum(m.w * np.abs(xl_ref * y_ref)))
    assert abs(float(xSx.item()) - d_ref) <= 4 * m.nloc * U * scale + 1e-300
    # gather returns each node's owner copy, bit-exact
    yg = S.gather(_torch(y)).cpu().numpy()
    assert np.array_equal(yg, ref.gather(y))
    return S, ref


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_spmv_assembled_parity(ctx, case):
    _, A, part, P = case
    _check_spmv(ctx, A, part, P)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_wdot_parity(ctx, case):
    import torch

    from paper_2108_13162_gb300.ssg import System

    _, A, part, P = case
    S = System(ctx, A, part, P)
    ref = oracle.Partition(A, part, P)
    rng = np.random.default_rng(5)
    u = ref.scatter(rng.uniform(-1, 1, A.n))
    v = rng.uniform(-1, 1, ref.maps.nloc)  # not consistent: the weighted sum is still defined
    out = S.wdot(_torch(u), _torch(v))
    d_ref = ref.wdot(u, v)
    scale = float(np.sum(ref.maps.w * np.abs(u * v)))
    assert abs(float(out.item()) - d_ref) <= 4 * ref.maps.nloc * U * scale
    # deterministic: same inputs, same bits
    out2 = S.wdot(_torch(u), _torch(v))
    torch.cuda.synchronize()
    assert out.item() == out2.item()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_spmv_f32_parity(ctx, case):
    """FP32 SpMV (mixed mode's inner operator): both sides round values and x
    to FP32 the same way; |dy_i| <= 4 (L_i + m_i) u32 (|A||x|)_i, u32 = 2^-24."""
    import torch

    from paper_2108_13162_gb300.ssg import System

    _, A, part, P = case
    S = System(ctx, A, part, P)
    ref = oracle.Partition(A, part, P)
    m = ref.maps
    x = np.random.default_rng(9).uniform(-1, 1, A.n)
    xl32 = ref.scatter(x).astype(np.float32)
    y_ref = ref.spmv32(xl32).astype(np.float64)
    y = torch.empty(m.nloc, dtype=torch.float32, device="cuda")
    S.spmv_prec(torch.from_numpy(xl32).cuda(), y, "fp32")
    yg = y.cpu().numpy().astype(np.float64)
    absAx = abs(A.to_scipy()) @ np.abs(x)
    L = np.diff(A.rowptr)
    bound = 4.0 * (L[m.l2g] + m.mult[m.l2g]) * 2.0**-24 * absAx[m.l2g] * 1.0001
    assert np.all(np.abs(yg - y_ref) <= bound)
    assert np.array_equal(yg, yg[m.own][m.l2g])  # copies consistent


def test_spmv_full_size_128cube(ctx):
    """The 128^3, 64-subdomain workload the benchmark times: every output checked."""
    p = config_problem(2)
    _check_spmv(ctx, p.A, p.part, p.P, seed=1)


def test_spmv_deterministic(ctx):
    import torch

    from paper_2108_13162_gb300.ssg import System

    p = config_problem(2, scale=32)
    S = System(ctx, p.A, p.part, p.P)
    x = S.scatter(_torch(np.random.default_rng(3).uniform(-1, 1, p.A.n)))
    y1 = S.spmv(x)
    y2 = S.spmv(x)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)


@pytest.mark.parametrize("seed", range(40))
def test_random_systems_product_and_iterates(ctx, seed):
    """The 40 seeded random systems and partitions of the host-map sweep
    (empty and unused subdomains, isolated nodes, one-node systems): the
    product on every local entry within 4 (L_i + m_i) u (|A||x|)_i of the
    oracle's, and a solve's first six iterates within 1e-10 of the oracle's,
    through the one-cluster solve (the default at these sizes) and the loop."""
    import torch

    from paper_2108_13162_gb300.ssg import System
    from tests.test_abi_host import _random_case

    A, part, P = _random_case(seed)
    S = System(ctx, A, part, P)
    ref = oracle.Partition(A, part, P)
    m = ref.maps
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, A.n)
    xl = ref.scatter(x)
    y = S.spmv(torch.from_numpy(xl).cuda()).cpu().numpy()
    absAx = abs(A.to_scipy()) @ np.abs(x)
    L = np.zeros(A.n)
    np.maximum.at(L, m.l2g, np.diff(m.lrowptr))
    assert np.all(np.abs(y - ref.spmv(xl)) <= 4.0 * (L[m.l2g] + m.mult[m.l2g]) * U * absAx[m.l2g])
    b = rng.uniform(-1, 1, A.n)
    k = min(6, A.n)
    r = ref.cg(b, 0.0, k)
    limit = ctx.cluster_solve()[0]
    for lim in (limit, 0):
        ctx.set_cluster_solve(lim)
        try:
            xg, rc, st = S.solve(torch.from_numpy(b).cuda(), rtol=0.0, max_iter=k)
        finally:
            ctx.set_cluster_solve(limit)
        rel = np.linalg.norm(xg.cpu().numpy() - r.x) / max(np.linalg.norm(r.x), 1e-300)
        assert rel <= 1e-10, (lim, rel)
    S.close()
