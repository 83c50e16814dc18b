"""GPU solves of several right-hand sides together (K columns per launch)
against the oracle's independent solves, through the C ABI.

Each column runs its own Algorithm 3 (own alpha, beta, stopping test); the
product with K vectors sums every row in the same order as the
single-vector product, so:
  * the K-vector product is bit-identical, column by column, to the
    single-vector GPU product, and within 4 (L_i + m_i) u (|A||x|)_i of the
    oracle's product;
  * per column, early iterates (k <= 6) match the oracle's to 1e-10, solutions
    converged to 1e-12 match to 1e-10, iteration counts at 1e-8 are within
    max(2, 3 %) (the readings of the single-RHS parity tests);
  * mixed mode: per column, refinements within +-1 and inner iterations within
    max(3 per refinement, 10 %) of the oracle's or_sub_cg_mixed, true residual <= rtol;
  * equal columns give equal bits; a zero column converges at once; the
    graph and host-loop drivers give the same bits; padding columns
    (k = 3, 5) and a split into a block plus a single solve (k = 17) work.
"""

import numpy as np
import pytest

import oracle
from synth import config_problem, random_spd

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


@pytest.fixture(scope="module")
def fv20():
    """Config 5's recipe on a 20^3 grid: 3x3x3 boxes, 16 right-hand sides."""
    p = config_problem(5, scale=20)
    return p, oracle.Partition(p.A, p.part, p.P)


@pytest.mark.parametrize("k", [2, 4, 8, 16])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_spmm_bitwise_vs_spmv_and_oracle_bound(ctx, fv20, k, prec):
    import torch

    from paper_2108_13162_gb300.ssg import System

    p, ref = fv20
    S = System(ctx, p.A, p.part, p.P)
    # the single-vector product reads the interface groups here, the
    # K-vector product the interface slices: two layouts, the same bits
    assert S.iface_layout()["groups"]
    m = ref.maps
    rng = np.random.default_rng(40 + k)
    Xg = rng.uniform(-1, 1, (p.A.n, k))
    Xl = np.stack([ref.scatter(Xg[:, j]) for j in range(k)], axis=1)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Xd = _t(Xl).to(dt)
    Y = S.spmm(Xd).cpu().numpy()
    absAx = abs(p.A.to_scipy()) @ np.abs(Xg)
    L = np.diff(p.A.rowptr)
    u = U if prec == "fp64" else 2.0**-24
    for j in range(k):
        col = Xd[:, j].contiguous()
        y1 = torch.empty_like(col)
        S.spmv_prec(col, y1, prec)
        assert np.array_equal(Y[:, j], y1.cpu().numpy()), "column %d differs from the single-vector product" % j
        if prec == "fp64":
            y_ref = ref.spmv(Xl[:, j])
        else:
            y_ref = ref.spmv32(Xl[:, j].astype(np.float32)).astype(np.float64)
        bound = 4.0 * (L[m.l2g] + m.mult[m.l2g]) * u * absAx[m.l2g, j] * 1.0001
        assert np.all(np.abs(Y[:, j].astype(np.float64) - y_ref) <= bound)
        assert np.array_equal(Y[:, j], Y[m.own, j][m.l2g])


def test_spmm_rejects_bad_arguments(ctx, fv20):
    import torch

    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p, ref = fv20
    S = System(ctx, p.A, p.part, p.P)
    X = torch.zeros((ref.maps.nloc, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(ssg.SSGError):
        S.spmm(X)
    X = torch.zeros((ref.maps.nloc, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(ssg.SSGError):
        S.spmm(X, out=X)


def test_block_early_iterates(ctx, fv20):
    """Six iterations of 16 columns together equal six iterations of each
    column's oracle solve to 1e-10."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p, ref = fv20
    S = System(ctx, p.A, p.part, p.P)
    B = p.b.T.copy()
    x, rc, st = S.solve(_t(B), rtol=0.0, max_iter=6)
    assert rc == ssg.SSG_E_NOT_CONVERGED
    X = x.cpu().numpy()
    for j in range(B.shape[0]):
        r = ref.cg(B[j], 0.0, 6)
        assert st[j]["iters"] == 6 and st[j]["block"] == 16
        assert _rel(X[j], r.x) <= 1e-10


def test_block_converged_and_counts(ctx, fv20):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p, ref = fv20
    S = System(ctx, p.A, p.part, p.P)
    B = p.b.T.copy()
    x, rc, st = S.solve(_t(B), rtol=1e-12, max_iter=100000)
    assert rc == ssg.SSG_OK
    X = x.cpu().numpy()
    for j in range(B.shape[0]):
        r = ref.cg(B[j], 1e-12, 100000)
        assert _rel(X[j], r.x) <= 1e-10
        assert st[j]["true_relres"] <= 1e-11
    x8, rc8, st8 = S.solve(_t(B), rtol=1e-8, max_iter=100000)
    assert rc8 == ssg.SSG_OK
    for j in range(B.shape[0]):
        r = ref.cg(B[j], 1e-8, 100000)
        assert abs(st8[j]["iters"] - r.iters) <= max(2, 0.03 * r.iters)
        kap = oracle.cond_from_lanczos(r.alpha, r.beta)
        assert _rel(x8.cpu().numpy()[j], p.xstar[:, j]) <= 2 * kap * 1e-8


def test_block_equal_and_zero_columns(ctx, fv20):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p, ref = fv20
    S = System(ctx, p.A, p.part, p.P)
    B = np.stack([p.b[:, 0], p.b[:, 0], np.zeros(p.A.n), p.b[:, 1], p.b[:, 0]])  # k = 5 -> K = 8, 3 padding
    x, rc, st = S.solve(_t(B), rtol=1e-9)
    assert rc == ssg.SSG_OK
    X = x.cpu().numpy()
    assert np.array_equal(X[0], X[1]) and np.array_equal(X[0], X[4])
    assert st[0]["iters"] == st[1]["iters"] == st[4]["iters"]
    assert st[2]["iters"] == 0 and np.all(X[2] == 0.0) and st[2]["status"] == ssg.SSG_OK
    assert st[0]["block"] == 8
    # the same right-hand side alone (single-vector path) converges at the same count within the tolerance
    ctx.set_rhs_block(1)
    try:
        x1, rc1, st1 = S.solve(_t(B[:1]), rtol=1e-9)
    finally:
        ctx.set_rhs_block(16)
    assert st1[0]["block"] == 1
    assert abs(st1[0]["iters"] - st[0]["iters"]) <= max(2, 0.03 * st1[0]["iters"])
    r = ref.cg(B[0], 1e-9, 100000)
    kap = oracle.cond_from_lanczos(r.alpha, r.beta)
    assert _rel(X[0], x1.cpu().numpy()[0]) <= 4 * kap * 1e-9


def test_block_split_and_padding(ctx):
    """k = 17 runs a block of 16 and one single solve; k = 3 pads to K = 4."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    rng = np.random.default_rng(17)
    A = random_spd(900, 7.0, rng)
    part = rng.integers(0, 6, A.n).astype(np.int32)
    ref = oracle.Partition(A, part, 6)
    S = System(ctx, A, part, 6)
    for k in (3, 17):
        B = rng.uniform(-1, 1, (k, A.n))
        x, rc, st = S.solve(_t(B), rtol=1e-12, max_iter=5000)
        assert rc == ssg.SSG_OK
        X = x.cpu().numpy()
        for j in range(k):
            r = ref.cg(B[j], 1e-12, 5000)
            assert _rel(X[j], r.x) <= 1e-10
        if k == 17:
            assert [s["block"] for s in st] == [16] * 16 + [1]
        else:
            assert [s["block"] for s in st] == [4] * 3


def test_block_with_guess_and_host_entry(ctx, fv20):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p, ref = fv20
    S = System(ctx, p.A, p.part, p.P)
    B = p.b.T[:4].copy()
    x0 = np.random.default_rng(3).uniform(-1, 1, B.shape)
    x, rc, st = S.solve(_t(B), x=_t(x0), rtol=1e-12)
    assert rc == ssg.SSG_OK
    for j in range(4):
        r = ref.cg(B[j], 1e-12, 100000, x0=x0[j])
        assert _rel(x.cpu().numpy()[j], r.x) <= 1e-10
    xh = np.zeros_like(B)
    rc, sth = S.solve_host(B, xh, rtol=1e-12)
    assert rc == ssg.SSG_OK
    for j in range(4):
        assert _rel(xh[j], p.xstar[:, j]) <= 1e-8


def test_block_drivers_agree(ctx, fv20):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p, _ = fv20
    S = System(ctx, p.A, p.part, p.P)
    B = _t(p.b.T.copy())
    for mode in (ssg.SSG_FP64, ssg.SSG_MIXED):
        x1, rc1, s1 = S.solve(B, rtol=1e-8, mode=mode)
        ctx.set_driver(ssg.SSG_DRIVER_HOST)
        try:
            x2, rc2, s2 = S.solve(B, rtol=1e-8, mode=mode)
        finally:
            ctx.set_driver(ssg.SSG_DRIVER_GRAPH)
        assert rc1 == rc2 == ssg.SSG_OK
        assert np.array_equal(x1.cpu().numpy(), x2.cpu().numpy())
        assert [(a["iters"], a["outer"]) for a in s1] == [(a["iters"], a["outer"]) for a in s2]


def test_block_mixed_matches_oracle(ctx, fv20):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p, ref = fv20
    S = System(ctx, p.A, p.part, p.P)
    B = p.b.T.copy()
    x, rc, st = S.solve(_t(B), rtol=1e-8, max_iter=100000, mode=ssg.SSG_MIXED)
    assert rc == ssg.SSG_OK
    X = x.cpu().numpy()
    for j in range(B.shape[0]):
        rm = ref.cg_mixed(B[j], 1e-8, 100000, 1e-4, 30)
        tr = np.linalg.norm(B[j] - oracle.spmv(p.A, X[j])) / np.linalg.norm(B[j])
        assert tr <= 1.0001e-8
        assert abs(st[j]["true_relres"] - tr) <= 1e-6 * tr + 1e-16
        assert abs(st[j]["outer"] - rm.outer) <= 1
        assert abs(st[j]["iters"] - rm.iters) <= max(3 * rm.outer, 0.10 * rm.iters)
        r64 = ref.cg(B[j], 1e-8, 100000)
        kap = oracle.cond_from_lanczos(r64.alpha, r64.beta)
        assert _rel(X[j], rm.x) <= 2 * kap * 1e-8


@pytest.mark.parametrize("k", [16, 4])
def test_block_autotune_same_bits(ctx, k):
    """ssg_autotune_block times six (entries at once, L2 look-ahead)
    candidates of the K-vector product in both precisions and keeps the
    fastest; none changes the arithmetic, so solves before and after tuning
    give the same bits and counts (FP64 and mixed)."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p = config_problem(5, scale=20)
    B = _t(p.b.T[:k].copy())
    S = System(ctx, p.A, p.part, p.P)
    before = [S.solve(B, rtol=1e-8, mode=m) for m in (ssg.SSG_FP64, ssg.SSG_MIXED)]
    t = S.autotune_block(k, reps=3)
    assert t["k"] == k
    assert 0 <= t["fp64_choice"] < ssg.TUNE_BLOCK_CANDIDATES and 0 <= t["fp32_choice"] < ssg.TUNE_BLOCK_CANDIDATES
    assert all(v > 0 for v in t["fp64_us"] + t["fp32_us"])
    assert t["fp32_us"][t["fp32_choice"]] == min(t["fp32_us"])
    assert sorted(set(t["nc"])) == [1, 2] and sorted(set(t["l2_ahead"])) == [0, 1, 2]
    after = [S.solve(B, rtol=1e-8, mode=m) for m in (ssg.SSG_FP64, ssg.SSG_MIXED)]
    for (x0, rc0, s0), (x1, rc1, s1) in zip(before, after):
        assert rc0 == rc1 == ssg.SSG_OK
        assert np.array_equal(x0.cpu().numpy(), x1.cpu().numpy())
        assert [(a["iters"], a["outer"]) for a in s0] == [(a["iters"], a["outer"]) for a in s1]
    with pytest.raises(ssg.SSGError):
        S.autotune_block(3)
    S.close()


@pytest.mark.parametrize("seed", range(0, 40, 3))
def test_spmm_random_systems_bitwise(ctx, seed):
    """The seeded random systems of the host-map sweep (empty and unused
    subdomains, isolated nodes): every column of the 2-, 4-, 8- and
    16-vector products, FP64 and FP32, bit-identical to the single-vector
    product of that column."""
    import torch

    from paper_2108_13162_gb300.ssg import System
    from tests.test_abi_host import _random_case

    A, part, P = _random_case(seed)
    S = System(ctx, A, part, P)
    ref = oracle.Partition(A, part, P)
    rng = np.random.default_rng(seed)
    for k in (2, 4, 8, 16):
        Xl = np.stack([ref.scatter(rng.uniform(-1, 1, A.n)) for _ in range(k)], axis=1)
        for dt, prec in ((torch.float64, "fp64"), (torch.float32, "fp32")):
            Xd = _t(Xl).to(dt)
            Y = S.spmm(Xd).cpu().numpy()
            for j in range(k):
                col = Xd[:, j].contiguous()
                y1 = torch.empty_like(col)
                S.spmv_prec(col, y1, prec)
                assert np.array_equal(Y[:, j], y1.cpu().numpy()), (k, prec, j)
    S.close()
