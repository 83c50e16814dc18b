"""GPU mixed-precision solve (SSG_MIXED: FP32 inner CG inside FP64 iterative
refinement) against the oracle's or_sub_cg_mixed, through the C ABI.

Checks (the refinement has no exact counterpart to compare bit for bit: the
inner FP32 sums are ordered differently on each side):
  * converged, and the FP64 true residual ||b - S x|| / ||b|| recomputed on
    the CPU with the oracle's global product is <= rtol;
  * the refinement count equals the oracle's (+-1) and the summed inner
    iterations are within max(3 per refinement, 10 %) of the oracle's (an
    empirical tolerance, see the exact-count cases below);
  * on matrices with d distinct eigenvalues every inner solve takes exactly d
    iterations (finite termination): counts equal the oracle's exactly;
  * the solution is within 2 kappa rtol of x* and of the oracle's solution
    (kappa from the Lanczos coefficients of the FP64 oracle run);
  * both drivers (graph, host loop) give the same bits; the parameters are
    validated; a one-refinement cap stops with SSG_E_NOT_CONVERGED;
  * several iterations per loop pass give the bits of one.
"""

import json
import os

import numpy as np
import pytest

import oracle
from synth import CSR, config_problem

pytestmark = pytest.mark.gpu

UNROLL_DEFAULT = 4  # CG iterations per loop pass unless ssg_set_unroll says otherwise


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


CASES = [
    ("config1", lambda: config_problem(1), 1e-10),
    ("fv3d_24", lambda: config_problem(2, scale=24), 1e-8),
    ("fv3d_40", lambda: config_problem(2, scale=40), 1e-8),
    ("fe2d_64", lambda: config_problem(3, scale=64), 1e-8),
]


@pytest.mark.parametrize("name,mk,rtol", CASES, ids=[c[0] for c in CASES])
def test_mixed_matches_oracle(ctx, name, mk, rtol):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p = mk()
    b = p.b[:, 0]
    S = System(ctx, p.A, p.part, p.P)
    ref = oracle.Partition(p.A, p.part, p.P)
    rm = ref.cg_mixed(b, rtol, 100000, 1e-4, 30)
    r64 = ref.cg(b, rtol, 100000)
    x, rc, st = S.solve(_t(b), rtol=rtol, max_iter=100000, mode=ssg.SSG_MIXED)
    assert rc == ssg.SSG_OK and rm.status == oracle.OK
    xg = x.cpu().numpy()
    tr = np.linalg.norm(b - oracle.spmv(p.A, xg)) / np.linalg.norm(b)
    assert tr <= 1.0001 * rtol
    assert abs(st[0]["true_relres"] - tr) <= 1e-6 * tr + 1e-16
    assert abs(st[0]["outer"] - rm.outer) <= 1
    assert abs(st[0]["iters"] - rm.iters) <= max(3 * rm.outer, 0.10 * rm.iters)
    kap = oracle.cond_from_lanczos(r64.alpha, r64.beta)
    assert _rel(xg, p.xstar[:, 0]) <= 2 * kap * rtol
    assert _rel(xg, rm.x) <= 2 * kap * rtol


# 2x2 blocks [[a, b], [b, a]] with d distinct eigenvalues, two refinements
# at rtol 1e-13 (both inner solves then run to the inner tolerance 1e-4):
# CG's finite termination fixes every inner solve at d iterations, so the
# counts of the GPU and of the oracle must agree exactly, not within a
# tolerance
COUNT_CASES = [
    ("d4_kappa27", [(14.0, 13.0), (6.0, 3.0)], 4),
    ("d3_kappa16", [(2.5, 1.5), (10.0, 6.0)], 3),
    ("d2_kappa4", [(5.0, 3.0)], 2),
]


@pytest.mark.parametrize("name,blocks,d", COUNT_CASES, ids=[c[0] for c in COUNT_CASES])
def test_mixed_counts_exact_on_finite_termination(ctx, name, blocks, d):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System
    from synth import pair_blocks

    ctx.set_mixed(1e-4, 2)
    try:
        for seed in range(2):
            rng = np.random.default_rng(seed)
            A = pair_blocks(blocks, 25)
            b = rng.uniform(-1, 1, A.n)
            part = rng.integers(0, 5, A.n).astype(np.int32)
            rm = oracle.Partition(A, part, 5).cg_mixed(b, 1e-13, 1000, 1e-4, 2)
            S = System(ctx, A, part, 5)
            x, rc, st = S.solve(_t(b), rtol=1e-13, max_iter=1000, mode=ssg.SSG_MIXED)
            assert rc in (ssg.SSG_OK, ssg.SSG_E_NOT_CONVERGED)
            assert (st[0]["iters"], st[0]["outer"]) == (rm.iters, rm.outer) == (2 * d, 2)
            tr = np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
            assert tr <= 1e-9
            S.close()
    finally:
        ctx.set_mixed(1e-4, 30)


def test_mixed_drivers_agree_and_deterministic(ctx):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p = config_problem(2, scale=20)
    S = System(ctx, p.A, p.part, p.P)
    b = _t(p.b[:, 0])
    x1, rc1, s1 = S.solve(b, rtol=1e-8, mode=ssg.SSG_MIXED)
    x2, rc2, s2 = S.solve(b, rtol=1e-8, mode=ssg.SSG_MIXED)
    assert np.array_equal(x1.cpu().numpy(), x2.cpu().numpy())
    ctx.set_driver(ssg.SSG_DRIVER_HOST)
    try:
        x3, rc3, s3 = S.solve(b, rtol=1e-8, mode=ssg.SSG_MIXED)
    finally:
        ctx.set_driver(ssg.SSG_DRIVER_GRAPH)
    assert rc1 == rc3 == ssg.SSG_OK
    assert (s3[0]["iters"], s3[0]["outer"]) == (s1[0]["iters"], s1[0]["outer"])
    assert np.array_equal(x3.cpu().numpy(), x1.cpu().numpy())


def test_mixed_parameters_and_caps(ctx):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    with pytest.raises(ssg.SSGError):
        ctx.set_mixed(0.0, 30)
    with pytest.raises(ssg.SSGError):
        ctx.set_mixed(1e-4, 0)
    p = config_problem(2, scale=16)
    S = System(ctx, p.A, p.part, p.P)
    ctx.set_mixed(1e-4, 1)
    try:
        x, rc, st = S.solve(_t(p.b[:, 0]), rtol=1e-10, mode=ssg.SSG_MIXED)
    finally:
        ctx.set_mixed(1e-4, 30)
    assert rc == ssg.SSG_E_NOT_CONVERGED and st[0]["outer"] == 1
    # identity: each refinement's inner solve ends after one iteration (its
    # alpha is 1 up to the FP32 rounding of two differently ordered sums)
    n = 500
    eye = CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    S2 = System(ctx, eye, (np.arange(n) % 5).astype(np.int32), 5)
    bb = np.float32(np.random.default_rng(1).uniform(-1, 1, n)).astype(np.float64)
    x, rc, st = S2.solve(_t(bb), rtol=1e-12, mode=ssg.SSG_MIXED)
    assert rc == 0 and st[0]["outer"] <= 3 and st[0]["iters"] == st[0]["outer"]
    assert _rel(x.cpu().numpy(), bb) <= 1e-12


def test_mixed_full_size_128cube(ctx):
    """The benchmark workload in mixed mode against the stored oracle run."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_fv3d_128_4x4x4.json")) as f:
        g = json.load(f)
    gm = g["mixed"]
    kap = [s for s in g["solves"] if s["rtol"] == 1e-8][0]["kappa_lanczos"]
    p = config_problem(2)
    b = p.b[:, 0]
    S = System(ctx, p.A, p.part, p.P)
    x, rc, st = S.solve(_t(b), rtol=1e-8, max_iter=100000, mode=ssg.SSG_MIXED)
    assert rc == 0
    xg = x.cpu().numpy()
    tr = np.linalg.norm(b - oracle.spmv(p.A, xg)) / np.linalg.norm(b)
    print("mixed 128^3: inner %d (oracle %d), outer %d (oracle %d), true relres %.3e" % (
        st[0]["iters"], gm["iters"], st[0]["outer"], gm["outer"], tr))
    assert tr <= 1.0001e-8
    assert abs(st[0]["outer"] - gm["outer"]) <= 1
    assert abs(st[0]["iters"] - gm["iters"]) <= max(3 * gm["outer"], 0.10 * gm["iters"])
    idx = np.array(g["sample_idx"])
    assert _rel(xg[idx], np.array(gm["sample_x"])) <= 2 * kap * 1e-8
    assert _rel(xg, p.xstar[:, 0]) <= 2 * kap * 1e-8


@pytest.mark.parametrize("mode", [0, 1, 2, 3], ids=["fp64", "mixed", "fp64_jacobi", "mixed_jacobi"])
def test_loop_unroll_same_bits(ctx, mode):
    """Several copies of an iteration per pass of the loop graph (the later
    copies of the last pass return at once) give the bits and counts of one
    copy per pass; the launch counts grow by the copies that ran idle (exact
    for the FP64 modes: u ceil(k / u) - k copies; whole copies, at most u - 1
    per refinement, for the mixed ones)."""
    import math

    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    with pytest.raises(ssg.SSGError):
        ctx.set_unroll(0)
    with pytest.raises(ssg.SSGError):
        ctx.set_unroll(9)
    p = config_problem(2, scale=24)
    b = _t(p.b[:, 0])
    out = {}
    limit = ctx.cluster_solve()[0]
    for u in (1, 3, 4, 8):
        ctx.set_unroll(u)
        try:
            S = System(ctx, p.A, p.part, p.P)
        finally:
            ctx.set_unroll(UNROLL_DEFAULT)
        ctx.set_cluster_solve(0)  # the loop graph, not the one-cluster kernel
        try:
            x, rc, st = S.solve(b, rtol=1e-8, mode=mode)
        finally:
            ctx.set_cluster_solve(limit)
        assert rc == ssg.SSG_OK
        out[u] = (x.cpu().numpy(), st[0])
        S.close()
    x1, s1 = out[1]
    for u, (x, st) in out.items():
        assert np.array_equal(x, x1), u
        assert (st["iters"], st["outer"]) == (s1["iters"], s1["outer"]), u
        extra = st["kernel_launches"] - s1["kernel_launches"]
        if mode in (ssg.SSG_FP64, ssg.SSG_FP64_JACOBI):
            assert extra == 3 * (u * math.ceil(s1["iters"] / u) - s1["iters"]), u
        else:
            assert extra % 3 == 0 and 0 <= extra <= 3 * (u - 1) * s1["outer"], u
