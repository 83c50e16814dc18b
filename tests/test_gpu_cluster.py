"""The one-cluster solve (k_cg_cluster: Algorithm 3 with M = I or the
diagonal preconditioner, every iteration inside one thread-block cluster)
through the C ABI, against the oracle and against the three-kernel loop.

Parity readings are those of the loop's tests: the first six iterates
within 1e-10 of the oracle's, a solution converged to 1e-12 within 1e-10 of
the oracle's, at 1e-8 the iteration count within max(2, 3 %) of the
oracle's and the recursive residual <= rtol.  The kernel groups its dots by
CTA and warp, not by block as the loop does, so against the loop the same
tolerances apply, not bit equality; repeated solves are bit-identical.

Cases: the systems the work items cover (sliced interior rows in every
layout, interface slices, rows longer than a slice, interface nodes whose
copy rows are long), systems smaller than a warp and smaller than one warp
per CTA (CTAs with no entries and no items), the size limit either side,
an initial guess, max_iter reached, b = 0, an indefinite matrix (breakdown
at the first iteration).
"""

import numpy as np
import pytest

import oracle
from synth import CSR, config_problem, laplace1d, poisson2d_5pt, random_spd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2108_13162_gb300 import build as ssg_build
    from paper_2108_13162_gb300.ssg import Context

    ssg_build.build()
    c = Context(0)
    if c.cluster_solve()[1] == 0:
        c.close()
        pytest.skip("the device places no cluster for the one-cluster solve")
    c.set_cluster_solve(FORCE)  # every case here through the cluster, whatever its size
    yield c
    torch.cuda.synchronize()
    c.close()


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# scatter, parameters, the cluster kernel, gather, true residual (product + dot)
CLUSTER_LAUNCHES = 6
DEFAULT_LIMIT = 12288  # local entries (ssg_set_cluster_solve's default)
FORCE = 1 << 20


def _hub(rng, n=3000):
    """Random SPD rows plus one node coupled to 200 others: a row longer than
    a slice, and with a random partition an interface node with long copy rows."""
    import scipy.sparse as sp

    A = random_spd(n, 7.0, rng)
    M = A.to_scipy().tolil()
    for j in range(1, 201):
        M[0, 10 * j] = M[10 * j, 0] = -0.01
        M[10 * j, 10 * j] += 0.01
    M[0, 0] += 2.0
    M = sp.csr_matrix(M)
    M.sort_indices()
    return CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))


def _cases():
    rng = np.random.default_rng(57)
    out = []
    p = config_problem(1)
    out.append(("p2d_64_2x2", p.A, p.part, p.P))
    p = config_problem(3, scale=96)
    out.append(("fe2d_96_rcb", p.A, p.part, p.P))
    A = random_spd(5000, 8.0, rng, shift=0.05)
    out.append(("rand5000_P13", A, rng.integers(0, 13, A.n).astype(np.int32), 13))
    A = _hub(rng)
    out.append(("hub3000_P4_interior", A, np.minimum(np.arange(A.n) * 4 // A.n, 3).astype(np.int32), 4))
    A = _hub(rng)
    out.append(("hub3000_P5_random", A, rng.integers(0, 5, A.n).astype(np.int32), 5))
    p = config_problem(2, scale=20)
    out.append(("fv3d_20", p.A, p.part, p.P))
    return out


CASES = _cases()


def _launches_say_cluster(st):
    return st["kernel_launches"] == CLUSTER_LAUNCHES


@pytest.mark.parametrize("mode", [0, 2], ids=["fp64", "fp64_jacobi"])
@pytest.mark.parametrize("name,A,part,P", CASES, ids=[c[0] for c in CASES])
def test_cluster_matches_oracle(ctx, name, A, part, P, mode):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    S = System(ctx, A, part, P)
    ref = oracle.Partition(A, part, P)
    b = np.random.default_rng(5).uniform(-1, 1, A.n)
    run = ref.pcg if mode == ssg.SSG_FP64_JACOBI else ref.cg
    r6 = run(b, 0.0, 6)
    x, rc, st = S.solve(_t(b), rtol=0.0, max_iter=6, mode=mode)
    assert _launches_say_cluster(st[0]), st[0]
    assert rc == ssg.SSG_E_NOT_CONVERGED and st[0]["iters"] == 6
    assert _rel(x.cpu().numpy(), r6.x) <= 1e-10
    r12 = run(b, 1e-12, 100000)
    x, rc, st = S.solve(_t(b), rtol=1e-12, max_iter=100000, mode=mode)
    assert rc == ssg.SSG_OK and r12.status == oracle.OK
    assert _rel(x.cpu().numpy(), r12.x) <= 1e-10
    r8 = run(b, 1e-8, 100000)
    x, rc, st = S.solve(_t(b), rtol=1e-8, max_iter=100000, mode=mode)
    assert rc == ssg.SSG_OK
    assert abs(st[0]["iters"] - r8.iters) <= max(2, 0.03 * r8.iters)
    assert st[0]["relres"] <= 1e-8
    tr = np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert abs(st[0]["true_relres"] - tr) <= 1e-6 * tr + 1e-15
    # repeated: the same bits
    x2, rc2, st2 = S.solve(_t(b), rtol=1e-8, max_iter=100000, mode=mode)
    assert np.array_equal(x.cpu().numpy(), x2.cpu().numpy()) and st2[0]["iters"] == st[0]["iters"]
    S.close()


@pytest.mark.parametrize("window", [1, 128, -1])
def test_cluster_sorted_layouts(ctx, window):
    """Interior slices sorted by row length (sorted-slice items): the same
    parity in every layout."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p = config_problem(3, scale=96)
    ctx.set_slice_sort(window)
    try:
        S = System(ctx, p.A, p.part, p.P)
    finally:
        ctx.set_slice_sort(0)
    if window != 1:
        assert S.layout()["sorted_subdomains"] > 0
    ref = oracle.Partition(p.A, p.part, p.P)
    b = p.b[:, 0]
    x, rc, st = S.solve(_t(b), rtol=0.0, max_iter=6)
    assert _launches_say_cluster(st[0])
    assert _rel(x.cpu().numpy(), ref.cg(b, 0.0, 6).x) <= 1e-10
    x, rc, st = S.solve(_t(b), rtol=1e-12, max_iter=100000, mode=ssg.SSG_FP64_JACOBI)
    assert rc == ssg.SSG_OK
    assert _rel(x.cpu().numpy(), ref.pcg(b, 1e-12, 100000).x) <= 1e-10
    S.close()


def test_cluster_against_loop(ctx):
    """The same system through both paths: early iterates and converged
    solutions agree to the parity tolerances, counts within max(2, 3 %)."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p = config_problem(2, scale=24)
    S = System(ctx, p.A, p.part, p.P)
    b = _t(p.b[:, 0])
    limit = ctx.cluster_solve()[0]
    out = {}
    for path, lim in (("cluster", limit), ("loop", 0)):
        ctx.set_cluster_solve(lim)
        try:
            x6, _, s6 = S.solve(b, rtol=0.0, max_iter=6)
            x12, rc12, s12 = S.solve(b, rtol=1e-12, max_iter=100000)
            x8, rc8, s8 = S.solve(b, rtol=1e-8, max_iter=100000, mode=ssg.SSG_FP64_JACOBI)
        finally:
            ctx.set_cluster_solve(limit)
        assert rc12 == ssg.SSG_OK and rc8 == ssg.SSG_OK
        assert _launches_say_cluster(s12[0]) == (path == "cluster")
        out[path] = (x6.cpu().numpy(), x12.cpu().numpy(), s12[0], x8.cpu().numpy(), s8[0])
    c, l = out["cluster"], out["loop"]
    assert _rel(c[0], l[0]) <= 1e-10
    assert _rel(c[1], l[1]) <= 1e-10
    assert abs(c[2]["iters"] - l[2]["iters"]) <= max(2, 0.03 * l[2]["iters"])
    assert abs(c[4]["iters"] - l[4]["iters"]) <= max(2, 0.03 * l[4]["iters"])
    S.close()


@pytest.mark.parametrize("n,P", [(1, 1), (7, 2), (31, 3), (300, 4), (600, 16), (2000, 7)])
def test_cluster_tiny_systems(ctx, n, P):
    """Fewer entries than one warp per CTA: CTAs with no entries and warps
    with no items take part in every barrier and sum."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    A = laplace1d(n) if n > 1 else CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.0]))
    part = (np.arange(n) * P // n).astype(np.int32)
    S = System(ctx, A, part, P)
    ref = oracle.Partition(A, part, P)
    b = np.random.default_rng(n).uniform(-1, 1, n)
    r = ref.cg(b, 1e-12, 10 * n + 10)
    x, rc, st = S.solve(_t(b), rtol=1e-12, max_iter=10 * n + 10)
    assert _launches_say_cluster(st[0])
    assert rc == ssg.SSG_OK and r.status == oracle.OK
    if n <= 64:
        assert st[0]["iters"] <= n  # finite termination, well-conditioned
    assert abs(st[0]["iters"] - r.iters) <= max(2, 0.03 * r.iters)
    assert _rel(x.cpu().numpy(), r.x) <= 1e-10
    S.close()


def test_cluster_size_limit(ctx):
    """A system with exactly max_nloc local entries runs as one cluster; one
    entry fewer allowed, the three-kernel loop runs."""
    from paper_2108_13162_gb300.ssg import System

    p = config_problem(1)
    S = System(ctx, p.A, p.part, p.P)
    nloc = S.sizes.nloc
    b = _t(p.b[:, 0])
    limit = ctx.cluster_solve()[0]
    try:
        ctx.set_cluster_solve(nloc)
        x1, _, s1 = S.solve(b, rtol=1e-10)
        ctx.set_cluster_solve(nloc - 1)
        x2, _, s2 = S.solve(b, rtol=1e-10)
    finally:
        ctx.set_cluster_solve(limit)
    assert _launches_say_cluster(s1[0])
    assert s2[0]["kernel_launches"] >= 3 * s2[0]["iters"]
    assert _rel(x1.cpu().numpy(), x2.cpu().numpy()) <= 1e-8


def test_cluster_guess_and_edges(ctx):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p = config_problem(1)
    S = System(ctx, p.A, p.part, p.P)
    ref = oracle.Partition(p.A, p.part, p.P)
    b = p.b[:, 0]
    # an initial guess (r = b - S x_1 from the guess's product)
    x0 = np.random.default_rng(3).uniform(-1, 1, p.A.n)
    x, rc, st = S.solve(_t(b), x=_t(x0), rtol=0.0, max_iter=6)
    # the product of the guess adds 2 launches before the cluster kernel
    assert st[0]["kernel_launches"] == CLUSTER_LAUNCHES + 2
    assert _rel(x.cpu().numpy(), ref.cg(b, 0.0, 6, x0).x) <= 1e-10
    x, rc, st = S.solve(_t(b), x=_t(x0), rtol=1e-12)
    assert rc == ssg.SSG_OK and _rel(x.cpu().numpy(), ref.cg(b, 1e-12, 100000, x0).x) <= 1e-10
    # max_iter = 1 from the guess: one iteration, not converged
    x, rc, st = S.solve(_t(b), x=_t(x0), rtol=1e-12, max_iter=1)
    assert rc == ssg.SSG_E_NOT_CONVERGED and st[0]["iters"] == 1
    assert _rel(x.cpu().numpy(), ref.cg(b, 1e-12, 1, x0).x) <= 1e-12
    # b = 0: converged before the first iteration, x = 0
    import torch

    x, rc, st = S.solve(torch.zeros(p.A.n, dtype=torch.float64, device="cuda"), rtol=1e-10)
    assert rc == ssg.SSG_OK and st[0]["iters"] == 0 and float(x.abs().max()) == 0.0
    # an indefinite matrix: (p, S p)_w < 0 at the first iteration
    A = poisson2d_5pt(10, 10)
    An = CSR(A.n, A.rowptr, A.colidx, -A.val)
    S2 = System(ctx, An, (np.arange(A.n) % 3).astype(np.int32), 3)
    x, rc, st = S2.solve(_t(np.ones(A.n)), rtol=1e-10)
    assert _launches_say_cluster(st[0])
    assert rc == ssg.SSG_E_BREAKDOWN and st[0]["iters"] == 0 and float(x.abs().max()) == 0.0
    S.close()
    S2.close()


def test_cluster_setting_checked(ctx):
    from paper_2108_13162_gb300 import ssg

    from paper_2108_13162_gb300.ssg import Context

    with pytest.raises(ssg.SSGError):
        ctx.set_cluster_solve(-1)
    limit, ctas = ctx.cluster_solve()
    with pytest.raises(ssg.SSGError):
        ctx.set_cluster_solve(limit, 3)
    assert limit == FORCE and ctas in (2, 4, 8, 16)
    c = Context(0)
    assert c.cluster_solve()[0] == DEFAULT_LIMIT
    c.close()


def test_cluster_not_under_host_driver(ctx):
    """The host-loop driver always runs the three-kernel loop, whatever the
    system's size; mixed precision too."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p = config_problem(1)
    S = System(ctx, p.A, p.part, p.P)
    b = _t(p.b[:, 0])
    ctx.set_driver(ssg.SSG_DRIVER_HOST)
    try:
        x, rc, st = S.solve(b, rtol=1e-10)
    finally:
        ctx.set_driver(ssg.SSG_DRIVER_GRAPH)
    assert rc == ssg.SSG_OK and st[0]["kernel_launches"] >= 3 * st[0]["iters"]
    x, rc, st = S.solve(b, rtol=1e-10, mode=ssg.SSG_MIXED)
    assert rc == ssg.SSG_OK and st[0]["kernel_launches"] > CLUSTER_LAUNCHES
    S.close()


@pytest.mark.parametrize("ctas", [2, 4, 8, 16])
def test_cluster_sizes(ctx, ctas):
    """Clusters of 2, 4, 8 and 16 CTAs (work items dealt to the CTAs in turn,
    vector entries in runs per CTA): the same parity with the oracle, the
    plain and the preconditioned solve."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    if ctas > ctx.cluster_solve()[1]:
        pytest.skip("the device places no cluster of %d CTAs" % ctas)
    p = config_problem(2, scale=16)
    ctx.set_cluster_solve(FORCE, ctas)
    try:
        S = System(ctx, p.A, p.part, p.P)
    finally:
        ctx.set_cluster_solve(FORCE, 0)
    ref = oracle.Partition(p.A, p.part, p.P)
    b = p.b[:, 0]
    for mode, run in ((ssg.SSG_FP64, ref.cg), (ssg.SSG_FP64_JACOBI, ref.pcg)):
        x, rc, st = S.solve(_t(b), rtol=0.0, max_iter=6, mode=mode)
        assert _launches_say_cluster(st[0])
        assert _rel(x.cpu().numpy(), run(b, 0.0, 6).x) <= 1e-10
        x, rc, st = S.solve(_t(b), rtol=1e-12, max_iter=100000, mode=mode)
        assert rc == ssg.SSG_OK and _rel(x.cpu().numpy(), run(b, 1e-12, 100000).x) <= 1e-10
    S.close()
