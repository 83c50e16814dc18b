"""GPU batch of independent systems (ssg_partition_batch / ssg_solve_batch)
against the oracle's independent solves of each system, through the C ABI.

Workload 4's recipe at test size: 12 2D finite-volume systems with sides
8..40, 4 to 16 box subdomains and 1 to 8 right-hand sides each, all solved in
one graph launch.  Per (system, right-hand side) the readings of the
single-system parity tests hold: early iterates (k <= 6) within 1e-10,
solutions converged to 1e-12 within 1e-10, iteration counts at 1e-8 within
max(2, 3 %); mixed mode: refinements within +-1, inner iterations within
max(3 per refinement, 10 %), true residual <= rtol.  The graph and host-loop drivers give the
same bits; bad batch tables are refused.  Systems are solved in classes of
equal column count K (the power of two >= their right-hand-side count, at
least 2); the statistics come back in (system, right-hand side) order.
"""

import numpy as np
import pytest

import oracle
from synth import batch_problem

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


@pytest.fixture(scope="module")
def bp():
    return batch_problem(12, 8, 40)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _make(ctx, bp):
    from paper_2108_13162_gb300.ssg import Batch

    return Batch(ctx, [(A, pt, P, b.shape[0]) for A, pt, P, b in zip(bp.A, bp.part, bp.P, bp.b)])


def _b_all(bp):
    import torch

    return torch.from_numpy(np.concatenate([b.ravel() for b in bp.b])).cuda()


def _split(B, bp, x):
    x = x.cpu().numpy()
    out = []
    for s, b in enumerate(bp.b):
        o = int(B.rhs_off[s])
        out.append(x[o:o + b.size].reshape(b.shape))
    return out


def _each(bp):
    for s, (A, pt, P, b) in enumerate(zip(bp.A, bp.part, bp.P, bp.b)):
        ref = oracle.Partition(A, pt, P)
        for j in range(b.shape[0]):
            yield s, j, ref, b[j]


def test_batch_early_iterates_and_converged(ctx, bp):
    from paper_2108_13162_gb300 import ssg

    B = _make(ctx, bp)
    x, rc, st = B.solve(_b_all(bp), rtol=0.0, max_iter=6)
    assert rc == ssg.SSG_E_NOT_CONVERGED
    xs = _split(B, bp, x)
    t = 0
    for s, j, ref, b in _each(bp):
        # systems are grouped by the power of two >= their right-hand-side count (at least 2)
        k = bp.b[s].shape[0]
        assert st[t]["iters"] == 6 and st[t]["block"] == (2 if k <= 2 else 4 if k <= 4 else 8)
        assert _rel(xs[s][j], ref.cg(b, 0.0, 6).x) <= 1e-10
        t += 1
    x, rc, st = B.solve(_b_all(bp), rtol=1e-12, max_iter=100000)
    assert rc == ssg.SSG_OK
    xs = _split(B, bp, x)
    for s, j, ref, b in _each(bp):
        assert _rel(xs[s][j], ref.cg(b, 1e-12, 100000).x) <= 1e-10


def test_batch_counts_at_1e8(ctx, bp):
    from paper_2108_13162_gb300 import ssg

    B = _make(ctx, bp)
    x, rc, st = B.solve(_b_all(bp), rtol=1e-8, max_iter=100000)
    assert rc == ssg.SSG_OK
    t = 0
    iters = []
    for s, j, ref, b in _each(bp):
        r = ref.cg(b, 1e-8, 100000)
        assert abs(st[t]["iters"] - r.iters) <= max(2, 0.03 * r.iters)
        assert st[t]["true_relres"] <= 1.01e-8
        iters.append(r.iters)
        t += 1
    assert max(iters) > 2 * min(iters)  # uneven systems: early finishers are frozen, others go on


def test_batch_mixed(ctx, bp):
    from paper_2108_13162_gb300 import ssg

    B = _make(ctx, bp)
    x, rc, st = B.solve(_b_all(bp), rtol=1e-8, max_iter=100000, mode=ssg.SSG_MIXED)
    assert rc == ssg.SSG_OK
    xs = _split(B, bp, x)
    t = 0
    for s, j, ref, b in _each(bp):
        rm = ref.cg_mixed(b, 1e-8, 100000, 1e-4, 30)
        tr = np.linalg.norm(b - oracle.spmv(bp.A[s], xs[s][j])) / np.linalg.norm(b)
        assert tr <= 1.0001e-8
        assert abs(st[t]["outer"] - rm.outer) <= 1
        assert abs(st[t]["iters"] - rm.iters) <= max(3 * rm.outer, 0.10 * rm.iters)
        t += 1


def test_batch_drivers_agree(ctx, bp):
    from paper_2108_13162_gb300 import ssg

    B = _make(ctx, bp)
    for mode in (ssg.SSG_FP64, ssg.SSG_MIXED):
        x1, rc1, s1 = B.solve(_b_all(bp), rtol=1e-8, mode=mode)
        ctx.set_driver(ssg.SSG_DRIVER_HOST)
        try:
            x2, rc2, s2 = B.solve(_b_all(bp), rtol=1e-8, mode=mode)
        finally:
            ctx.set_driver(ssg.SSG_DRIVER_GRAPH)
        assert rc1 == rc2 == ssg.SSG_OK
        assert np.array_equal(x1.cpu().numpy(), x2.cpu().numpy())
        assert [(a["iters"], a["outer"]) for a in s1] == [(a["iters"], a["outer"]) for a in s2]
        # the column groups on streams of their own (the form a solve falls
        # back to when the one-graph form cannot be built): the same bits
        ssg.ssg_set_batch_graph(B.h, False)
        try:
            x3, rc3, s3 = B.solve(_b_all(bp), rtol=1e-8, mode=mode)
        finally:
            ssg.ssg_set_batch_graph(B.h, True)
        assert rc3 == ssg.SSG_OK
        assert np.array_equal(x1.cpu().numpy(), x3.cpu().numpy())
        assert [(a["iters"], a["outer"]) for a in s1] == [(a["iters"], a["outer"]) for a in s3]


def test_batch_rejects_bad_tables(ctx, bp):
    import scipy.sparse as sp

    from paper_2108_13162_gb300 import ssg

    A0, A1 = bp.A[0], bp.A[1]
    U = sp.block_diag([A0.to_scipy(), A1.to_scipy()], format="lil")
    U[0, A0.n] = -0.1  # couples the two systems
    U[A0.n, 0] = -0.1
    U = U.tocsr()
    U.sort_indices()
    part = np.concatenate([bp.part[0], bp.part[1] + bp.P[0]]).astype(np.int32)
    node_off = [0, A0.n, A0.n + A1.n]
    sub_off = [0, bp.P[0], bp.P[0] + bp.P[1]]
    with pytest.raises(ssg.SSGError):
        ssg.ssg_partition_batch(ctx.h, node_off, sub_off, [1, 1], U.indptr, U.indices, U.data, part)
    V = sp.block_diag([A0.to_scipy(), A1.to_scipy()], format="csr")
    V.sort_indices()
    bad = part.copy()
    bad[0] = bp.P[0]  # a node of system 0 in a subdomain of system 1
    with pytest.raises(ssg.SSGError):
        ssg.ssg_partition_batch(ctx.h, node_off, sub_off, [1, 1], V.indptr, V.indices, V.data, bad)
    with pytest.raises(ssg.SSGError):
        ssg.ssg_partition_batch(ctx.h, node_off, sub_off, [1, 17], V.indptr, V.indices, V.data, part)


def test_batch_mixed_shapes_and_guess(ctx):
    """Systems of different kinds and sizes (one subdomain, tiny, irregular),
    1-2 right-hand sides each (K = 2 with padding columns), with and without
    an initial guess: every solution converged to 1e-12 within 1e-10 of the
    oracle's."""
    import torch

    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Batch
    from synth import laplace1d, poisson2d_5pt, random_spd

    rng = np.random.default_rng(12)
    A0 = poisson2d_5pt(5, 4)
    A1 = random_spd(50, 5.0, rng)
    A2 = laplace1d(7)
    systems = [(A0, np.zeros(A0.n, np.int32), 1, 1), (A1, rng.integers(0, 3, A1.n).astype(np.int32), 3, 2),
               (A2, (np.arange(7) // 4).astype(np.int32), 2, 1)]
    B = Batch(ctx, systems)
    bs = [rng.uniform(-1, 1, (k, A.n)) for A, _, _, k in systems]
    b = torch.from_numpy(np.concatenate([v.ravel() for v in bs])).cuda()
    x0 = torch.from_numpy(rng.uniform(-1, 1, b.numel())).cuda()
    for guess in (None, x0):
        x, rc, st = B.solve(b, x=guess, rtol=1e-12, max_iter=10000)
        assert rc == ssg.SSG_OK
        xs = x.cpu().numpy()
        t = 0
        for s_, (A, part, P, k) in enumerate(systems):
            ref = oracle.Partition(A, part, P)
            o = int(B.rhs_off[s_])
            for j in range(k):
                g = None if guess is None else x0.cpu().numpy()[o + j * A.n:o + (j + 1) * A.n]
                r = ref.cg(bs[s_][j], 1e-12, 10000, x0=g)
                assert _rel(xs[o + j * A.n:o + (j + 1) * A.n], r.x) <= 1e-10
                assert st[t]["block"] == 2
                t += 1


def test_batch_jacobi(ctx, bp):
    """The batch with the diagonal preconditioner: SSG_FP64_JACOBI per (system,
    right-hand side) against or_sub_pcg (early iterates within 1e-10, counts
    at 1e-8 within max(2, 3 %)), SSG_MIXED_JACOBI against or_sub_pcg_mixed
    (refinements within +-1, inner iterations within max(3 per refinement,
    10 %), FP64 true residual <= rtol)."""
    from paper_2108_13162_gb300 import ssg

    B = _make(ctx, bp)
    x, rc, st = B.solve(_b_all(bp), rtol=0.0, max_iter=6, mode=ssg.SSG_FP64_JACOBI)
    assert rc == ssg.SSG_E_NOT_CONVERGED
    xs = _split(B, bp, x)
    t = 0
    for s, j, ref, b in _each(bp):
        assert st[t]["iters"] == 6
        assert _rel(xs[s][j], ref.pcg(b, 0.0, 6).x) <= 1e-10
        t += 1
    x, rc, st = B.solve(_b_all(bp), rtol=1e-8, max_iter=100000, mode=ssg.SSG_FP64_JACOBI)
    assert rc == ssg.SSG_OK
    t = 0
    for s, j, ref, b in _each(bp):
        r = ref.pcg(b, 1e-8, 100000)
        assert abs(st[t]["iters"] - r.iters) <= max(2, 0.03 * r.iters)
        assert st[t]["true_relres"] <= 1.01e-8
        t += 1
    x, rc, st = B.solve(_b_all(bp), rtol=1e-8, max_iter=100000, mode=ssg.SSG_MIXED_JACOBI)
    assert rc == ssg.SSG_OK
    xs = _split(B, bp, x)
    t = 0
    for s, j, ref, b in _each(bp):
        rm = ref.pcg_mixed(b, 1e-8, 100000, 1e-4, 30)
        tr = np.linalg.norm(b - oracle.spmv(bp.A[s], xs[s][j])) / np.linalg.norm(b)
        assert tr <= 1.0001e-8
        assert abs(st[t]["outer"] - rm.outer) <= 1
        assert abs(st[t]["iters"] - rm.iters) <= max(3 * rm.outer, 0.10 * rm.iters)
        t += 1


def test_batch_autotune_same_bits(ctx, bp):
    """Tuning every column group's K-vector product keeps the bits of the
    batch solve (FP64 and mixed)."""
    from paper_2108_13162_gb300 import ssg

    B = _make(ctx, bp)
    before = [B.solve(_b_all(bp), rtol=1e-8, mode=m) for m in (ssg.SSG_FP64, ssg.SSG_MIXED)]
    t = B.autotune_block(reps=3)
    assert t["k"] == 8  # the batch's largest column group (1-8 right-hand sides)
    after = [B.solve(_b_all(bp), rtol=1e-8, mode=m) for m in (ssg.SSG_FP64, ssg.SSG_MIXED)]
    for (x0, rc0, s0), (x1, rc1, s1) in zip(before, after):
        assert rc0 == rc1 == ssg.SSG_OK
        assert np.array_equal(x0.cpu().numpy(), x1.cpu().numpy())
        assert [(a["iters"], a["outer"]) for a in s0] == [(a["iters"], a["outer"]) for a in s1]
    B.close()
