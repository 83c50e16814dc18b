"""The owner-mask weighting of the weighted dots (ssg_set_weights,
SSG_WEIGHT_OWNER: w = 1 on a node's owner copy, 0 on its other copies)
through the C ABI, against the oracle with the same weights
(Partition.set_weights).

Parity readings are those of the default weighting's tests: the dot of
arbitrary local vectors within a rounding bound of the oracle's (the GPU sums
in another order: |d - d_ref| <= 2 nloc u sum_k |w_k u_k v_k|), the dot of
consistent vectors within the same bound of the global dot, a solve's first
six iterates within 1e-10 of the oracle's, a solution converged to 1e-12
within 1e-10 of the oracle's, iteration counts at 1e-8 within max(2, 3 %),
the mixed mode's FP64 true residual <= rtol.  Paths: the three-kernel loop,
the one-cluster solve, the diagonal preconditioner, mixed precision, several
right-hand sides together, a batch, element sub-structures (owner in the
lowest subdomain); switching back gives the default weighting's bits.
"""

import numpy as np
import pytest

import oracle
from synth import batch_problem, config_problem, fe_element_problem

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


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
    out = []
    p = config_problem(1)
    out.append(("p2d_64_2x2", p.A, p.part, p.P))  # one-cluster solve (small)
    p = config_problem(2, scale=24)
    out.append(("fv3d_24", p.A, p.part, p.P))  # three-kernel loop
    p = config_problem(3, scale=96)
    out.append(("fe2d_96_rcb", p.A, p.part, p.P))
    return out


CASES = _cases()


@pytest.mark.parametrize("name,A,part,P", CASES, ids=[c[0] for c in CASES])
def test_owner_dot(ctx, name, A, part, P):
    import torch

    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    S = System(ctx, A, part, P)
    ref = oracle.Partition(A, part, P)
    m = ref.maps
    rng = np.random.default_rng(2)
    ul = rng.uniform(-1, 1, m.nloc)
    vl = rng.uniform(-1, 1, m.nloc)
    d_inv = float(S.wdot(_t(ul), _t(vl)).cpu())
    S.set_weights(ssg.SSG_WEIGHT_OWNER)
    ref.set_weights(oracle.WEIGHT_OWNER)
    own = np.zeros(m.nloc)
    own[m.own] = 1.0
    bound = 2 * m.nloc * U * float(np.sum(own * np.abs(ul * vl)))
    assert abs(float(S.wdot(_t(ul), _t(vl)).cpu()) - ref.wdot(ul, vl)) <= bound
    # consistent vectors: the global dot
    u = rng.uniform(-1, 1, A.n)
    v = rng.uniform(-1, 1, A.n)
    g = float(u @ v)
    assert abs(float(S.wdot(_t(ref.scatter(u)), _t(ref.scatter(v))).cpu()) - g) <= 2 * m.nloc * U * float(
        np.abs(u) @ np.abs(v))
    # back to 1/m: the same bits as before
    S.set_weights(ssg.SSG_WEIGHT_INV_MULT)
    assert float(S.wdot(_t(ul), _t(vl)).cpu()) == d_inv
    with pytest.raises(ssg.SSGError):
        S.set_weights(2)
    torch.cuda.synchronize()
    S.close()


@pytest.mark.parametrize("mode", [0, 1, 2, 3], ids=["fp64", "mixed", "fp64_jacobi", "mixed_jacobi"])
@pytest.mark.parametrize("name,A,part,P", CASES, ids=[c[0] for c in CASES])
def test_owner_solves(ctx, name, A, part, P, mode):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    S = System(ctx, A, part, P)
    S.set_weights(ssg.SSG_WEIGHT_OWNER)
    ref = oracle.Partition(A, part, P)
    ref.set_weights(oracle.WEIGHT_OWNER)
    b = np.random.default_rng(9).uniform(-1, 1, A.n)
    if mode in (ssg.SSG_MIXED, ssg.SSG_MIXED_JACOBI):
        x, rc, st = S.solve(_t(b), rtol=1e-8, max_iter=100000, mode=mode)
        assert rc == ssg.SSG_OK
        tr = np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
        assert tr <= 1.0001e-8
        x12 = (ref.pcg if mode == ssg.SSG_MIXED_JACOBI else ref.cg)(b, 1e-12, 100000).x
        kap = oracle.cond_from_lanczos(*[getattr(ref.cg(b, 1e-8, 100000), k) for k in ("alpha", "beta")])
        assert _rel(x.cpu().numpy(), x12) <= 2 * kap * 1e-8
        S.close()
        return
    run = ref.pcg if mode == ssg.SSG_FP64_JACOBI else ref.cg
    x, rc, st = S.solve(_t(b), rtol=0.0, max_iter=6, mode=mode)
    assert _rel(x.cpu().numpy(), run(b, 0.0, 6).x) <= 1e-10
    x, rc, st = S.solve(_t(b), rtol=1e-12, max_iter=100000, mode=mode)
    assert rc == ssg.SSG_OK
    assert _rel(x.cpu().numpy(), run(b, 1e-12, 100000).x) <= 1e-10
    r8 = run(b, 1e-8, 100000)
    x, rc, st = S.solve(_t(b), rtol=1e-8, max_iter=100000, mode=mode)
    assert rc == ssg.SSG_OK and abs(st[0]["iters"] - r8.iters) <= max(2, 0.03 * r8.iters)
    tr = np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert abs(st[0]["true_relres"] - tr) <= 1e-6 * tr + 1e-15
    S.close()


def test_owner_switch_back_same_bits(ctx):
    """A loop solve and a one-cluster solve with the default weights, then with
    the owner mask, then the default again: the first and the last agree bit
    for bit (the graphs are rebuilt on each switch)."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    for p in (config_problem(1), config_problem(2, scale=24)):
        S = System(ctx, p.A, p.part, p.P)
        b = _t(p.b[:, 0])
        x0, _, s0 = S.solve(b, rtol=1e-10)
        S.set_weights(ssg.SSG_WEIGHT_OWNER)
        x1, rc1, s1 = S.solve(b, rtol=1e-10)
        assert rc1 == ssg.SSG_OK
        assert _rel(x1.cpu().numpy(), x0.cpu().numpy()) <= 1e-8
        S.set_weights(ssg.SSG_WEIGHT_INV_MULT)
        x2, _, s2 = S.solve(b, rtol=1e-10)
        assert np.array_equal(x2.cpu().numpy(), x0.cpu().numpy()) and s2[0]["iters"] == s0[0]["iters"]
        S.close()


def test_owner_several_rhs(ctx):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p = config_problem(2, scale=20)
    S = System(ctx, p.A, p.part, p.P)
    S.set_weights(ssg.SSG_WEIGHT_OWNER)
    ref = oracle.Partition(p.A, p.part, p.P)
    ref.set_weights(oracle.WEIGHT_OWNER)
    B = np.random.default_rng(4).uniform(-1, 1, (4, p.A.n))
    X, rc, st = S.solve(_t(B), rtol=0.0, max_iter=6)
    assert st[0]["block"] == 4
    for j in range(4):
        assert _rel(X[j].cpu().numpy(), ref.cg(B[j], 0.0, 6).x) <= 1e-10
    X, rc, st = S.solve(_t(B), rtol=1e-12, max_iter=100000)
    assert rc == ssg.SSG_OK
    for j in range(4):
        assert _rel(X[j].cpu().numpy(), ref.cg(B[j], 1e-12, 100000).x) <= 1e-10
    S.close()


def test_owner_batch(ctx):
    import torch

    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Batch

    bp = batch_problem(8, 8, 40)
    B = Batch(ctx, [(A, pt, P, b.shape[0]) for A, pt, P, b in zip(bp.A, bp.part, bp.P, bp.b)])
    B.set_weights(ssg.SSG_WEIGHT_OWNER)
    bb = torch.from_numpy(np.concatenate([b.ravel() for b in bp.b])).cuda()
    x, rc, st = B.solve(bb, rtol=1e-12, max_iter=100000)
    assert rc == ssg.SSG_OK
    xh = x.cpu().numpy()
    for s, (A, pt, P, b) in enumerate(zip(bp.A, bp.part, bp.P, bp.b)):
        ref = oracle.Partition(A, pt, P)
        ref.set_weights(oracle.WEIGHT_OWNER)
        o = int(B.rhs_off[s])
        xs = xh[o:o + b.size].reshape(b.shape)
        for j in range(b.shape[0]):
            assert _rel(xs[j], ref.cg(b[j], 1e-12, 100000).x) <= 1e-10
    B.close()


def test_owner_element_substructures(ctx):
    """Element sub-structures: the owner copy is the one in the lowest subdomain."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    ids, Ke, epart, P, A, xs, b = fe_element_problem(40, 3)
    S = System.from_elements(ctx, A.n, ids, Ke, epart, P)
    S.set_weights(ssg.SSG_WEIGHT_OWNER)
    ref = oracle.Partition.from_elements(A.n, ids, Ke, epart, P)
    ref.set_weights(oracle.WEIGHT_OWNER)
    bb = b[:, 0] if b.ndim == 2 else b
    x, rc, st = S.solve(_t(bb), rtol=0.0, max_iter=6)
    assert _rel(x.cpu().numpy(), ref.cg(bb, 0.0, 6).x) <= 1e-10
    x, rc, st = S.solve(_t(bb), rtol=1e-12, max_iter=100000)
    assert rc == ssg.SSG_OK and _rel(x.cpu().numpy(), ref.cg(bb, 1e-12, 100000).x) <= 1e-10
    S.close()


@pytest.mark.parametrize("seed", range(0, 40, 4))
def test_owner_dot_random_systems(ctx, seed):
    """The owner-mask dot on the seeded random systems of the host-map sweep:
    within the rounding bound of the oracle's, for arbitrary local vectors."""
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System
    from tests.test_abi_host import _random_case

    A, part, P = _random_case(seed)
    S = System(ctx, A, part, P)
    S.set_weights(ssg.SSG_WEIGHT_OWNER)
    ref = oracle.Partition(A, part, P)
    ref.set_weights(oracle.WEIGHT_OWNER)
    m = ref.maps
    rng = np.random.default_rng(seed)
    ul = rng.uniform(-1, 1, m.nloc)
    vl = rng.uniform(-1, 1, m.nloc)
    own = np.zeros(m.nloc)
    own[m.own] = 1.0
    bound = 2 * m.nloc * U * float(np.sum(own * np.abs(ul * vl))) + 1e-300
    assert abs(float(S.wdot(_t(ul), _t(vl)).cpu()) - ref.wdot(ul, vl)) <= bound
    S.close()
