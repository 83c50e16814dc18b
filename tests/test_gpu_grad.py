"""GPU differentiable solve (ssg_set_values, ssg_pattern_grad, ssg_fv7_*,
paper_2108_13162_gb300.autograd) against the oracle, through the C ABI.

  * ssg_fv7_values equals the generator's 7-point matrix to 4 ulp per entry
    (CUDA's exp and numpy's may differ in the last bit);
  * after ssg_set_values the device operator is bit-identical to one built
    by ssg_partition from the new values (FP64 and FP32 products);
  * ssg_pattern_grad equals -sum_j lam_j[i] x_j[c] within the FMA-chain bound;
  * ssg_fv7_adjoint equals the oracle's face rule on the same lambda, x to
    rounding (1e-12 relative);
  * end to end on 16^3 (the 96^3 workload's recipe, 3x3x3 boxes, 16
    right-hand sides): dL/dB and dL/dlogk match the oracle's adjoint gradients
    (solves to 1e-12: 1e-8 relative), and central finite differences of the
    GPU loss (solves to 1e-13) along random directions;
  * mixed mode (FP32 inner solves) gives gradients within 2 kappa rtol.
"""

import numpy as np
import pytest

import oracle
from oracle import adjoint
from synth import config_problem, fv3d_7pt

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


@pytest.fixture(scope="module")
def fv16():
    p = config_problem(5, scale=16)
    s = 16
    rng = np.random.default_rng(2108)
    T = rng.uniform(-1, 1, (16, p.A.n))
    return p, (s, s, s), p.meta["log_kappa"].ravel().copy(), T


def test_fv7_values_match_generator(ctx, fv16):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p, dims, logk, _ = fv16
    S = System(ctx, p.A, p.part, p.P)
    val = _t(np.zeros(p.A.nnz))
    ssg.ssg_fv7_values(S.h, *dims, _t(logk), val)
    v = val.cpu().numpy()
    assert np.all(np.abs(v - p.A.val) <= 4 * U * np.abs(p.A.val))
    # a grid that does not match the matrix is refused
    with pytest.raises(ssg.SSGError):
        ssg.ssg_fv7_values(S.h, 8, 32, 16, _t(logk), val)


def test_set_values_bitwise_equals_fresh_partition(ctx, fv16):
    import torch

    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p, dims, logk, _ = fv16
    nx, ny, nz = dims
    A1 = fv3d_7pt(nx, ny, nz, np.exp(0.5 * logk).reshape(nz, ny, nx))
    S0 = System(ctx, p.A, p.part, p.P)
    S1 = System(ctx, A1, p.part, p.P)
    ssg.ssg_set_values(S0.h, _t(A1.val))
    x = S0.scatter(_t(np.random.default_rng(1).uniform(-1, 1, p.A.n)))
    assert torch.equal(S0.spmv(x), S1.spmv(x))
    x32 = x.float()
    y0 = torch.empty_like(x32)
    y1 = torch.empty_like(x32)
    S0.spmv_prec(x32, y0, "fp32")
    S1.spmv_prec(x32, y1, "fp32")
    assert torch.equal(y0, y1)
    X = torch.stack([x] * 4, dim=1).contiguous()
    assert torch.equal(S0.spmm(X), S1.spmm(X))


def test_pattern_grad(ctx, fv16):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p, dims, logk, _ = fv16
    S = System(ctx, p.A, p.part, p.P)
    rng = np.random.default_rng(4)
    lam = rng.uniform(-1, 1, (5, p.A.n))
    x = rng.uniform(-1, 1, (5, p.A.n))
    g = _t(np.zeros(p.A.nnz))
    ssg.ssg_pattern_grad(S.h, 5, _t(lam), _t(x), g)
    ref = adjoint.pattern_grad(p.A, lam, x)
    rows = np.repeat(np.arange(p.A.n), np.diff(p.A.rowptr))
    scale = np.sum(np.abs(lam[:, rows] * x[:, p.A.colidx]), axis=0)
    assert np.all(np.abs(g.cpu().numpy() - ref) <= 8 * U * scale)


def test_fv7_adjoint_matches_face_rule(ctx, fv16):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p, dims, logk, _ = fv16
    S = System(ctx, p.A, p.part, p.P)
    rng = np.random.default_rng(6)
    lam = rng.uniform(-1, 1, (3, p.A.n))
    x = rng.uniform(-1, 1, (3, p.A.n))
    g = adjoint.pattern_grad(p.A, lam, x)
    out = _t(np.zeros(p.A.n))
    ssg.ssg_fv7_adjoint(S.h, *dims, _t(logk), _t(g), out)
    ref = adjoint.face_grad_logk(dims, logk, lam, x)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))


def _gpu_loss(S, dims, logk, B, T, rtol, mode=0, grad=True):
    import torch

    from paper_2108_13162_gb300 import autograd as ag

    lk = _t(logk).requires_grad_(grad)
    Bt = _t(B).requires_grad_(grad)
    X = ag.solve(S, ag.fv7_values(S, dims, lk), Bt, rtol=rtol, mode=mode)
    L = torch.sum((X - _t(T)) ** 2)
    if not grad:
        return float(L.item())
    L.backward()
    return float(L.item()), Bt.grad.cpu().numpy(), lk.grad.cpu().numpy(), X.detach().cpu().numpy()


def test_end_to_end_gradients_vs_oracle(ctx, fv16):
    from paper_2108_13162_gb300.ssg import System

    p, dims, logk, T = fv16
    S = System(ctx, p.A, p.part, p.P)
    B = p.b.T.copy()
    L, gB, gk, X = _gpu_loss(S, dims, logk, B, T, 1e-12)
    nx, ny, nz = dims
    Lr, lam_r, gk_r, X_r = adjoint.loss_and_grads(
        lambda v: fv3d_7pt(nx, ny, nz, np.exp(v).reshape(nz, ny, nx)), dims, logk, B, T, p.part, p.P, 1e-12)
    assert abs(L - Lr) <= 1e-9 * Lr
    assert np.linalg.norm(gB - lam_r) <= 1e-8 * np.linalg.norm(lam_r)
    assert np.linalg.norm(gk - gk_r) <= 1e-8 * np.linalg.norm(gk_r)


def test_end_to_end_finite_differences(ctx, fv16):
    p, dims, logk, T = fv16
    from paper_2108_13162_gb300.ssg import System

    S = System(ctx, p.A, p.part, p.P)
    B = p.b.T.copy()
    L, gB, gk, _ = _gpu_loss(S, dims, logk, B, T, 1e-13)
    rng = np.random.default_rng(9)
    h = 1e-3
    for _ in range(3):
        dk = rng.standard_normal(logk.shape)
        dk /= np.linalg.norm(dk)
        fd = (_gpu_loss(S, dims, logk + h * dk, B, T, 1e-13, grad=False)
              - _gpu_loss(S, dims, logk - h * dk, B, T, 1e-13, grad=False)) / (2 * h)
        an = float(np.dot(gk, dk))
        assert abs(an - fd) <= 2e-5 * max(abs(fd), np.linalg.norm(gk))
        db = rng.standard_normal(B.shape)
        db /= np.linalg.norm(db)
        fd = (_gpu_loss(S, dims, logk, B + h * db, T, 1e-13, grad=False)
              - _gpu_loss(S, dims, logk, B - h * db, T, 1e-13, grad=False)) / (2 * h)
        an = float(np.sum(gB * db))
        assert abs(an - fd) <= 2e-5 * max(abs(fd), np.linalg.norm(gB))


def test_mixed_mode_gradients(ctx, fv16):
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    p, dims, logk, T = fv16
    S = System(ctx, p.A, p.part, p.P)
    B = p.b.T.copy()
    L64, gB64, gk64, _ = _gpu_loss(S, dims, logk, B, T, 1e-12)
    Lm, gBm, gkm, _ = _gpu_loss(S, dims, logk, B, T, 1e-8, mode=ssg.SSG_MIXED)
    r = oracle.Partition(p.A, p.part, p.P).cg(B[0], 1e-8, 100000)
    kap = oracle.cond_from_lanczos(r.alpha, r.beta)
    assert abs(Lm - L64) <= 2 * kap * 1e-8 * L64
    assert np.linalg.norm(gBm - gB64) <= 4 * kap * 1e-8 * np.linalg.norm(gB64)
    assert np.linalg.norm(gkm - gk64) <= 4 * kap * 1e-8 * np.linalg.norm(gk64)
