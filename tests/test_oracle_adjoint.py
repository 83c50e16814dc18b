"""Pins for the oracle of the differentiable solve (oracle/adjoint.py).

The adjoint gradients dL/dB and dL/dlogk of
    L = sum_j || S(exp(logk))^-1 b_j - t_j ||^2
must equal central finite differences of L evaluated with dense LAPACK solves
(a route that shares nothing with the oracle's CG or its face rule), and the
pattern gradient must equal the derivative of L along a symmetric pair of
stored entries.  Planted mistakes in the face rule must each break a pin.
"""

import os
import types

import numpy as np
import pytest

import oracle
from oracle import adjoint
from synth import CSR, box_partition_3d, fv3d_7pt

DIMS = (5, 4, 6)


def _setup(seed=3, k=3):
    rng = np.random.default_rng(seed)
    nx, ny, nz = DIMS
    n = nx * ny * nz
    logk = rng.standard_normal(n)
    B = rng.uniform(-1, 1, (k, n))
    T = rng.uniform(-1, 1, (k, n))
    part = box_partition_3d(nx, ny, nz, 2, 2, 2)
    return logk, B, T, part


def _A(logk):
    nx, ny, nz = DIMS
    return fv3d_7pt(nx, ny, nz, np.exp(logk).reshape(nz, ny, nx))


def _loss_dense(logk, B, T):
    D = _A(logk).to_scipy().toarray()
    X = np.linalg.solve(D, B.T).T
    return float(np.sum((X - T) ** 2))


def _fd(f, v, h):
    g = np.zeros_like(v)
    for i in range(v.size):
        e = np.zeros_like(v)
        e.flat[i] = h
        g.flat[i] = (f(v + e) - f(v - e)) / (2 * h)
    return g


def pin_grads(mod=adjoint):
    logk, B, T, part = _setup()
    L, lam, glogk, X = mod.loss_and_grads(_A, DIMS, logk, B, T, part, 8, 1e-13)
    assert abs(L - _loss_dense(logk, B, T)) <= 1e-10 * L
    g_fd = _fd(lambda v: _loss_dense(v, B, T), logk, 1e-5)
    assert np.max(np.abs(glogk - g_fd)) <= 1e-6 * np.max(np.abs(g_fd))
    gb_fd = _fd(lambda v: _loss_dense(logk, v.reshape(B.shape), T), B.ravel(), 1e-5).reshape(B.shape)
    assert np.max(np.abs(lam - gb_fd)) <= 1e-6 * np.max(np.abs(gb_fd))


def test_adjoint_gradients_match_finite_differences():
    pin_grads()


def test_pattern_grad_matches_directional_derivative():
    """dL/dS_ic + dL/dS_ci equals d/de L(S + e (E_ic + E_ci)) for an
    off-diagonal pair, and dL/dS_ii equals d/de L(S + e E_ii)."""
    logk, B, T, part = _setup(seed=5)
    A = _A(logk)
    D = A.to_scipy().toarray()
    X = np.linalg.solve(D, B.T).T
    lam = np.linalg.solve(D, (2 * (X - T)).T).T
    g = adjoint.pattern_grad(A, lam, X)

    def L_of(Dm):
        Xm = np.linalg.solve(Dm, B.T).T
        return float(np.sum((Xm - T) ** 2))

    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    rng = np.random.default_rng(0)
    for e in rng.choice(A.nnz, 12, replace=False):
        i, c = rows[e], A.colidx[e]
        E = np.zeros_like(D)
        E[i, c] += 1.0
        if i != c:
            E[c, i] += 1.0
        h = 1e-6
        fd = (L_of(D + h * E) - L_of(D - h * E)) / (2 * h)
        # the symmetric partner's gradient
        pe = np.nonzero((rows == c) & (A.colidx == i))[0][0]
        an = g[e] + (g[pe] if i != c else 0.0)
        assert abs(an - fd) <= 1e-6 * max(1.0, abs(fd))


FACE_MUTATIONS = {
    "no_boundary_faces": ("    g += nbf * 2.0 * dLdt_b\n", "\n"),
    "wrong_derivative_operand": ("        g[lo] += dLdt * 2.0 * kb * kb / (s * s)",
                                 "        g[lo] += dLdt * 2.0 * ka * ka / (s * s)"),
    "sign_of_face_term": ("        dLdt = -np.sum((la - lb) * (xa - xb), axis=0)",
                          "        dLdt = np.sum((la - lb) * (xa - xb), axis=0)"),
    "no_chain_to_log": ("    return (k * g).ravel()", "    return g.ravel()"),
}


@pytest.mark.parametrize("name", sorted(FACE_MUTATIONS))
def test_face_rule_planted_mistake_is_caught(name):
    old, new = FACE_MUTATIONS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "adjoint.py")).read()
    assert src.count(old) == 1, name
    mod = types.ModuleType("oracle.adjoint_mutant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), "adjoint_mutant.py", "exec"), mod.__dict__)
    with pytest.raises(AssertionError):
        pin_grads(mod)
