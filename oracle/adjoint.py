"""FP64 CPU oracle of the differentiable solve (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU leg may
import this module; the CUDA library never calls it.

The loss of the differentiable workload is
    L(logk, B) = sum_j || x_j - t_j ||^2,   S(kappa) x_j = b_j,  kappa = exp(logk),
with S the 7-point finite-volume operator (harmonic-mean interior faces,
2 kappa on boundary faces).  Its gradient by the adjoint method:
    lambda_j = S^-1 dL/dx_j = S^-1 2 (x_j - t_j)     (S symmetric)
    dL/db_j  = lambda_j
    dL/dS_ic = -sum_j lambda_j[i] x_j[c]               (each stored entry)
    dL/dt_f  = -sum_j (lambda_j[a] - lambda_j[b]) (x_j[a] - x_j[b])   interior face (a, b)
             = -sum_j lambda_j[i] x_j[i]                              boundary face of i
    dL/dlogk_i = kappa_i sum over the faces f of i of dL/dt_f dt_f/dkappa_i,
    dt_f/dkappa_a = 2 kappa_b^2 / (kappa_a + kappa_b)^2 (interior), 2 (boundary).
The solves are the oracle's sub-structured CG (``Partition.cg``); the face
sums are written out per axis with numpy.  Pinned by central finite
differences of L computed with dense solves (tests/test_oracle_adjoint.py).
"""

from __future__ import annotations

import numpy as np

from . import Partition


def face_grad_logk(dims, logk, lam, x):
    """dL/dlogk from the adjoint and forward solutions (rows = right-hand sides)."""
    nx, ny, nz = dims
    k = np.exp(np.asarray(logk, dtype=np.float64)).reshape(nz, ny, nx)
    lam = np.asarray(lam, dtype=np.float64).reshape(-1, nz, ny, nx)
    x = np.asarray(x, dtype=np.float64).reshape(-1, nz, ny, nx)
    g = np.zeros((nz, ny, nx))
    for axis in range(3):  # z, y, x faces
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = slice(0, -1)
        hi[axis] = slice(1, None)
        lo, hi = tuple(lo), tuple(hi)
        ka, kb = k[lo], k[hi]
        la = lam[(slice(None),) + lo]
        lb = lam[(slice(None),) + hi]
        xa = x[(slice(None),) + lo]
        xb = x[(slice(None),) + hi]
        dLdt = -np.sum((la - lb) * (xa - xb), axis=0)
        s = ka + kb
        g[lo] += dLdt * 2.0 * kb * kb / (s * s)
        g[hi] += dLdt * 2.0 * ka * ka / (s * s)
    # boundary faces: one per side of the box a cell touches
    nbf = np.zeros((nz, ny, nx))
    nbf[0, :, :] += 1
    nbf[-1, :, :] += 1
    nbf[:, 0, :] += 1
    nbf[:, -1, :] += 1
    nbf[:, :, 0] += 1
    nbf[:, :, -1] += 1
    dLdt_b = -np.sum(lam * x, axis=0)
    g += nbf * 2.0 * dLdt_b
    return (k * g).ravel()


def pattern_grad(A, lam, x):
    """dL/dS over the stored entries of A (CSR order): -sum_j lam_j[i] x_j[c]."""
    lam = np.atleast_2d(lam)
    x = np.atleast_2d(x)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    return -np.sum(lam[:, rows] * x[:, A.colidx], axis=0)


def loss_and_grads(A_of_logk, dims, logk, B, T, part, P, rtol, max_iter=100000):
    """L and its gradients with respect to B (rows) and logk, by the adjoint
    method with the oracle's sub-structured CG.  A_of_logk builds the matrix."""
    A = A_of_logk(logk)
    Pt = Partition(A, part, P)
    B = np.atleast_2d(B)
    T = np.atleast_2d(T)
    X = np.stack([Pt.cg(B[j], rtol, max_iter).x for j in range(B.shape[0])])
    R = X - T
    L = float(np.sum(R * R))
    lam = np.stack([Pt.cg(2.0 * R[j], rtol, max_iter).x for j in range(B.shape[0])])
    return L, lam, face_grad_logk(dims, logk, lam, X), X
