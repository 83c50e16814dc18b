"""Differentiable sub-structured solves for torch.autograd.

Two functions with hand-written adjoints, every step in the library's CUDA
kernels (through the C ABI):

* ``solve(system, val, B)``: X with S(val) X_j = B_j for the k rows of B
  (Algorithm 3, all right-hand sides iterating together).  Backward: one
  more solve with the same operator, Lambda_j = S^-1 dL/dX_j (S symmetric),
  then dL/dB = Lambda and dL/dval_e = -sum_j Lambda_j[i] X_j[c] over the stored
  entries e = (i, c) (ssg_pattern_grad).
* ``fv7_values(system, dims, logk)``: the CSR values of the 7-point
  finite-volume operator with conductivity exp(logk) (ssg_fv7_values).
  Backward: dL/dlogk from dL/dval through the face coefficients
  (ssg_fv7_adjoint).

Composed, ``solve(system, fv7_values(system, dims, logk), B)`` is
differentiable in logk and B.
"""

from __future__ import annotations

import torch

from . import ssg


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, val, B, system, rtol, max_iter, mode):
        if not (B.is_cuda and B.dtype == torch.float64):
            raise TypeError("B must be a float64 CUDA tensor")
        n = system.sizes.n
        Bc = B.reshape(-1, n).contiguous()
        k = Bc.shape[0]
        ssg.ssg_set_values(system.h, val.contiguous())
        X = torch.zeros_like(Bc)
        rc, st = ssg.ssg_solve(system.h, k, Bc, X, False, rtol, max_iter, mode)
        if rc != ssg.SSG_OK:
            raise ssg.SSGError(rc, "forward solve")
        ctx.system = system
        ctx.args = (rtol, max_iter, mode, B.shape)
        ctx.stats = st
        ctx.save_for_backward(val, X)
        return X.reshape(B.shape)

    @staticmethod
    def backward(ctx, gX):
        val, X = ctx.saved_tensors
        rtol, max_iter, mode, shape = ctx.args
        system = ctx.system
        n = system.sizes.n
        G = gX.reshape(-1, n).contiguous()
        k = G.shape[0]
        ssg.ssg_set_values(system.h, val.contiguous())
        lam = torch.zeros_like(G)
        rc, st = ssg.ssg_solve(system.h, k, G, lam, False, rtol, max_iter, mode)
        if rc != ssg.SSG_OK:
            raise ssg.SSGError(rc, "adjoint solve")
        gval = None
        if ctx.needs_input_grad[0]:
            gval = torch.empty_like(val)
            ssg.ssg_pattern_grad(system.h, k, lam, X, gval)
        gB = lam.reshape(shape) if ctx.needs_input_grad[1] else None
        return gval, gB, None, None, None, None


class _Fv7(torch.autograd.Function):
    @staticmethod
    def forward(ctx, logk, system, dims):
        if not (logk.is_cuda and logk.dtype == torch.float64):
            raise TypeError("logk must be a float64 CUDA tensor")
        lk = logk.reshape(-1).contiguous()
        val = torch.empty(system.sizes.nnz, dtype=torch.float64, device=logk.device)
        ssg.ssg_fv7_values(system.h, *dims, lk, val)
        ctx.system = system
        ctx.dims = dims
        ctx.shape = logk.shape
        ctx.save_for_backward(lk)
        return val

    @staticmethod
    def backward(ctx, gval):
        (lk,) = ctx.saved_tensors
        glogk = torch.empty_like(lk)
        ssg.ssg_fv7_adjoint(ctx.system.h, *ctx.dims, lk, gval.contiguous(), glogk)
        return glogk.reshape(ctx.shape), None, None


def solve(system, val, B, rtol: float = 1e-10, max_iter: int = 0, mode: int = ssg.SSG_FP64):
    """X (same shape as B, rows = right-hand sides) with S(val) X_j = B_j."""
    return _Solve.apply(val, B, system, rtol, max_iter, mode)


def fv7_values(system, dims, logk):
    """CSR values of the 7-point finite-volume operator of an (nx, ny, nz)
    grid with conductivity exp(logk) (logk: n cells, x fastest)."""
    return _Fv7.apply(logk, system, tuple(int(d) for d in dims))
