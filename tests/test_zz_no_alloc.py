"""The allocation-free weighted dot (ssg_wdot_noalloc) through the C ABI.

ssg_wdot_noalloc exists for callers that cannot let a library allocate
device memory: programs whose own allocator owns the device memory under a
fixed budget, and loops that must not take the implicit synchronisation of
cudaMalloc.  Its scratch is a static __device__ array shared by every call.
Its result is checked against the system's ssg_wdot and against the
oracle's weighted dot (Section 3.4.2, w = 1/m) on two calls in a row, and on
the edge cases: no entries, one block, and entries of multiplicity 0.
This file sorts last so that a stop-at-first-failure run has run every
other test first; it must also pass on its own in a fresh process.
"""

import ctypes as C
import math

import numpy as np
import pytest

import oracle
from synth import config_problem

pytestmark = pytest.mark.gpu

U = 2.0**-53


def _bound(n, w, u, v):
    # both sides are within gamma_n of the exact weighted sum
    return 4 * max(n, 1) * U * float(np.sum(w * np.abs(u * v)))


def test_noalloc_wdot_matches_system_and_oracle_twice():
    import torch

    from paper_2108_13162_gb300 import build as ssg_build
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Context, System

    ssg_build.build()
    p = config_problem(2, scale=40)
    ctx = Context(0)
    S = System(ctx, p.A, p.part, p.P)
    m = S.maps()
    mult_np = m["mult"][m["l2g"]].astype(np.uint8)
    mult_loc = torch.from_numpy(mult_np).cuda()
    w = 1.0 / mult_np
    Po = oracle.Partition(p.A, p.part, p.P)
    assert np.array_equal(Po.maps.w, w)
    rng = np.random.default_rng(17)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = S.sizes.nloc
    assert n > 4096  # several blocks
    for call in range(2):
        un = rng.uniform(-1, 1, n)
        vn = rng.uniform(-1, 1, n)
        u = torch.from_numpy(un).cuda()
        v = torch.from_numpy(vn).cuda()
        ref = S.wdot(u, v).item()
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        ssg.ssg_wdot_noalloc(u, v, mult_loc, out, stream)
        torch.cuda.synchronize()
        got = out.item()
        tol = _bound(n, w, un, vn)
        assert abs(got - ref) <= 2 * tol, (call, got, ref)
        assert abs(got - Po.wdot(un, vn)) <= 2 * tol, (call, got)

    # no entries: the result is 0 and nothing is read
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    ssg.ssg_wdot_noalloc(u[:0], v[:0], mult_loc[:0], out, stream)
    torch.cuda.synchronize()
    assert out.item() == 0.0

    # one block (fewer than 4096 entries), against the exact sum
    k = 1000
    ssg.ssg_wdot_noalloc(u[:k], v[:k], mult_loc[:k], out, stream)
    torch.cuda.synchronize()
    un, vn = u[:k].cpu().numpy(), v[:k].cpu().numpy()
    exact = math.fsum(w[:k] * un * vn)  # products rounded once, sum exact
    assert abs(out.item() - exact) <= _bound(k, w[:k], un, vn)

    # entries of multiplicity 0 carry weight 0, as in the system's weight table
    m0 = mult_loc.clone()
    m0[::7] = 0
    ssg.ssg_wdot_noalloc(u, v, m0, out, stream)
    torch.cuda.synchronize()
    un, vn = u.cpu().numpy(), v.cpu().numpy()
    w0 = w.copy()
    w0[::7] = 0.0
    exact = math.fsum(w0 * un * vn)
    assert math.isfinite(out.item())
    assert abs(out.item() - exact) <= _bound(n, w0, un, vn)

    # sizes beyond the static scratch are refused with a message, nothing launched
    L = ssg.lib()
    rc = L.ssg_wdot_noalloc(u.data_ptr(), v.data_ptr(), mult_loc.data_ptr(), 33554432 + 1, out.data_ptr(), None)
    assert rc == ssg.SSG_E_INVALID and "33554432" in ssg.last_error()
    S.close()
    ctx.close()
