"""The allocation-free weighted dot (ssg_wdot_noalloc) against the system's
ssg_wdot, through the C ABI.

ssg_wdot_noalloc exists for callers that cannot let a library allocate
device memory (during graph capture, under a framework-owned memory budget,
or where the implicit synchronisation of cudaMalloc is not acceptable); its
scratch is a static __device__ array shared by every call.  This file sorts
last so that a stop-at-first-failure run has run every other test first; it
must also pass on its own in a fresh process.
"""

import ctypes as C

import numpy as np
import pytest

from synth import config_problem

pytestmark = pytest.mark.gpu

U = 2.0**-53


def test_noalloc_wdot_matches_system_wdot_twice():
    import torch

    from paper_2108_13162_gb300 import build as ssg_build
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Context, System

    ssg_build.build()
    p = config_problem(2, scale=40)
    ctx = Context(0)
    S = System(ctx, p.A, p.part, p.P)
    m = S.maps()
    mult_loc = torch.from_numpy(m["mult"][m["l2g"]].astype(np.uint8)).cuda()
    rng = np.random.default_rng(17)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        u = torch.from_numpy(rng.uniform(-1, 1, S.sizes.nloc)).cuda()
        v = torch.from_numpy(rng.uniform(-1, 1, S.sizes.nloc)).cuda()
        ref = S.wdot(u, v)
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        ssg.ssg_wdot_noalloc(u, v, mult_loc, out, stream)
        torch.cuda.synchronize()
        w = 1.0 / m["mult"][m["l2g"]]
        scale = float(np.sum(w * np.abs(u.cpu().numpy() * v.cpu().numpy())))
        assert abs(out.item() - ref.item()) <= 4 * S.sizes.nloc * U * scale, (call, out.item(), ref.item())
    # sizes beyond the static scratch are refused with a message, nothing launched
    L = ssg.lib()
    rc = L.ssg_wdot_noalloc(u.data_ptr(), v.data_ptr(), mult_loc.data_ptr(), 33554432 + 1, out.data_ptr(), None)
    assert rc == ssg.SSG_E_INVALID and "33554432" in ssg.last_error()
    S.close()
    ctx.close()
