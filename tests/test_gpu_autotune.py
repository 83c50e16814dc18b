"""ssg_autotune: the chosen single-vector SpMV instances keep every parity
reading (SpMV entries within 4 (L_i + m_i) u (|A||x|)_i, converged solutions
within 1e-10 of the oracle's, iteration counts within max(2, 3 %)), report a
time per candidate, and solve bit-for-bit repeatably once chosen."""

import numpy as np
import pytest

import oracle
from synth import config_problem, random_spd

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


def _cases():
    rng = np.random.default_rng(77)
    p = config_problem(2, scale=40)
    out = [("fv3d_40", p.A, p.part, p.P, p.b[:, 0])]
    p = config_problem(3, scale=96)
    out.append(("fe2d_96", p.A, p.part, p.P, p.b[:, 0]))
    A = random_spd(4000, 9.0, rng)
    out.append(("rand4000_P11", A, rng.integers(0, 11, A.n).astype(np.int32), 11, rng.uniform(-1, 1, A.n)))
    return out


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_autotuned_parity(ctx, case):
    import torch

    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System

    _, A, part, P, b = case
    S = System(ctx, A, part, P)
    t = S.autotune(reps=5)
    assert 0 <= t["fp64_choice"] < ssg.TUNE_CANDIDATES and 0 <= t["fp32_choice"] < ssg.TUNE_CANDIDATES
    assert len(t["fp64_us"]) == len(t["fp32_us"]) == ssg.TUNE_CANDIDATES
    assert all(v > 0 for v in t["fp64_us"] + t["fp32_us"])
    assert t["fp64_us"][t["fp64_choice"]] == min(t["fp64_us"])
    ref = oracle.Partition(A, part, P)
    m = ref.maps
    x = np.random.default_rng(3).uniform(-1, 1, A.n)
    xl = ref.scatter(x)
    y = S.spmv(_t(xl)).cpu().numpy()
    absAx = abs(A.to_scipy()) @ np.abs(x)
    L = np.diff(A.rowptr)
    assert np.all(np.abs(y - ref.spmv(xl)) <= 4.0 * (L[m.l2g] + m.mult[m.l2g]) * U * absAx[m.l2g])
    x1, rc, st = S.solve(_t(b), rtol=1e-12, max_iter=100000)
    assert rc == ssg.SSG_OK
    assert np.linalg.norm(x1.cpu().numpy() - ref.cg(b, 1e-12, 100000).x) <= 1e-10 * np.linalg.norm(x1.cpu().numpy())
    x2, rc2, st2 = S.solve(_t(b), rtol=1e-12, max_iter=100000)
    assert torch.equal(x1, x2)
    x8, rc8, st8 = S.solve(_t(b), rtol=1e-8, max_iter=100000, mode=ssg.SSG_MIXED)
    assert rc8 == ssg.SSG_OK and st8[0]["true_relres"] <= 1.0001e-8
