"""The oracle's multi-threaded sub-structured CG (or_sub_cg_omp), the CPU
baseline on all host cores, against the single-threaded oracle it restates.

It differs from or_sub_cg only in how each weighted dot groups its sums
(per subdomain, then ascending s, as the paper's processes form them), so:
  * its result does not depend on the number of threads (bit for bit);
  * with one subdomain it is or_sub_cg bit for bit;
  * converged to 1e-12 it agrees with or_sub_cg to 1e-10, and at 1e-8 its
    iteration count is within max(2, 3 %) and its solution within 2 kappa rtol
    of x*.
"""

import numpy as np

import oracle
from synth import config_problem, laplace1d


def test_omp_same_bits_for_any_thread_count():
    p = config_problem(2, scale=20)
    Pt = oracle.Partition(p.A, p.part, p.P)
    b = p.b[:, 0]
    ref = Pt.cg_omp(b, 1e-8, 5000, 1)
    assert ref.status == oracle.OK
    for nt in (2, 3, 8):
        r = Pt.cg_omp(b, 1e-8, 5000, nt)
        assert r.iters == ref.iters and np.array_equal(r.x, ref.x), nt


def test_omp_one_subdomain_is_serial_oracle():
    for A in (laplace1d(50), config_problem(2, scale=12).A):
        b = np.random.default_rng(4).uniform(-1, 1, A.n)
        Pt = oracle.Partition(A, np.zeros(A.n, np.int32), 1)
        r0 = Pt.cg(b, 1e-10, 10 * A.n)
        r1 = Pt.cg_omp(b, 1e-10, 10 * A.n, 4)
        assert r0.status == r1.status == oracle.OK
        assert r0.iters == r1.iters and np.array_equal(r0.x, r1.x)


def test_omp_agrees_with_serial_oracle():
    p = config_problem(2, scale=24)
    Pt = oracle.Partition(p.A, p.part, p.P)
    b = p.b[:, 0]
    r0 = Pt.cg(b, 1e-12, 10000)
    r1 = Pt.cg_omp(b, 1e-12, 10000, 0)
    assert r1.status == oracle.OK
    assert np.linalg.norm(r1.x - r0.x) <= 1e-10 * np.linalg.norm(r0.x)
    r0 = Pt.cg(b, 1e-8, 10000)
    r1 = Pt.cg_omp(b, 1e-8, 10000, 0)
    assert abs(r1.iters - r0.iters) <= max(2, 0.03 * r0.iters)
    kap = oracle.cond_from_lanczos(r0.alpha, r0.beta)
    xs = p.xstar[:, 0]
    assert np.linalg.norm(r1.x - xs) <= 2 * kap * 1e-8 * np.linalg.norm(xs)
    tr = np.linalg.norm(b - oracle.spmv(p.A, r1.x)) / np.linalg.norm(b)
    assert tr <= 1.01e-8
