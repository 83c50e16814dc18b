"""Write tests/golden/oracle_fv3d_128_4x4x4.json from the FP64 CPU oracle.

The full 128^3 finite-volume workload (4x4x4 boxes, kappa = exp(g),
g ~ N(0,1), x* ~ U[-1,1], b = A x*) solved by the oracle's sub-structured CG
(Algorithm 3, M = I) to a recursive relative residual of 1e-8 and of 1e-12, the
mixed-precision refinement (FP32 inner CG, FP64 residuals) to 1e-8,
Algorithm 3 with the diagonal preconditioner to 1e-8, and the refinement with
diagonal-preconditioned inner solves to 1e-8.  Stored per solve: the
iteration count, final residuals, the Lanczos condition estimate (M = I) and
the solution at 4096 seeded sample indices.  Also writes
tests/golden/oracle_p2d_64_2x2.json: the 64x64 Poisson system on 2x2
subdomains solved to 1e-10, with its whole solution.  Calls only oracle/ and
synth/; takes about three minutes of one CPU core.

    python tests/golden/make_oracle_golden.py            # everything
    python tests/golden/make_oracle_golden.py jacobi     # one part, merged into the file
    python tests/golden/make_oracle_golden.py p2d        # the 64x64 Poisson system (its own file)
"""

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from synth import config_problem  # noqa: E402

OUT = os.path.join(HERE, "oracle_fv3d_128_4x4x4.json")
OUT_P2D = os.path.join(HERE, "oracle_p2d_64_2x2.json")


ALL = ("cg", "mixed", "jacobi", "mixed_jacobi", "p2d")


def p2d():
    """The 64x64 5-point Poisson system on 2x2 subdomains (x* ~ U[-1,1],
    b = A x*) solved by the oracle's sub-structured CG (M = I) to 1e-10:
    iterations, residuals and the whole solution (4096 values)."""
    p = config_problem(1)
    part = oracle.Partition(p.A, p.part, p.P)
    b = p.b[:, 0]
    r = part.cg(b, 1e-10, 20000)
    assert r.status == oracle.OK
    rec = {
        "workload": p.name, "n": p.A.n, "nnz": p.A.nnz, "rtol": 1e-10, "iters": r.iters, "relres": r.relres,
        "true_relres": float(np.linalg.norm(b - oracle.spmv(p.A, r.x)) / np.linalg.norm(b)),
        "err_vs_xstar": float(np.linalg.norm(r.x - p.xstar[:, 0]) / np.linalg.norm(p.xstar[:, 0])),
        "x": [float(v) for v in r.x],
    }
    with open(OUT_P2D, "w") as f:
        json.dump(rec, f)
    print("p2d: %d iterations; wrote %s" % (r.iters, OUT_P2D))


def main(parts=ALL):
    if "p2d" in parts:
        p2d()
        parts = tuple(q for q in parts if q != "p2d")
        if not parts:
            return
    p = config_problem(2)
    part = oracle.Partition(p.A, p.part, p.P)
    b = p.b[:, 0]
    idx = np.sort(np.random.default_rng(2108).choice(p.A.n, 4096, replace=False))
    rec = {"workload": p.name, "n": p.A.n, "nnz": p.A.nnz, "sample_seed": 2108, "sample_idx": idx.tolist(),
           "solves": []}
    if set(parts) != set(ALL) and os.path.exists(OUT):
        with open(OUT) as f:
            old = json.load(f)
        assert old["sample_idx"] == rec["sample_idx"]
        rec = old
    for rtol in ((1e-8, 1e-12) if "cg" in parts else ()):
        t0 = time.time()
        r = part.cg(b, rtol, 20000)
        dt = time.time() - t0
        assert r.status == oracle.OK
        tr = float(np.linalg.norm(b - oracle.spmv(p.A, r.x)) / np.linalg.norm(b))
        rec["solves"].append({
            "rtol": rtol,
            "iters": r.iters,
            "relres": r.relres,
            "true_relres": tr,
            "kappa_lanczos": oracle.cond_from_lanczos(r.alpha, r.beta),
            "err_vs_xstar": float(np.linalg.norm(r.x - p.xstar[:, 0]) / np.linalg.norm(p.xstar[:, 0])),
            "sample_x": [float(v) for v in r.x[idx]],
            "oracle_seconds_one_core": dt,
        })
        print("rtol %g: %d iterations, %.1f s" % (rtol, r.iters, dt))
    if "cg" in parts:
        rec["solves"] = rec["solves"][-2:]
    if "mixed" in parts:
        mixed(p, part, b, idx, rec)
    if "jacobi" in parts:
        t0 = time.time()
        r = part.pcg(b, 1e-8, 20000)
        dt = time.time() - t0
        assert r.status == oracle.OK
        rec["jacobi"] = {
            "rtol": 1e-8,
            "iters": r.iters,
            "relres": r.relres,
            "true_relres": float(np.linalg.norm(b - oracle.spmv(p.A, r.x)) / np.linalg.norm(b)),
            "err_vs_xstar": float(np.linalg.norm(r.x - p.xstar[:, 0]) / np.linalg.norm(p.xstar[:, 0])),
            "sample_x": [float(v) for v in r.x[idx]],
            "oracle_seconds_one_core": dt,
        }
        print("jacobi: %d iterations, %.1f s" % (r.iters, dt))
    if "mixed_jacobi" in parts:
        t0 = time.time()
        r = part.pcg_mixed(b, 1e-8, 100000, 1e-4, 30)
        dt = time.time() - t0
        assert r.status == oracle.OK
        rec["mixed_jacobi"] = {
            "rtol": 1e-8,
            "inner_rtol": 1e-4,
            "iters": r.iters,
            "outer": r.outer,
            "relres": r.relres,
            "err_vs_xstar": float(np.linalg.norm(r.x - p.xstar[:, 0]) / np.linalg.norm(p.xstar[:, 0])),
            "sample_x": [float(v) for v in r.x[idx]],
            "oracle_seconds_one_core": dt,
        }
        print("mixed jacobi: %d inner iterations, %d refinements, %.1f s" % (r.iters, r.outer, dt))
    with open(OUT, "w") as f:
        json.dump(rec, f)
    print("wrote %s" % OUT)


def mixed(p, part, b, idx, rec):
    # mixed precision: FP32 inner CG (tolerance 1e-4) inside FP64 refinement to 1e-8
    t0 = time.time()
    r = part.cg_mixed(b, 1e-8, 100000, 1e-4, 30)
    dt = time.time() - t0
    assert r.status == oracle.OK
    rec["mixed"] = {
        "rtol": 1e-8,
        "inner_rtol": 1e-4,
        "iters": r.iters,
        "outer": r.outer,
        "relres": r.relres,
        "err_vs_xstar": float(np.linalg.norm(r.x - p.xstar[:, 0]) / np.linalg.norm(p.xstar[:, 0])),
        "sample_x": [float(v) for v in r.x[idx]],
        "oracle_seconds_one_core": dt,
    }
    print("mixed: %d inner iterations, %d refinements, %.1f s" % (r.iters, r.outer, dt))


if __name__ == "__main__":
    main(tuple(sys.argv[1:]) or ALL)
