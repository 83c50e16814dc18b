"""Seeded synthetic inputs shared by the tests, the oracle and the bench.

This package only builds input data: sparse SPD matrices in CSR form from
discretised model problems (Section 2.4 of the paper: -div(k grad u) = f with
homogeneous Dirichlet data, by finite differences, finite volumes or P1 finite
elements), node-to-subdomain partition vectors, and manufactured right-hand
sides.  It contains none of the sub-structuring method's arithmetic (no local
matrices, no interface maps, no CG); both the CUDA path and the CPU oracle take
its arrays as plain inputs.
"""

from .problems import (  # noqa: F401
    CSR,
    Problem,
    poisson2d_5pt,
    laplace1d,
    fv3d_7pt,
    fv2d_5pt,
    BatchProblem,
    batch_problem,
    fe2d_p1_jittered,
    fe2d_p1_elements,
    fe_assemble,
    fe_element_problem,
    random_spd,
    pair_blocks,
    box_partition_2d,
    box_partition_3d,
    rcb_partition,
    manufactured_rhs,
    config_problem,
    CONFIG_SEED_BASE,
)
