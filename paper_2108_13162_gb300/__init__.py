"""Sub-structured Conjugate Gradient on one GB300 (sm_103a).

Cheik Ahamed & Magoules, "Parallel Sub-Structuring Methods for solving Sparse
Linear Systems on a cluster of GPU": a sparse SPD system is split into
subdomain matrices plus interface maps (Section 2.4) and solved with CG
(Algorithm 3) whose SpMV is local products plus interface assembly
(Section 3.4.1) and whose dots are interface-weighted (Section 3.4.2).  Here
all subdomains live on one GPU; the library is the C ABI in include/ssg.h,
built from csrc/ into _build/libssg.so, and ``ssg`` is its ctypes binding.
"""

from .ssg import Context, System  # noqa: F401
