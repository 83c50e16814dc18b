"""Seeded generators for sparse SPD systems, partitions and right-hand sides.

Every generator is deterministic for a given ``numpy.random.Generator`` state
(PCG64).  The matrices are the discretised model problem of Section 2.4
(Eq. model_problem / linear_systems: an elliptic operator with homogeneous
Dirichlet data gives a sparse symmetric positive-definite S), in CSR form as
described in Section 1.2 (values, column indices, row pointers), but 0-based
with int32 indices and float64 values.

Symmetry is exact: every off-diagonal value is computed once per edge/face and
written to both (i, j) and (j, i), so A == A^T bit for bit.  The partition
vectors assign every node (unknown) to one subdomain id in [0, P); the
sub-structuring itself (local matrices, interface maps) is not done here.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

CONFIG_SEED_BASE = 13162


@dataclass
class CSR:
    """0-based CSR matrix: ``rowptr`` (n+1, int32), ``colidx`` (nnz, int32),
    ``val`` (nnz, float64).  Columns are sorted and unique within each row."""

    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.colidx, self.rowptr), shape=(self.n, self.n))

    def digest(self) -> str:
        import hashlib

        h = hashlib.sha256()
        for a in (self.rowptr, self.colidx, self.val):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()


@dataclass
class Problem:
    """One synthetic system: matrix, node partition, manufactured solution(s)."""

    name: str
    A: CSR
    part: np.ndarray  # int32 [n], subdomain id of every node
    P: int
    xstar: np.ndarray  # float64 [n, k]
    b: np.ndarray  # float64 [n, k], b = A xstar
    meta: dict = field(default_factory=dict)


def _csr_from_stencil(cols: np.ndarray, vals: np.ndarray, mask: np.ndarray) -> CSR:
    """Build CSR from per-row candidate columns (already ascending) and a mask."""
    n = cols.shape[0]
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colidx = cols[mask].astype(np.int32)
    val = vals[mask].astype(np.float64)
    return CSR(n, rowptr.astype(np.int32), colidx, val)


def laplace1d(n: int) -> CSR:
    """Tridiagonal [-1, 2, -1] Dirichlet Laplacian on n interior points."""
    idx = np.arange(n)
    cols = np.stack([idx - 1, idx, idx + 1], axis=1)
    vals = np.tile(np.array([-1.0, 2.0, -1.0]), (n, 1))
    mask = (cols >= 0) & (cols < n)
    return _csr_from_stencil(cols, vals, mask)


def poisson2d_5pt(nx: int, ny: int) -> CSR:
    """5-point finite-difference Laplacian on an nx x ny interior grid.

    Node (ix, iy) has id ix + nx*iy.  Diagonal 4, neighbours -1; neighbours on
    the Dirichlet boundary are dropped; no h^2 scaling.
    """
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ix = ix.ravel()
    iy = iy.ravel()
    gid = ix + nx * iy
    cols = np.stack([gid - nx, gid - 1, gid, gid + 1, gid + nx], axis=1)
    mask = np.stack([iy > 0, ix > 0, np.ones_like(ix, bool), ix < nx - 1, iy < ny - 1], axis=1)
    vals = np.tile(np.array([-1.0, -1.0, 4.0, -1.0, -1.0]), (nx * ny, 1))
    return _csr_from_stencil(cols, vals, mask)


def fv3d_7pt(nx: int, ny: int, nz: int, kappa: np.ndarray) -> CSR:
    """Cell-centred finite-volume diffusion on an nx x ny x nz grid.

    Cell (ix, iy, iz) has id ix + nx*(iy + ny*iz); ``kappa`` is indexed
    [iz, iy, ix].  An interior face between cells a and b carries the harmonic
    mean t = 2 k_a k_b / (k_a + k_b); a boundary face (u = 0 outside) carries
    t = 2 k_i (half-cell distance).  A_ij = -t for each interior face and
    A_ii = sum of the six face coefficients of cell i, summed in the order
    z-, y-, x-, x+, y+, z+.
    """
    k = np.asarray(kappa, dtype=np.float64).reshape(nz, ny, nx)

    def harm(a, b):
        return 2.0 * a * b / (a + b)

    bnd = 2.0 * k
    # face coefficients seen from each cell, boundary faces use 2k
    txm = bnd.copy()
    txp = bnd.copy()
    tym = bnd.copy()
    typ = bnd.copy()
    tzm = bnd.copy()
    tzp = bnd.copy()
    fx = harm(k[:, :, :-1], k[:, :, 1:])
    txp[:, :, :-1] = fx
    txm[:, :, 1:] = fx
    fy = harm(k[:, :-1, :], k[:, 1:, :])
    typ[:, :-1, :] = fy
    tym[:, 1:, :] = fy
    fz = harm(k[:-1, :, :], k[1:, :, :])
    tzp[:-1, :, :] = fz
    tzm[1:, :, :] = fz
    diag = tzm + tym
    diag = diag + txm
    diag = diag + txp
    diag = diag + typ
    diag = diag + tzp

    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ix = ix.ravel()
    iy = iy.ravel()
    iz = iz.ravel()
    gid = ix + nx * (iy + ny * iz)
    sxy = nx * ny
    cols = np.stack([gid - sxy, gid - nx, gid - 1, gid, gid + 1, gid + nx, gid + sxy], axis=1)
    vals = np.stack(
        [-tzm.ravel(), -tym.ravel(), -txm.ravel(), diag.ravel(), -txp.ravel(), -typ.ravel(), -tzp.ravel()],
        axis=1,
    )
    mask = np.stack(
        [iz > 0, iy > 0, ix > 0, np.ones_like(ix, bool), ix < nx - 1, iy < ny - 1, iz < nz - 1], axis=1
    )
    return _csr_from_stencil(cols, vals, mask)


def fv2d_5pt(nx: int, ny: int, kappa: np.ndarray) -> CSR:
    """Cell-centred finite volumes on an nx x ny grid, the 2D counterpart of
    ``fv3d_7pt``: cell (ix, iy) has id ix + nx*iy, ``kappa`` is indexed
    [iy, ix], interior faces carry 2 k_a k_b / (k_a + k_b), boundary faces
    2 k, A_ii sums the four face coefficients in the order y-, x-, x+, y+."""
    k = np.asarray(kappa, dtype=np.float64).reshape(ny, nx)

    def harm(a, b):
        return 2.0 * a * b / (a + b)

    bnd = 2.0 * k
    txm, txp, tym, typ = bnd.copy(), bnd.copy(), bnd.copy(), bnd.copy()
    fx = harm(k[:, :-1], k[:, 1:])
    txp[:, :-1] = fx
    txm[:, 1:] = fx
    fy = harm(k[:-1, :], k[1:, :])
    typ[:-1, :] = fy
    tym[1:, :] = fy
    diag = tym + txm
    diag = diag + txp
    diag = diag + typ
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    ix = ix.ravel()
    iy = iy.ravel()
    gid = ix + nx * iy
    cols = np.stack([gid - nx, gid - 1, gid, gid + 1, gid + nx], axis=1)
    vals = np.stack([-tym.ravel(), -txm.ravel(), diag.ravel(), -txp.ravel(), -typ.ravel()], axis=1)
    mask = np.stack([iy > 0, ix > 0, np.ones_like(ix, bool), ix < nx - 1, iy < ny - 1], axis=1)
    return _csr_from_stencil(cols, vals, mask)


@dataclass
class BatchProblem:
    """Independent systems solved together: system s is (A[s], part[s], P[s])
    with right-hand sides b[s] (k_s x n_s)."""

    name: str
    A: list
    part: list
    P: list
    b: list
    meta: dict


def batch_problem(nsys: int = 512, side_lo: int = 32, side_hi: int = 512, seed: int = CONFIG_SEED_BASE + 4,
                  sigma: float = 0.5) -> BatchProblem:
    """Workload 4: nsys 2D variable-coefficient finite-volume Poisson systems,
    side uniform in [side_lo, side_hi], log kappa ~ N(0, sigma^2) per cell,
    px x py boxes with px, py uniform in {2, 3, 4} (4 to 16 subdomains), 1 to 8
    right-hand sides uniform in [-1, 1].  Stream order per system: side, kappa,
    boxes, right-hand-side count, right-hand sides."""
    rng = np.random.default_rng(seed)
    As, parts, Ps, bs, sides = [], [], [], [], []
    for _ in range(nsys):
        n = int(rng.integers(side_lo, side_hi + 1))
        kap = np.exp(sigma * rng.standard_normal((n, n)))
        px, py = (int(v) for v in rng.integers(2, 5, size=2))
        k = int(rng.integers(1, 9))
        b = rng.uniform(-1.0, 1.0, size=(k, n * n))
        As.append(fv2d_5pt(n, n, kap))
        parts.append(box_partition_2d(n, n, px, py))
        Ps.append(px * py)
        bs.append(b)
        sides.append(n)
    return BatchProblem("fv2d_5pt_batch%d_side%d-%d" % (nsys, side_lo, side_hi), As, parts, Ps, bs,
                        {"sides": sides, "sigma": sigma})


def fe2d_p1_jittered(N: int, rng: np.random.Generator, jitter: float = 0.3):
    """Assembled P1 finite-element Laplacian of ``fe2d_p1_elements`` (same
    random stream): returns (CSR, coords [n,2], n_inverted_triangles)."""
    ids, Ke, coords, n_inv = fe2d_p1_elements(N, rng, jitter)
    return fe_assemble(N * N, ids, Ke), coords, n_inv


def fe_assemble(n: int, ids: np.ndarray, Ke: np.ndarray) -> CSR:
    """Global matrix sum_e K_e over the free nodes (ids -1 dropped), made
    exactly symmetric from its upper triangle."""
    import scipy.sparse as sp

    nv = ids.shape[1]
    I = np.repeat(ids, nv, axis=1).reshape(-1, nv, nv)
    J = np.tile(ids, (1, nv)).reshape(-1, nv, nv)
    keep = (I >= 0) & (J >= 0)
    A = sp.coo_matrix((Ke[keep], (I[keep], J[keep])), shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    U = sp.triu(A, 0, format="csr")
    S = (U + sp.triu(U, 1, format="csr").T).tocsr()
    S.sort_indices()
    return CSR(n, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))


def fe2d_p1_elements(N: int, rng: np.random.Generator, jitter: float = 0.3):
    """P1 finite-element Laplacian on a jittered N x N free-node mesh, by elements.

    The N x N free nodes sit inside a ring of fixed (unjittered) Dirichlet
    nodes, (N+2)^2 nodes in all, spacing h = 1/(N+1).  Every free node is moved
    by independent uniform[-jitter*h, jitter*h] offsets in x and y (drawn first),
    then every one of the (N+1)^2 squares is split into two triangles along a
    diagonal chosen by a fair seeded coin (drawn second).  The element matrix
    uses |area|, so an inverted triangle still gives a symmetric positive
    semi-definite contribution.  Free node (ix, iy), 1 <= ix, iy <= N, has id
    (ix-1) + N*(iy-1).

    Returns (ids [ne, 3] free node of each vertex or -1 for a Dirichlet
    node, Ke [ne, 3, 3] element matrices, coords [n, 2] of the free nodes,
    n_inverted_triangles).
    """
    h = 1.0 / (N + 1)
    M = N + 2
    gx, gy = np.meshgrid(np.arange(M) * h, np.arange(M) * h, indexing="xy")
    X = gx.copy()
    Y = gy.copy()
    d = rng.uniform(-jitter * h, jitter * h, size=(2, N, N))
    X[1:-1, 1:-1] += d[0]
    Y[1:-1, 1:-1] += d[1]
    flip = rng.integers(0, 2, size=(N + 1, N + 1))

    # node numbering over the full (N+2)^2 grid; free ids or -1
    fid = -np.ones((M, M), dtype=np.int64)
    fid[1:-1, 1:-1] = np.arange(N * N).reshape(N, N)
    jj, ii = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")  # jj = row (y), ii = col (x)
    v00 = (jj, ii)
    v10 = (jj, ii + 1)
    v01 = (jj + 1, ii)
    v11 = (jj + 1, ii + 1)
    f = flip.astype(bool)
    # f == 0 (diagonal 00-11): triangles (00, 10, 11) and (00, 11, 01)
    # f == 1 (diagonal 10-01): triangles (00, 10, 01) and (10, 11, 01)
    # (all counter-clockwise before jitter)
    t1 = (v00, v10, tuple(np.where(f, v01[q], v11[q]) for q in range(2)))
    t2 = (tuple(np.where(f, v10[q], v00[q]) for q in range(2)), v11, v01)
    tri_r = []
    tri_c = []
    for t in (t1, t2):
        tri_r.append(np.stack([t[0][0].ravel(), t[1][0].ravel(), t[2][0].ravel()], axis=1))
        tri_c.append(np.stack([t[0][1].ravel(), t[1][1].ravel(), t[2][1].ravel()], axis=1))
    tr = np.concatenate(tri_r)
    tc = np.concatenate(tri_c)
    x = X[tr, tc]
    y = Y[tr, tc]
    ids = fid[tr, tc]
    bvec = np.stack([y[:, 1] - y[:, 2], y[:, 2] - y[:, 0], y[:, 0] - y[:, 1]], axis=1)
    cvec = np.stack([x[:, 2] - x[:, 1], x[:, 0] - x[:, 2], x[:, 1] - x[:, 0]], axis=1)
    det = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    n_inv = int(np.count_nonzero(det <= 0.0))
    scale = 1.0 / (2.0 * np.abs(det))
    Ke = (bvec[:, :, None] * bvec[:, None, :] + cvec[:, :, None] * cvec[:, None, :]) * scale[:, None, None]
    coords = np.stack([X[1:-1, 1:-1].ravel(), Y[1:-1, 1:-1].ravel()], axis=1)
    return ids.astype(np.int32), Ke, coords, n_inv


def random_spd(n: int, avg_deg: float, rng: np.random.Generator, shift: float = 0.5) -> CSR:
    """Random sparse SPD matrix: a weighted graph Laplacian plus a positive shift.

    Edges (i < j) are drawn uniformly, weights uniform[0.1, 1]; A = D - W + s*I
    with D the weighted degrees, so A is strictly diagonally dominant and SPD.
    """
    m = int(round(avg_deg * n / 2))
    i = rng.integers(0, n, size=m)
    j = rng.integers(0, n, size=m)
    keep = i != j
    i, j = np.minimum(i[keep], j[keep]), np.maximum(i[keep], j[keep])
    key = np.unique(i.astype(np.int64) * n + j)
    i = (key // n).astype(np.int64)
    j = (key % n).astype(np.int64)
    w = rng.uniform(0.1, 1.0, size=i.size)
    import scipy.sparse as sp

    W = sp.coo_matrix((w, (i, j)), shape=(n, n)).tocsr()
    W = (W + W.T).tocsr()
    deg = np.asarray(W.sum(axis=1)).ravel()
    A = (sp.diags(deg + shift) - W).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    U = sp.triu(A, 0, format="csr")
    S = (U + sp.triu(U, 1, format="csr").T).tocsr()
    S.sort_indices()
    return CSR(n, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))


def pair_blocks(blocks, nrep: int) -> CSR:
    """Block-diagonal SPD matrix of 2x2 blocks [[a, b], [b, a]] on the node
    pairs (2j, 2j+1), block j taking ``blocks[j % len(blocks)]``, repeated
    until there are len(blocks) * nrep blocks.  Its eigenvalues are the
    a - b and a + b of the blocks, so the number of distinct eigenvalues is
    known by construction, and a partition that splits pairs gives interface
    nodes."""
    nb = len(blocks) * nrep
    ab = np.array([blocks[j % len(blocks)] for j in range(nb)], dtype=np.float64)
    n = 2 * nb
    rowptr = np.arange(0, 2 * n + 1, 2, dtype=np.int32)
    first = 2 * np.arange(nb)
    colidx = np.stack([first, first + 1, first, first + 1], axis=1).ravel().astype(np.int32)
    val = np.stack([ab[:, 0], ab[:, 1], ab[:, 1], ab[:, 0]], axis=1).ravel()
    return CSR(n, rowptr, colidx, val)


def box_partition_2d(nx: int, ny: int, px: int, py: int) -> np.ndarray:
    """part = bx + px*by with bx = floor(ix*px/nx), by = floor(iy*py/ny)."""
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    bx = (ix * px) // nx
    by = (iy * py) // ny
    return (bx + px * by).ravel().astype(np.int32)


def box_partition_3d(nx: int, ny: int, nz: int, px: int, py: int, pz: int) -> np.ndarray:
    """part = bx + px*(by + py*bz), each b = floor(i*p/n) along its axis."""
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    bx = (ix * px) // nx
    by = (iy * py) // ny
    bz = (iz * pz) // nz
    return (bx + px * (by + py * bz)).ravel().astype(np.int32)


def fe_element_problem(N: int, levels: int, seed: int = CONFIG_SEED_BASE + 3):
    """Workload 3's mesh by elements: the jittered P1 mesh of side N, its
    element matrices, and an element partition by recursive coordinate
    bisection of the element centroids (free vertices only; an element with
    no free vertex goes to subdomain 0).  Stream order: jitter, diagonals,
    x*, RCB ratios.  Returns (ids, Ke, epart, P, A, xstar, b)."""
    rng = np.random.default_rng(seed)
    ids, Ke, coords, _ = fe2d_p1_elements(N, rng)
    n = N * N
    A = fe_assemble(n, ids, Ke)
    xs = rng.uniform(-1.0, 1.0, size=n)
    b = A.to_scipy() @ xs
    free = ids >= 0
    cnt = np.maximum(free.sum(axis=1), 1)
    cx = np.where(free, coords[np.maximum(ids, 0), 0], 0.0).sum(axis=1) / cnt
    cy = np.where(free, coords[np.maximum(ids, 0), 1], 0.0).sum(axis=1) / cnt
    epart = rcb_partition(np.stack([cx, cy], axis=1), levels, rng)
    epart[free.sum(axis=1) == 0] = 0
    return ids, Ke, epart, 2**levels, A, xs, b


def rcb_partition(coords: np.ndarray, levels: int, rng: np.random.Generator, lo=0.3, hi=0.7) -> np.ndarray:
    """Recursive coordinate bisection with random split ratios.

    Level by level, every current node set (in order of its part id) is cut
    along its longer coordinate extent: nodes are ordered by (coordinate,
    global id) and the first floor(r*size) go to child 2*id, the rest to
    2*id+1, with r ~ uniform[lo, hi] drawn per cut.  ``levels`` cuts give
    2**levels parts.
    """
    n = coords.shape[0]
    part = np.zeros(n, dtype=np.int64)
    gid = np.arange(n)
    for _ in range(levels):
        new = np.empty_like(part)
        nparts = int(part.max()) + 1 if n else 0
        order_all = np.argsort(part, kind="stable")
        sp = np.searchsorted(part[order_all], np.arange(nparts + 1))
        for p in range(nparts):
            idx = order_all[sp[p] : sp[p + 1]]
            r = rng.uniform(lo, hi)
            c = coords[idx]
            ext = c.max(axis=0) - c.min(axis=0) if idx.size else np.zeros(2)
            ax = int(np.argmax(ext))
            o = np.lexsort((gid[idx], c[:, ax]))
            cut = int(np.floor(r * idx.size))
            sel = idx[o]
            new[sel[:cut]] = 2 * p
            new[sel[cut:]] = 2 * p + 1
        part = new
    return part.astype(np.int32)


def manufactured_rhs(A: CSR, rng: np.random.Generator, k: int = 1):
    """x* ~ uniform[-1, 1]^(n x k); b = A x* (scipy sparse product)."""
    xs = rng.uniform(-1.0, 1.0, size=(A.n, k))
    b = A.to_scipy() @ xs
    return xs, np.ascontiguousarray(b)


def config_problem(idx: int, scale: int | None = None) -> Problem:
    """The synthetic workloads, by number.

    1: 2D 5-point Poisson, 64x64 interior grid, 2x2 box split.
    2: 3D 7-point FV, kappa = exp(g), g ~ N(0,1) per cell, 128^3, 4x4x4 boxes.
    3: 2D P1 FE on a jittered 1024x1024 free-node mesh, 256-part RCB.
    5: 3D 7-point FV, 96^3, log kappa ~ N(0,1), 3x3x3 boxes, 16 right-hand sides.

    ``scale`` overrides the grid side (same recipe, smaller) for tests.
    Seed = 13162 + idx; stream order: kappa, x*, jitter, diagonals, RCB ratios.
    """
    rng = np.random.default_rng(CONFIG_SEED_BASE + idx)
    if idx == 1:
        s = scale or 64
        A = poisson2d_5pt(s, s)
        part = box_partition_2d(s, s, 2, 2)
        xs, b = manufactured_rhs(A, rng)
        return Problem("poisson2d_5pt_%dx%d_2x2" % (s, s), A, part, 4, xs, b, {"grid": (s, s)})
    if idx in (2, 5):
        s = scale or (128 if idx == 2 else 96)
        pd = 4 if idx == 2 else 3
        g = rng.standard_normal(size=(s, s, s))
        kap = np.exp(g)
        A = fv3d_7pt(s, s, s, kap)
        part = box_partition_3d(s, s, s, pd, pd, pd)
        k = 1 if idx == 2 else 16
        xs, b = manufactured_rhs(A, rng, k)
        return Problem(
            "fv3d_7pt_%d^3_%dx%dx%d" % (s, pd, pd, pd), A, part, pd**3, xs, b, {"grid": (s, s, s), "log_kappa": g}
        )
    if idx == 3:
        s = scale or 1024
        n = s * s
        xs = rng.uniform(-1.0, 1.0, size=(n, 1))
        A, coords, n_inv = fe2d_p1_jittered(s, rng)
        levels = 8 if scale is None else max(2, min(8, int(np.log2(max(4, n // 256)))))
        part = rcb_partition(coords, levels, rng)
        b = np.ascontiguousarray(A.to_scipy() @ xs)
        return Problem(
            "fe2d_p1_jittered_%d^2_rcb%d" % (s, 2**levels),
            A,
            part,
            2**levels,
            xs,
            b,
            {"grid": (s, s), "inverted_triangles": n_inv, "coords": coords},
        )
    raise ValueError("unknown workload %r" % idx)
