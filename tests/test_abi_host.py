"""CPU-side checks of the C ABI (no GPU): the library loads, exports every
entry point include/ssg.h declares, and its host partitioner produces maps
bit-identical to the oracle's (Section 2.4 sub-structures, Section 3.4.2
interface lists).  Device entry points are not called here except on a
host-only system, where they must refuse with SSG_E_INVALID."""

import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from synth import CSR, config_problem, poisson2d_5pt, random_spd
from paper_2108_13162_gb300 import build as ssg_build
from paper_2108_13162_gb300 import ssg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    ssg_build.build()


def _declared():
    text = open(os.path.join(ROOT, "include", "ssg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ssg_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol():
    names = _declared()
    assert len(names) >= 14
    assert set(names) == set(ssg.EXPORTS)
    L = C.CDLL(ssg.library_path())
    for n in names:
        assert hasattr(L, n), "missing export %s" % n


def _cases():
    rng = np.random.default_rng(21)
    out = []
    p = config_problem(1)
    out.append(("config1", p.A, p.part, p.P))
    p = config_problem(2, scale=24)
    out.append(("fv3d_24", p.A, p.part, p.P))
    p = config_problem(3, scale=40)
    out.append(("fe_40", p.A, p.part, p.P))
    A = random_spd(300, 7.0, rng)
    out.append(("rand300", A, rng.integers(0, 9, 300).astype(np.int32), 9))
    A = poisson2d_5pt(9, 7)
    out.append(("p2d_P1", A, np.zeros(A.n, np.int32), 1))
    return out


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_host_maps_bit_exact_vs_oracle(case):
    _, A, part, P = case
    sys_ = ssg.ssg_partition(None, A.n, A.rowptr, A.colidx, A.val, part, P)
    try:
        got = ssg.ssg_copy_maps(sys_)
        sz = ssg.ssg_get_sizes(sys_)
    finally:
        ssg.ssg_system_destroy(sys_)
    ref = oracle.Partition(A, part, P).maps
    assert (sz.n, sz.P, sz.nnz, sz.nloc, sz.ngamma, sz.ncopies) == (
        ref.n, ref.P, ref.nnz, ref.nloc, ref.ngamma, ref.ncopies)
    assert sz.max_mult == int(ref.mult.max())
    for k in ("off", "nint", "l2g", "mult", "lrowptr", "lcol", "gamma", "iptr", "icopy", "own"):
        assert np.array_equal(got[k], getattr(ref, k)), k
    assert np.array_equal(got["lval"].view(np.int64), ref.lval.view(np.int64))


def _random_case(seed):
    """A small random SPD system and partition: random, contiguous, with
    more subdomains than nodes, or with every node in the top subdomain."""
    import scipy.sparse as sp

    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 120))
    if seed % 5 == 4:
        # a diagonal-only (isolated) node block next to a coupled one
        A = random_spd(max(n - 3, 1), float(rng.uniform(1.0, 6.0)), rng).to_scipy()
        A = sp.block_diag([A, sp.diags(rng.uniform(1.0, 2.0, 3))]).tocsr()
        A.sort_indices()
        A = CSR(A.shape[0], A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64))
    else:
        A = random_spd(n, float(rng.uniform(1.0, 8.0)), rng)
    n = A.n
    kind = seed % 4
    P = int(rng.integers(1, 12))
    if kind == 0:
        part = rng.integers(0, P, n)
    elif kind == 1:
        part = np.arange(n) * P // n
    elif kind == 2:
        P = n + int(rng.integers(1, 5))  # more subdomains than nodes: some empty
        part = rng.integers(0, P, n)
    else:
        part = np.full(n, P - 1)  # only the top id used
    return A, part.astype(np.int32), P


@pytest.mark.parametrize("seed", range(40))
def test_host_maps_bit_exact_random(seed):
    A, part, P = _random_case(seed)
    sys_ = ssg.ssg_partition(None, A.n, A.rowptr, A.colidx, A.val, part, P)
    try:
        got = ssg.ssg_copy_maps(sys_)
        sz = ssg.ssg_get_sizes(sys_)
    finally:
        ssg.ssg_system_destroy(sys_)
    ref = oracle.Partition(A, part, P).maps
    assert (sz.n, sz.P, sz.nnz, sz.nloc, sz.ngamma, sz.ncopies) == (
        ref.n, ref.P, ref.nnz, ref.nloc, ref.ngamma, ref.ncopies)
    for k in ("off", "nint", "l2g", "mult", "lrowptr", "lcol", "gamma", "iptr", "icopy", "own"):
        assert np.array_equal(got[k], getattr(ref, k)), k
    assert np.array_equal(got["lval"].view(np.int64), ref.lval.view(np.int64))


def test_full_size_maps_bit_exact():
    """The 128^3 / 4x4x4 workload: counts and maps identical to the oracle's."""
    p = config_problem(2)
    sys_ = ssg.ssg_partition(None, p.A.n, p.A.rowptr, p.A.colidx, p.A.val, p.part, p.P)
    try:
        got = ssg.ssg_copy_maps(sys_)
    finally:
        ssg.ssg_system_destroy(sys_)
    ref = oracle.Partition(p.A, p.part, p.P).maps
    assert ref.nloc == 2244608 and ref.ngamma == 144027 and ref.ncopies == 291483
    for k in ("off", "nint", "l2g", "lrowptr", "lcol", "iptr", "icopy", "own"):
        assert np.array_equal(got[k], getattr(ref, k)), k


def test_invalid_inputs():
    A = poisson2d_5pt(6, 6)
    part = np.zeros(A.n, np.int32)
    bad = part.copy()
    bad[5] = 3
    with pytest.raises(ssg.SSGError) as e:
        ssg.ssg_partition(None, A.n, A.rowptr, A.colidx, A.val, bad, 2)
    assert e.value.status == ssg.SSG_E_INVALID and "part id" in str(e.value)
    v = A.val.copy()
    v[1] = 7.0
    with pytest.raises(ssg.SSGError) as e:
        ssg.ssg_partition(None, A.n, A.rowptr, A.colidx, v, part, 1)
    assert "symmetric" in str(e.value)
    c = A.colidx.copy()
    c[0], c[1] = c[1], c[0]
    with pytest.raises(ssg.SSGError):
        ssg.ssg_partition(None, A.n, A.rowptr, c, A.val, part, 1)
    with pytest.raises(ssg.SSGError):
        ssg.ssg_partition(None, A.n, A.rowptr, A.colidx, A.val, part, 0)
    # the non-symmetric worked example of Section 1.2
    ex = CSR(5, np.array([0, 2, 4, 6, 9, 11], np.int32), np.array([0, 1, 1, 2, 0, 2, 1, 3, 4, 2, 4], np.int32),
             np.array([-5, 14, 8, 1, 2, 10, 4, 2, 9, 15, 7], np.float64))
    with pytest.raises(ssg.SSGError):
        ssg.ssg_partition(None, 5, ex.rowptr, ex.colidx, ex.val, np.zeros(5, np.int32), 1)


def test_host_only_system_refuses_device_calls():
    A = poisson2d_5pt(4, 4)
    sys_ = ssg.ssg_partition(None, A.n, A.rowptr, A.colidx, A.val, np.zeros(A.n, np.int32), 1)
    try:
        L = ssg.lib()
        assert L.ssg_spmv_assembled(sys_, None, None, None) == ssg.SSG_E_INVALID
        assert L.ssg_solve(sys_, 1, None, None, 0, 1e-8, 10, 0, None) == ssg.SSG_E_INVALID
        assert L.ssg_wdot(sys_, None, None, None) == ssg.SSG_E_INVALID
        assert "host maps only" in ssg.last_error()
    finally:
        ssg.ssg_system_destroy(sys_)


def test_layout_reports_refuse_null_arguments():
    """The layout reports take a system and a host buffer; a null either is
    SSG_E_INVALID with a message, and nothing is written."""
    import ctypes as C

    L = ssg.lib()
    buf = (C.c_int64 * 4)()
    for fn in (L.ssg_get_layout, L.ssg_get_iface_layout):
        f = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p)(C.cast(fn, C.c_void_p).value)
        assert f(None, C.addressof(buf)) == ssg.SSG_E_INVALID
        assert "null" in ssg.last_error()
    A = poisson2d_5pt(4, 4)
    sys_ = ssg.ssg_partition(None, A.n, A.rowptr, A.colidx, A.val, (np.arange(A.n) % 2).astype(np.int32), 2)
    try:
        f = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p)(C.cast(L.ssg_get_iface_layout, C.c_void_p).value)
        assert f(sys_, None) == ssg.SSG_E_INVALID
    finally:
        ssg.ssg_system_destroy(sys_)


def test_error_strings():
    for code in range(7):
        assert ssg.ssg_error_string(code)
    assert "breakdown" in ssg.ssg_error_string(ssg.SSG_E_BREAKDOWN).lower()


@pytest.mark.parametrize("N,levels", [(14, 3), (33, 4), (8, 0)])
def test_element_maps_bit_exact_vs_oracle(N, levels):
    """Sub-structures from finite elements (ssg_partition_fe vs
    or_partition_fe): every map and every summed local value identical."""
    from synth import fe_element_problem

    ids, Ke, epart, P, A, xs, b = fe_element_problem(N, levels)
    sys_ = ssg.ssg_partition_fe(None, A.n, ids, Ke, epart, P)
    try:
        got = ssg.ssg_copy_maps(sys_)
        sz = ssg.ssg_get_sizes(sys_)
    finally:
        ssg.ssg_system_destroy(sys_)
    ref = oracle.Partition.from_elements(A.n, ids, Ke, epart, P).maps
    assert (sz.n, sz.P, sz.nnz, sz.nloc, sz.ngamma, sz.ncopies) == (
        ref.n, ref.P, ref.nnz, ref.nloc, ref.ngamma, ref.ncopies)
    for k in ("off", "nint", "l2g", "mult", "lrowptr", "lcol", "gamma", "iptr", "icopy", "own"):
        assert np.array_equal(got[k], getattr(ref, k)), k
    assert np.array_equal(got["lval"].view(np.int64), ref.lval.view(np.int64))


def test_element_input_rejected():
    from synth import fe_element_problem

    ids, Ke, epart, P, A, xs, b = fe_element_problem(6, 1)
    bad = epart.copy()
    bad[1] = -1
    with pytest.raises(ssg.SSGError):
        ssg.ssg_partition_fe(None, A.n, ids, Ke, bad, P)
    K2 = Ke.copy()
    K2[0, 1, 2] += 1.0
    with pytest.raises(ssg.SSGError):
        ssg.ssg_partition_fe(None, A.n, ids, K2, epart, P)
    ids2 = ids.copy()
    ids2[ids2 == 3] = 4
    with pytest.raises(ssg.SSGError):
        ssg.ssg_partition_fe(None, A.n, ids2, Ke, epart, P)


def test_noalloc_dot_arguments_refused_before_launch(monkeypatch):
    """ssg_wdot_noalloc cannot see buffer lengths or devices, so the binding
    refuses mismatched lengths, non-contiguous buffers, an empty output, wrong
    dtypes and non-CUDA tensors itself; the library is never reached."""
    import torch

    def no_library():
        raise AssertionError("the library was called with arguments the binding must refuse")

    monkeypatch.setattr(ssg, "lib", no_library)
    u = torch.zeros(100, dtype=torch.float64)
    v = torch.zeros(100, dtype=torch.float64)
    m = torch.ones(100, dtype=torch.uint8)
    out = torch.zeros(1, dtype=torch.float64)
    bad = [
        ((u, v[:99], m, out), ValueError),                       # v shorter than u
        ((u, v, m[:50], out), ValueError),                       # mult shorter than u
        ((u, v, m, torch.zeros(0, dtype=torch.float64)), ValueError),  # no room for the result
        ((u, torch.zeros(200, dtype=torch.float64)[::2], m, out), ValueError),  # strided v
        ((u, v, m.to(torch.int32), out), TypeError),             # mult not bytes
        ((u.float(), v, m, out), TypeError),                     # u not float64
        ((u, v, m, out), TypeError),                             # consistent, but host tensors
    ]
    for args, exc in bad:
        with pytest.raises(exc):
            ssg.ssg_wdot_noalloc(*args)


def test_slice_layout_rule_from_row_lengths():
    """The interior slice layout chosen from the row-length histogram (host
    only): the jittered P1 mesh (rows of 3-9 entries) gets its rows sorted
    by length in windows, which cuts the padding of 32-row slices from about
    27 % to a few % (2 % on the 1024^2 mesh); the finite-volume and Poisson grids (rows of equal
    length but at the boundary) stay unsorted."""
    p = config_problem(3, scale=96)
    S = ssg.System(None, p.A, p.part, p.P)
    lay = S.layout()
    assert lay["sorted_subdomains"] == p.P and lay["max_window"] in (128, 256, 512)
    # (at this size a subdomain holds about 290 rows, and the part-empty
    # last slice of each window weighs; the 1024^2 mesh gets about 1.02)
    assert lay["slice_entries"] == _interior_nnz(p) and lay["padding_ratio"] < 1.10
    S.close()
    for q in (config_problem(2, scale=24), config_problem(1)):
        S = ssg.System(None, q.A, q.part, q.P)
        lay = S.layout()
        assert lay["sorted_subdomains"] == 0 and lay["max_window"] == 1
        assert lay["slice_entries"] == _interior_nnz(q) and lay["padding_ratio"] < 1.10
        S.close()


def _iface_slots(m):
    """Entries the two interface layouts store, recomputed from the oracle's
    maps: slices of whole nodes in ascending node order (up to 32 copy rows,
    each padded to the slice's longest) and groups of up to 32 nodes of one
    multiplicity (in windows of 512 nodes ordered by decreasing copy-row
    lengths, rank by rank; each rank padded to the group's longest).  Nodes
    with a copy row longer than 64, or more copies than a layout takes (32,
    8), are left to items of their own."""
    clen = np.diff(m.lrowptr)[m.icopy]
    mult = np.diff(m.iptr)
    long_row = np.array([clen[m.iptr[g]:m.iptr[g + 1]].max() > 64 for g in range(m.ngamma)], bool)
    slots, g = 0, 0
    while g < m.ngamma:
        if mult[g] > 32 or long_row[g]:
            g += 1
            continue
        c0, g1, w = m.iptr[g], g, 0
        while g1 < m.ngamma and not (mult[g1] > 32 or long_row[g1]) and m.iptr[g1 + 1] - c0 <= 32:
            w = max(w, int(clen[m.iptr[g1]:m.iptr[g1 + 1]].max()))
            g1 += 1
        slots += 32 * w
        g = g1
    gslots = 0
    for mm in range(1, 9):
        nodes = [g for g in range(m.ngamma) if mult[g] == mm and not long_row[g]]
        for w0 in range(0, len(nodes), 512):
            win = sorted(nodes[w0:w0 + 512], key=lambda g: tuple(-int(clen[m.iptr[g] + r]) for r in range(mm)))
            for i in range(0, len(win), 32):
                grp = win[i:i + 32]
                gslots += sum(32 * max(int(clen[m.iptr[g] + r]) for g in grp) for r in range(mm))
    return slots, gslots


def test_iface_layout_rule():
    """The interface layout (host only): the entries both layouts store match
    a recomputation from the oracle's maps, and the single-vector product
    takes the groups exactly when they store at least 4 % of all its sliced
    entries fewer: on the finite-volume boxes (a node's copy in the lower
    subdomain holds one entry, the owner's six) but not on the Poisson square
    or the P1 mesh."""
    for q, want in ((config_problem(2, scale=24), True), (config_problem(1), False),
                    (config_problem(3, scale=96), None)):
        S = ssg.System(None, q.A, q.part, q.P)
        lay, il = S.layout(), S.iface_layout()
        slots, gslots = _iface_slots(oracle.Partition(q.A, q.part, q.P).maps)
        assert (il["iface_slots"], il["group_slots"]) == (slots, gslots)
        rule = slots > gslots and slots - gslots >= 0.04 * (lay["slice_slots"] + slots)
        assert il["groups"] == rule
        if want is not None:
            assert il["groups"] == want
        S.close()


@pytest.mark.parametrize("seed", range(0, 40, 3))
def test_iface_layout_random_systems(seed):
    """The interface layout's entry counts and choice on the seeded random
    systems (random degrees: multiplicities up to the subdomain count,
    nodes with more copies than a group takes, empty subdomains), against the
    recomputation from the oracle's maps."""
    A, part, P = _random_case(seed)
    S = ssg.System(None, A, part, P)
    lay, il = S.layout(), S.iface_layout()
    slots, gslots = _iface_slots(oracle.Partition(A, part, P).maps)
    assert (il["iface_slots"], il["group_slots"]) == (slots, gslots)
    assert il["groups"] == (slots > gslots and slots - gslots >= 0.04 * (lay["slice_slots"] + slots))
    S.close()


def _interior_nnz(p):
    """Stored entries of the interior (multiplicity 1) rows of the local
    matrices, from the oracle's maps."""
    m = oracle.Partition(p.A, p.part, p.P).maps
    lens = np.diff(m.lrowptr)
    interior = np.concatenate([np.arange(m.off[s], m.off[s] + m.nint[s]) for s in range(m.P)])
    return int(lens[interior].sum())
