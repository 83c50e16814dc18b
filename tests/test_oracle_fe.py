"""Pins for the oracle's sub-structures built from finite elements
(or_partition_fe, Section 2.4: each subdomain's local matrix is the sum of
its own element matrices).

  * the local matrices add up to the globally assembled matrix (Eq.
    interface_summation) within the rounding of the differently grouped sums;
  * multiplicities equal the number of distinct subdomains among a node's
    elements (counted here from the element lists);
  * every local matrix is symmetric positive semi-definite (a Neumann
    matrix), and its rows over elements without Dirichlet vertices sum to
    zero (P1 element matrices annihilate constants);
  * the sub-structured product equals the global product, and sub-structured
    CG and the diagonal-preconditioned CG recover the manufactured solution;
  * planted mistakes in or_partition_fe each break a pin.
"""

import os

import numpy as np
import pytest

import oracle
from synth import fe_element_problem

U = 2.0**-53


def _setup(N=14, levels=3):
    return fe_element_problem(N, levels)


def _local_dense(m, s):
    o0, o1 = m.off[s], m.off[s + 1]
    ns = o1 - o0
    D = np.zeros((ns, ns))
    for r in range(ns):
        for k in range(m.lrowptr[o0 + r], m.lrowptr[o0 + r + 1]):
            D[r, m.lcol[k]] += m.lval[k]
    return D


def pin_fe(mod_lib=None):
    ids, Ke, epart, P, A, xs, b = _setup()
    Pt = oracle.Partition.from_elements(A.n, ids, Ke, epart, P)
    m = Pt.maps
    # reassembly within rounding
    sub = np.searchsorted(m.off, np.arange(m.nloc), side="right") - 1
    rows = np.repeat(m.l2g, np.diff(m.lrowptr))
    cols = m.l2g[m.off[np.repeat(sub, np.diff(m.lrowptr))] + m.lcol]
    R = np.zeros((A.n, A.n))
    np.add.at(R, (rows, cols), m.lval)
    D = A.to_scipy().toarray()
    absK = np.zeros((A.n, A.n))
    cnt = np.zeros((A.n, A.n))
    for e in range(ids.shape[0]):
        for a in range(3):
            for c in range(3):
                if ids[e, a] >= 0 and ids[e, c] >= 0:
                    absK[ids[e, a], ids[e, c]] += abs(Ke[e, a, c])
                    cnt[ids[e, a], ids[e, c]] += 1
    assert np.all(np.abs(R - D) <= 2 * cnt * U * absK + 1e-300)
    # multiplicities from the element lists
    mult = np.zeros(A.n, np.int64)
    for i in range(A.n):
        mult[i] = len(set(epart[np.any(ids == i, axis=1)]))
    assert np.array_equal(m.mult, mult)
    # Neumann local matrices
    for s in range(P):
        L = _local_dense(m, s)
        if L.size == 0:
            continue
        assert np.allclose(L, L.T, rtol=0, atol=0)
        ev = np.linalg.eigvalsh(L)
        assert ev[0] >= -1e-12 * max(1.0, ev[-1])
        g = m.l2g[m.off[s]:m.off[s + 1]]
        mine = epart == s
        touched_bnd = set(ids[mine & np.any(ids < 0, axis=1)].ravel()) - {-1}
        for r, gi in enumerate(g):
            if gi in touched_bnd:
                continue
            assert abs(L[r].sum()) <= 64 * U * np.abs(L[r]).sum()
    # product and solves
    x = np.random.default_rng(2).uniform(-1, 1, A.n)
    y = Pt.spmv(Pt.scatter(x))
    absAx = abs(A.to_scipy()) @ np.abs(x)
    assert np.all(np.abs(y[m.own] - A.to_scipy() @ x) <= 64 * U * absAx)
    r = Pt.cg(b, 1e-10, 10 * A.n)
    assert r.status == oracle.OK
    kap = oracle.cond_from_lanczos(r.alpha, r.beta)
    assert np.linalg.norm(r.x - xs) / np.linalg.norm(xs) <= 2 * kap * 1e-10
    rp = Pt.pcg(b, 1e-10, 10 * A.n)
    assert rp.status == oracle.OK
    assert np.linalg.norm(rp.x - xs) / np.linalg.norm(xs) <= 2 * kap * 1e-10


def test_fe_pins():
    pin_fe()


def test_fe_rejects_bad_input():
    ids, Ke, epart, P, A, xs, b = _setup(6, 1)
    bad = epart.copy()
    bad[0] = P
    with pytest.raises(ValueError):
        oracle.Partition.from_elements(A.n, ids, Ke, bad, P)
    K2 = Ke.copy()
    K2[3, 0, 1] += 1.0
    with pytest.raises(ValueError):
        oracle.Partition.from_elements(A.n, ids, K2, epart, P)
    ids2 = ids.copy()
    ids2[ids2 == 5] = 6  # node 5 in no element
    with pytest.raises(ValueError):
        oracle.Partition.from_elements(A.n, ids2, Ke, epart, P)


FE_MUTATIONS = {
    # a local entry keeps only its last element contribution
    "no_element_sum": ("while (u < nent && ent[u].s == ent[t].s && ent[u].r == ent[t].r && ent[u].c == ent[t].c) v = v + ent[u++].v;",
                       "while (u < nent && ent[u].s == ent[t].s && ent[u].r == ent[t].r && ent[u].c == ent[t].c) v = ent[u++].v;"),
    # eliminated (Dirichlet) vertices not dropped from the element rows
    "keep_dirichlet_columns": ("                const int32_t j = elem[(int64_t)e * nv + b];\n                if (j < 0) continue;",
                               "                int32_t j = elem[(int64_t)e * nv + b];\n                if (j < 0) j = 0;"),
    # membership from the first element of a node only
    "single_membership": ("            if (t > 0 && pairs[t].node == pairs[t - 1].node && pairs[t].s == pairs[t - 1].s) continue;",
                          "            if (t > 0 && pairs[t].node == pairs[t - 1].node) continue;"),
}


@pytest.mark.parametrize("name", sorted(FE_MUTATIONS))
def test_fe_planted_mistake_is_caught(name):
    old, new = FE_MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, name
    path = oracle.compile_variant(src.replace(old, new), name)
    caught = False
    try:
        with oracle.use_library(path):
            try:
                pin_fe()
            except (AssertionError, ValueError):
                caught = True
    finally:
        os.remove(path)
    assert caught, "planted mistake %s slipped through" % name
