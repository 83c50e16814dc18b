"""Pins of the oracle's two weightings of the weighted dots (Section 3.4.2
asks for a weighted combination of the subdomains' sums without giving the
weights): w = 1/m on every copy (the default) and the owner mask, w = 1 on a
node's owner copy (its copy in subdomain part(i)) and 0 on its other copies.

What fixes them, independently of the oracle's code:
  - either set sums to 1 over the copies of each node, so the dot of
    consistent (scattered) vectors is the global dot u . v to rounding
    (<= 1e-14 relative, the tolerance of the sub-structuring reading);
  - the owner-mask dot of arbitrary local vectors is the plain sum of
    u_k v_k over the owner entries k = own[i], in concatenated order
    (brute force from the maps, bit for bit);
  - switching back restores the 1/m dot bit for bit;
  - with the owner mask, sub-structured CG still solves tiny SPD systems to
    the dense Cholesky solution (1e-10 at rtol 1e-12), converges for A = I in
    one iteration and for the 1D Laplacian within n iterations.
Planted mistakes in the owner mask (every copy weighted 1, the first copy
instead of the owner) must each fail one of them.
"""

import os

import numpy as np
import pytest

import oracle
from synth import CSR, laplace1d
from tests.test_oracle_pins import SMALL, _dense


def pin_weights_sum_to_one(A, part, P, seed=3):
    """Dots of scattered (consistent) vectors equal the global dot, both weightings."""
    rng = np.random.default_rng(seed)
    ref = oracle.Partition(A, part, P)
    for _ in range(3):
        u = rng.uniform(-1, 1, A.n)
        v = rng.uniform(-1, 1, A.n)
        g = float(np.dot(u, v))
        scale = float(np.dot(np.abs(u), np.abs(v)))
        ul, vl = ref.scatter(u), ref.scatter(v)
        for mode in (oracle.WEIGHT_OWNER, oracle.WEIGHT_INV_MULT):
            ref.set_weights(mode)
            assert abs(ref.wdot(ul, vl) - g) <= 1e-14 * scale, mode


def pin_owner_brute_force(A, part, P, seed=4):
    """Owner-mask dot of inconsistent local vectors = the sum over owner entries."""
    rng = np.random.default_rng(seed)
    ref = oracle.Partition(A, part, P)
    m = ref.maps
    ul = rng.uniform(-1, 1, m.nloc)
    vl = rng.uniform(-1, 1, m.nloc)
    d_inv = ref.wdot(ul, vl)
    ref.set_weights(oracle.WEIGHT_OWNER)
    s = 0.0
    for k in sorted(int(i) for i in m.own):
        s += ul[k] * vl[k]
    assert ref.wdot(ul, vl) == s
    ref.set_weights(oracle.WEIGHT_INV_MULT)
    assert ref.wdot(ul, vl) == d_inv


def pin_owner_cg(A, part, P, seed=5):
    """Owner-mask sub-structured CG against dense Cholesky."""
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1, 1, A.n)
    x_chol = oracle.cholesky_solve(_dense(A), b)
    ref = oracle.Partition(A, part, P)
    ref.set_weights(oracle.WEIGHT_OWNER)
    r = ref.cg(b, 1e-12, 20 * A.n)
    assert r.status == oracle.OK
    assert np.linalg.norm(r.x - x_chol) <= 1e-10 * np.linalg.norm(x_chol)


def pin_owner_termination():
    rng = np.random.default_rng(11)
    n = 60
    eye = CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    ref = oracle.Partition(eye, rng.integers(0, 3, n).astype(np.int32), 3)
    ref.set_weights(oracle.WEIGHT_OWNER)
    r = ref.cg(rng.uniform(-1, 1, n), 1e-12, 10)
    assert r.status == oracle.OK and r.iters == 1
    for nn in (16, 64):
        ref = oracle.Partition(laplace1d(nn), (np.arange(nn) * 4 // nn).astype(np.int32), 4)
        ref.set_weights(oracle.WEIGHT_OWNER)
        r = ref.cg(rng.uniform(-1, 1, nn), 1e-10, 10 * nn)
        assert r.status == oracle.OK and r.iters <= nn


def _run_weight_pins():
    failures = []
    checks = [
        ("sum_to_one", lambda: [pin_weights_sum_to_one(*c[1:]) for c in SMALL[:4]]),
        ("owner_brute_force", lambda: [pin_owner_brute_force(*c[1:]) for c in SMALL[:4]]),
        ("owner_cg", lambda: [pin_owner_cg(*c[1:]) for c in SMALL[:3]]),
        ("owner_termination", pin_owner_termination),
    ]
    for name, fn in checks:
        try:
            fn()
        except Exception as e:  # noqa: BLE001 - any failure counts as caught
            failures.append((name, type(e).__name__))
    return failures


def test_weight_pins_pass_on_oracle():
    assert _run_weight_pins() == []


def test_bad_weight_mode_refused():
    c = SMALL[0]
    with pytest.raises(ValueError):
        oracle.Partition(*c[1:]).set_weights(2)


WEIGHT_MUTATIONS = {
    # the mask never clears a copy: every copy weighted 1
    "owner_all_copies": ("        for (int64_t k = 0; k < h->nloc; ++k) h->w[k] = 0.0;\n",
                         "        for (int64_t k = 0; k < h->nloc; ++k) h->w[k] = 1.0;\n"),
    # the first copy of each interface node (lowest subdomain) instead of the owner
    "owner_first_copy": ("        for (int32_t i = 0; i < h->n; ++i) h->w[h->own[i]] = 1.0;\n",
                         "        for (int32_t i = 0; i < h->n; ++i) if (h->mult[i] == 1) h->w[h->own[i]] = 1.0;\n"
                         "        for (int32_t g = 0; g < h->ngamma; ++g) h->w[h->icopy[h->iptr[g]]] = 1.0;\n"),
}


@pytest.mark.parametrize("name", sorted(WEIGHT_MUTATIONS))
def test_planted_weight_mistake_is_caught(name):
    old, new = WEIGHT_MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, "mutation anchor not found: %s" % name
    path = oracle.compile_variant(src.replace(old, new), name)
    try:
        with oracle.use_library(path):
            failures = _run_weight_pins()
    finally:
        os.remove(path)
    assert failures, "planted mistake %s slipped through every pin" % name
