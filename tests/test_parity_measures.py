"""The element-wise parity measures (tests/parity.py) catch the mistakes that
a norm over everything hides. Mistakes are planted in oracle results on the
CPU, never in the GPU path."""
import numpy as np

import oracle
import parity
from paper_2002_04894_gb300 import inputs


def _tree(levels=8, p=8, n=8000):
    x = inputs.points("plummer", n, seed=3)
    q = inputs.charges_uniform(n, seed=3)
    T = oracle.Tree(x, levels, p, 0.5)
    phi, E = T.eval(q)
    return T, phi, E


def test_one_wrong_leaf_is_caught_per_target_not_in_l2():
    T, phi, E = _tree()
    t = T.tree()
    leaf = (1 << 8) - 1 + 17
    b, c = int(t["begin"][leaf]), int(t["count"][leaf])
    idx = t["perm"][b:b + c]
    bad = phi.copy()
    i = idx[int(np.argmax(np.abs(phi[idx])))]
    bad[i] *= 1 + 1e-6               # one target of one leaf off by 1e-6 relative
    assert parity.rel_l2(bad, phi) < 1e-7          # hidden by the norm over 4000 points
    assert parity.pointwise_phi(bad, phi) > 5e-7  # seen per target
    badE = E.copy()
    mag = np.linalg.norm(E, axis=1)
    i = idx[int(np.argmax(mag[idx]))]
    badE[i, 1] += 1e-6 * mag[i]
    assert parity.rel_l2(badE, E) < 1e-7
    assert parity.pointwise_field(badE, E) > 5e-7


def test_high_degree_of_a_deep_box_is_caught_after_scaling():
    T, _, _ = _tree()
    M = T.expansions("M")
    r = T.tree()["radius"]
    p = 8
    first = (1 << 8) - 1
    leaf = first + int(np.argmin(r[first:]))   # the smallest leaf, near the core
    k = p * (p + 1) // 2 + p           # coefficient (p, p)
    bad = M.copy()
    bad[leaf, k] += 1e-6 * np.abs(M[leaf] * r[leaf] ** -parity.degree_of_coef(p)).max() * r[leaf] ** p
    # invisible against one global scale ...
    assert np.abs(bad - M).max() <= 1e-12 * np.abs(M).max()
    # ... but a 1e-6 error of that box once every degree is scaled to its size
    assert 5e-7 < parity.box_degree(bad, M, r, p, "M") < 2e-6
    L = T.expansions("L")
    assert np.abs(L[leaf]).max() > 0
    badL = L.copy()
    badL[leaf, k] += 1e-6 * np.abs(L[leaf] * r[leaf] ** parity.degree_of_coef(p)).max() / r[leaf] ** p
    assert 5e-7 < parity.box_degree(badL, L, r, p, "L") < 2e-6


def test_zero_boxes_must_stay_zero():
    p = 3
    O = np.zeros((4, oracle.ncoef(p)), np.complex128)
    O[1, 0] = 1.0
    r = np.ones(4)
    assert parity.box_degree(O, O, r, p, "M") == 0.0
    G = O.copy()
    G[2, 3] = 1e-30
    assert parity.box_degree(G, O, r, p, "M") == float("inf")


def test_floor_keeps_zero_crossings_finite():
    o = np.array([1.0, -1.0, 0.0, 2.0])
    g = o + np.array([0.0, 0.0, 1e-9, 0.0])
    v = parity.pointwise_phi(g, o)
    rms = np.sqrt(np.mean(o * o))
    assert v == 1e-9 / (parity.FLOOR * rms)
