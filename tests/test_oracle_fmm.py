"""Pins for the whole oracle FMM (Algorithm 1): special cases that reduce to
the direct sum, the convergence experiment of Sec. 3.1, and accuracy vs Eq. 2.1."""
import math

import numpy as np
import pytest

import oracle
from paper_2002_04894_gb300 import inputs


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_theta_zero_is_direct_sum():
    x = inputs.points("uniform", 600, 1); q = inputs.charges_uniform(600, 1)
    phi, E = oracle.Tree(x, 5, 6, 0.0).eval(q)
    p0, E0 = oracle.direct(x, q)
    assert rel(phi, p0) < 1e-14 and rel(E, E0) < 1e-14


def test_zero_levels_is_direct_sum():
    x = inputs.points("plummer", 500, 2); q = inputs.charges_uniform(500, 2)
    phi, E = oracle.Tree(x, 0, 4, 0.5).eval(q)
    p0, E0 = oracle.direct(x, q)
    assert rel(phi, p0) < 1e-14 and rel(E, E0) < 1e-14


def test_convergence_experiment_sec31():
    """N = 1000 random points, positive charges: the relative error
    |(phi0 - phi)/phi0| falls geometrically with p, roughly by theta per order,
    to the double-precision floor, and stays under C theta^(p+1)/(1-theta)^2."""
    n, theta = 1000, 0.5
    x = inputs.points("uniform", n, 0)
    q = np.abs(inputs.charges_uniform(n, 0))
    p0 = oracle.direct(x, q, field=False)
    errs = []
    for p in range(1, 32, 3):
        phi = oracle.Tree(x, 6, p, theta).eval(q, field=False)
        errs.append((p, np.max(np.abs((p0 - phi) / p0))))
    es = np.array([e for _, e in errs])
    ps = np.array([p for p, _ in errs])
    C = np.max(es / (theta ** (ps + 1) / (1 - theta) ** 2))
    assert C < 1.0
    assert es[-1] < 1e-13                                   # reaches the FP64 floor
    fit = np.polyfit(ps[es > 1e-12], np.log(es[es > 1e-12]), 1)[0]
    assert math.exp(fit) < theta                           # at least as fast as theta^p


@pytest.mark.parametrize("kind,levels,p,theta,tol", [
    ("uniform", 7, 8, 0.5, 5e-6), ("plummer", 8, 10, 0.5, 1e-6),
    ("gmm", 8, 6, 0.4, 1e-5), ("uniform", 6, 3, 0.6, 1e-2)])
def test_fmm_error_vs_direct_on_sampled_targets(kind, levels, p, theta, tol):
    n = 6000
    x = inputs.points(kind, n, 3); q = inputs.charges_uniform(n, 3)
    phi, E = oracle.Tree(x, levels, p, theta).eval(q)
    t = inputs.sample_targets(n, 300, 3)
    p0, E0 = oracle.direct(x, q, targets=t)
    assert rel(phi[t], p0) < tol
    assert rel(E[t], E0) < 10 * tol


def test_expansions_monopole_is_box_charge():
    x = inputs.points("uniform", 900, 5); q = inputs.charges_uniform(900, 5)
    T = oracle.Tree(x, 4, 3, 0.5)
    T.eval(q)
    M = T.expansions("M")
    t = T.tree()
    for g in range(T.nbox):
        pts = t["perm"][t["begin"][g]:t["begin"][g] + t["count"][g]]
        assert M[g, 0].real == pytest.approx(q[pts].sum(), abs=1e-12)
