"""Pins for the oracle's expansion operators (Algorithm 1, 3 and 4 stages):
exactness of the polynomial re-centrings, closed forms at low order and
convergence to the direct sum (the a-priori bound of Sec. 3.1)."""
import numpy as np
import pytest

import oracle


def cluster(seed, n, centre, half):
    rng = np.random.default_rng(seed)
    return np.asarray(centre) + half * (2 * rng.random((n, 3)) - 1), rng.uniform(-1, 1, n)


def far_direct(xs, qs, targets):
    """Potential and field of sources at far targets, via the oracle's Eq. 2.1
    sum with zero-charge probes."""
    x = np.vstack([xs, targets])
    q = np.r_[qs, np.zeros(len(targets))]
    return oracle.direct(x, q, targets=np.arange(len(xs), len(x)))


def eval_multipole(M, c, p, x):
    """phi(x) = sum_{n,m} M_n^m Theta_n^m(x - c), real-charge symmetry."""
    I = oracle.irregular(np.asarray(x) - c, p)
    s = 0.0
    for n in range(p + 1):
        s += M[n * (n + 1) // 2].real * I[n * (n + 1) // 2].real
        for m in range(1, n + 1):
            s += 2 * ((-1) ** m * M[n * (n + 1) // 2 + m] * I[n * (n + 1) // 2 + m]).real
    return s


def test_p2m_low_order_closed_forms():
    xs, qs = cluster(0, 30, [0.2, 0.1, -0.3], 0.2)
    c = np.array([0.2, 0.1, -0.3])
    M = oracle.p2m(xs, qs, c, 2)
    d = xs - c
    assert M[0] == pytest.approx(qs.sum())                       # monopole
    assert M[1] == pytest.approx(np.sum(qs * d[:, 2]))           # M_1^0 = sum q z
    # M_1^1 = sum q conj(Upsilon_1^1) = sum q * (-(x - i y)/2)
    assert M[2] == pytest.approx(np.sum(qs * -(d[:, 0] - 1j * d[:, 1]) / 2))


@pytest.mark.parametrize("p", [0, 4, 8, 16])
def test_p2m_far_field_converges_to_direct(p):
    xs, qs = cluster(1, 50, [0, 0, 0], 0.25)
    M = oracle.p2m(xs, qs, np.zeros(3), p)
    rng = np.random.default_rng(2)
    t = rng.normal(size=(20, 3)); t *= 2.0 / np.linalg.norm(t, axis=1, keepdims=True)
    ref = far_direct(xs, qs, t)[0]
    got = np.array([eval_multipole(M, np.zeros(3), p, x) for x in t])
    rho = np.sqrt(3) * 0.25 / 2.0
    err = np.abs(got - ref).max() / np.abs(qs).sum() * 2.0
    assert err <= 2 * rho ** (p + 1) / (1 - rho) + 1e-14


def test_m2m_is_exact():
    """M2M(P2M(child points), child -> parent) equals P2M(parent points): the
    shift of a truncated multipole expansion is exact (Algorithm 1, M2M)."""
    p = 10
    xa, qa = cluster(3, 40, [0.1, 0.2, 0.3], 0.1)
    xb, qb = cluster(4, 35, [0.35, 0.1, 0.2], 0.1)
    ca, cb, cp = np.array([0.1, 0.2, 0.3]), np.array([0.35, 0.1, 0.2]), np.array([0.2, 0.16, 0.27])
    Mp = oracle.m2m(oracle.p2m(xa, qa, ca, p), ca, cp, p)
    oracle.m2m(oracle.p2m(xb, qb, cb, p), cb, cp, p, Mp)
    ref = oracle.p2m(np.vstack([xa, xb]), np.r_[qa, qb], cp, p)
    assert np.abs(Mp - ref).max() <= 1e-14 * np.abs(ref).max()


def test_l2l_is_exact():
    """Re-centring a truncated local expansion is exact: L2P(L2L(L)) = L2P(L)."""
    p = 9
    rng = np.random.default_rng(6)
    xs, qs = cluster(5, 30, [3, 0, 0], 0.3)
    L = oracle.m2l(oracle.p2m(xs, qs, [3, 0, 0], p), [3, 0, 0], [0, 0, 0], p)
    cc = np.array([0.1, -0.05, 0.08])
    Lc = oracle.l2l(L, np.zeros(3), cc, p)
    for x in 0.1 * rng.normal(size=(10, 3)):
        f1, e1 = oracle.l2p(L, np.zeros(3), p, x)
        f2, e2 = oracle.l2p(Lc, cc, p, x)
        assert f2 == pytest.approx(f1, rel=1e-13)
        np.testing.assert_allclose(e2, e1, rtol=1e-12, atol=1e-13 * np.abs(e1).max())


def test_l2p_field_is_minus_gradient():
    p = 8
    xs, qs = cluster(8, 20, [2, 1, 0], 0.3)
    L = oracle.m2l(oracle.p2m(xs, qs, [2, 1, 0], p), [2, 1, 0], [0, 0, 0], p)
    x = np.array([0.05, -0.1, 0.07]); h = 1e-5
    _, E = oracle.l2p(L, np.zeros(3), p, x)
    g = [(oracle.l2p(L, np.zeros(3), p, x + h * e)[0] - oracle.l2p(L, np.zeros(3), p, x - h * e)[0]) / (2 * h)
         for e in np.eye(3)]
    np.testing.assert_allclose(E, -np.array(g), rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7])
def test_m2l_converges_within_theta_bound(theta):
    """Two boxes at the theta-criterion's limit (R + theta*r = theta*d):
    L2P(M2L(P2M)) approaches the direct far-field sum geometrically in p, and
    the relative error stays below C theta^(p+1)/(1 - theta)^2 (Sec. 3.1)."""
    half = 0.1
    rad = half * np.sqrt(3)
    d = (rad + theta * rad) / theta
    cs, ct = np.zeros(3), np.array([d, 0.0, 0.0]) / np.sqrt(1.0)
    xs, qs = cluster(11, 60, cs, half)
    qs = np.abs(qs)                          # positive charges, as in Sec. 3.1
    xt = ct + half * (2 * np.random.default_rng(12).random((25, 3)) - 1)
    ref, Eref = far_direct(xs, qs, xt)
    errs = []
    for p in range(2, 15, 2):
        L = oracle.m2l(oracle.p2m(xs, qs, cs, p), cs, ct, p)
        got = np.array([oracle.l2p(L, ct, p, x)[0] for x in xt])
        errs.append(np.abs((got - ref) / ref).max())
        assert errs[-1] <= 1.0 * theta ** (p + 1) / (1 - theta) ** 2
    assert errs[-1] < 1e-3 * errs[0]
    ratios = np.array(errs[1:]) / np.array(errs[:-1])
    assert np.median(ratios) < theta ** 2 * 1.5 + 0.05  # two orders per step


def test_m2l_matches_direct_at_high_order_any_direction():
    p = 20
    rng = np.random.default_rng(13)
    for _ in range(3):
        v = rng.normal(size=3); v /= np.linalg.norm(v)
        cs, ct = np.zeros(3), 1.5 * v
        xs, qs = cluster(int(rng.integers(100)), 20, cs, 0.12)
        xt = ct + 0.12 * (2 * rng.random((5, 3)) - 1)
        ref, Eref = far_direct(xs, qs, xt)
        L = oracle.m2l(oracle.p2m(xs, qs, cs, p), cs, ct, p)
        for x, r0, e0 in zip(xt, ref, Eref):
            f, e = oracle.l2p(L, ct, p, x)
            assert f == pytest.approx(r0, rel=1e-10, abs=1e-12)
            np.testing.assert_allclose(e, e0, rtol=1e-8, atol=1e-9)
