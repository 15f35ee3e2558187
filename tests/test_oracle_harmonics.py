"""Pins for the oracle's solid harmonics: textbook Legendre functions, low-degree
closed forms and the addition theorem for 1/|x - y| (Sec. 2.1's expansions)."""
import math

import numpy as np
import pytest
from scipy.special import lpmv

import oracle


def tri(n, m):
    return n * (n + 1) // 2 + m


def sph(x):
    r = np.linalg.norm(x)
    return r, x[2] / r, math.atan2(x[1], x[0])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_regular_and_irregular_match_legendre_definition(seed):
    """R_n^m = r^n P_n^m e^{im phi}/(n+m)!, I_n^m = (n-m)! P_n^m e^{im phi}/r^{n+1};
    scipy's lpmv carries the Condon-Shortley phase (-1)^m, removed here."""
    x = np.random.default_rng(seed).normal(size=3)
    p = 12
    R, I = oracle.regular(x, p), oracle.irregular(x, p)
    r, ct, ph = sph(x)
    for n in range(p + 1):
        for m in range(n + 1):
            P = (-1) ** m * lpmv(m, n, ct)
            Rref = r**n * P * np.exp(1j * m * ph) / math.factorial(n + m)
            Iref = math.factorial(n - m) * P * np.exp(1j * m * ph) / r ** (n + 1)
            assert abs(R[tri(n, m)] - Rref) <= 1e-12 * max(1.0, abs(Rref))
            assert abs(I[tri(n, m)] - Iref) <= 1e-12 * abs(Iref) + 1e-300


def test_low_degree_closed_forms():
    x, y, z = 0.3, -0.7, 0.45
    r2 = x * x + y * y + z * z
    R = oracle.regular([x, y, z], 2)
    I = oracle.irregular([x, y, z], 1)
    assert R[tri(0, 0)] == 1
    assert R[tri(1, 0)] == pytest.approx(z)
    assert R[tri(1, 1)] == pytest.approx((x + 1j * y) / 2)
    assert R[tri(2, 0)] == pytest.approx((3 * z * z - r2) / 4)
    assert R[tri(2, 1)] == pytest.approx(z * (x + 1j * y) / 2)
    assert R[tri(2, 2)] == pytest.approx((x + 1j * y) ** 2 / 8)
    assert I[tri(0, 0)] == pytest.approx(1 / math.sqrt(r2))
    assert I[tri(1, 0)] == pytest.approx(z / r2**1.5)
    assert I[tri(1, 1)] == pytest.approx((x + 1j * y) / r2**1.5)


def _signed(H, n, m):
    if abs(m) > n:
        return 0
    if m >= 0:
        return (-1) ** m * H[tri(n, m)]
    return np.conj(H[tri(n, -m)])


@pytest.mark.parametrize("ratio", [0.1, 0.3, 0.6])
def test_addition_theorem_reproduces_inverse_distance(ratio):
    rng = np.random.default_rng(4)
    xv = rng.normal(size=3); xv /= np.linalg.norm(xv)
    yv = rng.normal(size=3); yv *= ratio / np.linalg.norm(yv)
    p = 60 if ratio > 0.5 else 30
    R, I = oracle.regular(yv, p), oracle.irregular(xv, p)
    s = sum(np.conj(_signed(R, n, m)) * _signed(I, n, m)
            for n in range(p + 1) for m in range(-n, n + 1))
    exact = 1 / np.linalg.norm(xv - yv)
    assert abs(s.imag) < 1e-14
    assert s.real == pytest.approx(exact, rel=max(1e-14, 3 * ratio ** (p + 1)))


def test_regular_harmonics_are_translation_polynomials():
    """Upsilon_n^m(a+b) = sum_{k,l} Upsilon_k^l(a) Upsilon_{n-k}^{m-l}(b): the
    identity the M2M and L2L operators rest on."""
    rng = np.random.default_rng(7)
    a, b = rng.normal(size=3), rng.normal(size=3)
    p = 8
    Ra, Rb, Rab = oracle.regular(a, p), oracle.regular(b, p), oracle.regular(a + b, p)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            s = sum(_signed(Ra, k, l) * _signed(Rb, n - k, m - l)
                    for k in range(n + 1) for l in range(-k, k + 1))
            assert abs(s - _signed(Rab, n, m)) < 1e-13 * max(1, abs(_signed(Rab, n, m)))
