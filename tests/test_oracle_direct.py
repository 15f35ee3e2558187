"""Pins for the oracle's exact pairwise sum (Eq. 2.1) against closed forms,
symmetry and Gauss's law -- nothing here re-derives the sum it checks."""
import math
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_two_charges_closed_form():
    x = np.array([[0.1, 0.2, 0.3], [0.4, -0.2, 1.5]])
    q = np.array([2.0, -0.5])
    phi, E = oracle.direct(x, q)
    d = x[0] - x[1]
    r = np.linalg.norm(d)
    assert phi[0] == pytest.approx(-0.5 / r, rel=1e-15)
    assert phi[1] == pytest.approx(2.0 / r, rel=1e-15)
    np.testing.assert_allclose(E[0], -0.5 * d / r**3, rtol=1e-14)
    np.testing.assert_allclose(E[1], 2.0 * (-d) / r**3, rtol=1e-14)


def test_cube_corners_golden():
    g = _golden("cube_corners.txt")
    corners = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], float)
    phi, E = oracle.direct(corners, np.ones(8))
    np.testing.assert_allclose(phi, g["phi_corner"], rtol=1e-15)
    for c, e in zip(corners, E):
        outward = (c - 0.5) / np.linalg.norm(c - 0.5)
        np.testing.assert_allclose(e, g["E_corner"] * outward, rtol=1e-14, atol=1e-15)
    # probe at the centre: symmetric, so E = 0; charge 0 so it adds nothing
    x = np.vstack([corners, [0.5, 0.5, 0.5]])
    phi, E = oracle.direct(x, np.r_[np.ones(8), 0.0], targets=[8])
    assert phi[0] == pytest.approx(g["phi_centre"], rel=1e-15)
    assert np.abs(E[0]).max() < 1e-14


def test_field_is_minus_gradient_of_potential():
    rng = np.random.default_rng(3)
    x = rng.random((40, 3))
    q = rng.uniform(-1, 1, 40)
    _, E = oracle.direct(x, q, targets=[7])
    h = 1e-5
    g = np.zeros(3)
    for a in range(3):
        xp, xm = x.copy(), x.copy()
        xp[7, a] += h
        xm[7, a] -= h
        g[a] = (oracle.direct(xp, q, [7], field=False)[0] - oracle.direct(xm, q, [7], field=False)[0]) / (2 * h)
    np.testing.assert_allclose(E[0], -g, rtol=1e-7, atol=1e-8)


def test_gauss_law_flux():
    """Flux of E through a sphere = 4*pi*(enclosed charge), Lebedev-free:
    a fine product rule over (cos theta, phi) on a probe sphere."""
    rng = np.random.default_rng(5)
    src = 0.3 * rng.random((6, 3)) + 0.35            # inside |x - c| < 0.35
    qs = rng.uniform(-1, 1, 6)
    c = np.array([0.5, 0.5, 0.5]); R = 0.9
    nt, npf = 64, 128
    ct, wt = np.polynomial.legendre.leggauss(nt)
    ph = (np.arange(npf) + 0.5) * 2 * np.pi / npf
    CT, PH = np.meshgrid(ct, ph, indexing="ij")
    st = np.sqrt(1 - CT**2)
    nrm = np.stack([st * np.cos(PH), st * np.sin(PH), CT], -1).reshape(-1, 3)
    probes = c + R * nrm
    x = np.vstack([src, probes])
    q = np.r_[qs, np.zeros(len(probes))]
    _, E = oracle.direct(x, q, targets=np.arange(6, len(x)))
    flux = (np.sum(E * nrm, 1).reshape(nt, npf) * wt[:, None]).sum() * (2 * np.pi / npf) * R**2
    assert flux == pytest.approx(4 * np.pi * qs.sum(), rel=1e-9, abs=1e-9)


def test_self_and_coincident_pairs_are_skipped():
    x = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    q = np.array([1.0, 5.0, 2.0])
    phi, E = oracle.direct(x, q)
    assert phi[0] == 2.0 and phi[1] == 2.0 and phi[2] == 6.0
    np.testing.assert_array_equal(E[0], [-2.0, 0.0, 0.0])


def test_targets_subset_matches_full():
    rng = np.random.default_rng(9)
    x = rng.random((300, 3)); q = rng.uniform(-1, 1, 300)
    phi, E = oracle.direct(x, q)
    t = np.array([0, 17, 299, 150])
    p2, E2 = oracle.direct(x, q, targets=t)
    np.testing.assert_array_equal(p2, phi[t])
    np.testing.assert_array_equal(E2, E[t])
