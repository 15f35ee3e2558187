"""Seeded synthetic point sets and charges for the FMM workloads.

This module holds no part of the method's arithmetic: it only draws inputs.
Both the CUDA path's tests and benchmark and the CPU oracle's tests take their
inputs from here, so the two sides always see the same bits.

Distributions (the paper's test sets, Sec. 3.2 and 3.3, give no parameters
beyond their names; the stand-ins below are stated in the design notes):
  uniform   points uniform in the unit cube
  plummer   Plummer sphere, scale radius a, truncated at rmax, centred at 0.5
  gmm       mixture of isotropic Gaussians, sigma log-uniform, centres uniform
  gaussian  one spherical Gaussian (sigma 0.1) centred at 0.5
  shell     spherical shell (radius 0.4, thickness 0.01) centred at 0.5
  helix     3-turn helix of radius 0.3 with 0.01 jitter
  galaxy    multiscale disc after the recipe of Sec. 3.5: a seed ring of
            10,000 points (radii 6000-18000 pc, two logarithmic arms), then
            generations that replace every point by 10 points uniform in an
            oblate spheroid around it (semi-axes R_k, R_k, R_k / 10 with
            R_0 = 18000 / 20 pc, R_{k+1} = 2/3 R_k), scaled into the unit cube
"""
from __future__ import annotations

import numpy as np


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def uniform(n: int, seed: int = 0) -> np.ndarray:
    return np.random.default_rng(seed).random((n, 3))


def plummer(n: int, seed: int = 0, a: float = 0.1, rmax_over_a: float = 10.0) -> np.ndarray:
    """Plummer radii r = a / sqrt(u^(-2/3) - 1), rejecting r > rmax."""
    rng = np.random.default_rng(seed)
    out = np.empty((0, 3))
    while len(out) < n:
        m = int((n - len(out)) * 1.05) + 16
        u = rng.random(m)
        u = u[u > 0]
        r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        r = r[r <= rmax_over_a * a]
        pts = 0.5 + r[:, None] * _isotropic(rng, len(r))
        out = np.concatenate([out, pts])
    return np.ascontiguousarray(out[:n])


def gmm(n: int, seed: int = 0, k: int = 16, log10_sigma=(-3.0, -1.0)) -> np.ndarray:
    """Equal-weight mixture of k isotropic Gaussians."""
    rng = np.random.default_rng(seed)
    centres = rng.random((k, 3))
    sigma = 10.0 ** rng.uniform(log10_sigma[0], log10_sigma[1], size=k)
    comp = rng.integers(0, k, size=n)
    return np.ascontiguousarray(centres[comp] + sigma[comp, None] * rng.normal(size=(n, 3)))


def gaussian(n: int, seed: int = 0, sigma: float = 0.1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return 0.5 + sigma * rng.normal(size=(n, 3))


def shell(n: int, seed: int = 0, radius: float = 0.4, thickness: float = 0.01) -> np.ndarray:
    rng = np.random.default_rng(seed)
    r = radius + thickness * (rng.random(n) - 0.5)
    return 0.5 + r[:, None] * _isotropic(rng, n)


def helix(n: int, seed: int = 0, turns: float = 3.0, radius: float = 0.3, jitter: float = 0.01) -> np.ndarray:
    rng = np.random.default_rng(seed)
    t = rng.random(n)
    ang = 2.0 * np.pi * turns * t
    pts = np.stack([0.5 + radius * np.cos(ang), 0.5 + radius * np.sin(ang), t], axis=1)
    return pts + jitter * rng.normal(size=(n, 3))


def _in_unit_ball(rng: np.random.Generator, n: int) -> np.ndarray:
    return _isotropic(rng, n) * rng.random(n)[:, None] ** (1.0 / 3.0)


def galaxy(n: int, seed: int = 0, seeds: int = 10_000, r_inner: float = 6000.0,
           r_outer: float = 18000.0, children: int = 10) -> np.ndarray:
    """Spiral-galaxy stand-in: seed ring with two logarithmic arms (pitch
    15 degrees, 0.1 rad azimuthal scatter, 300 pc thickness), refined by
    generations of `children` points per parent in shrinking oblate
    spheroids; the last generation refines a random subset of parents."""
    rng = np.random.default_rng([seed, 7])
    m0 = min(seeds, n)
    r = r_inner + (r_outer - r_inner) * rng.random(m0)
    arm = rng.integers(0, 2, size=m0)
    phi = np.log(r / r_inner) / np.tan(np.radians(15.0)) + np.pi * arm + 0.1 * rng.normal(size=m0)
    pts = np.stack([r * np.cos(phi), r * np.sin(phi), 300.0 * rng.normal(size=m0)], axis=1)
    big = r_outer / 20.0
    while len(pts) < n:
        need = min(n, len(pts) * children)
        parents = pts[rng.permutation(len(pts))][: -(-need // children)]
        kids = np.repeat(parents, children, axis=0)[:need]
        off = _in_unit_ball(rng, need) * np.array([big, big, big / 10.0])
        pts = kids + off
        big *= 2.0 / 3.0
    scale = 1.0 / (2.2 * r_outer)
    return np.ascontiguousarray(0.5 + scale * pts[:n])


DISTRIBUTIONS = dict(uniform=uniform, plummer=plummer, gmm=gmm, gaussian=gaussian,
                     shell=shell, helix=helix, galaxy=galaxy)


def points(kind: str, n: int, seed: int = 0) -> np.ndarray:
    return np.ascontiguousarray(DISTRIBUTIONS[kind](n, seed), dtype=np.float64)


def charges_uniform(n: int, seed: int = 0) -> np.ndarray:
    """Charges uniform in [-1, 1); drawn from an independent stream."""
    return np.random.default_rng([seed, 1]).uniform(-1.0, 1.0, size=n)


def charges_pm1(n: int, seed: int = 0) -> np.ndarray:
    """Charges +1 or -1 with equal probability."""
    return np.random.default_rng([seed, 1]).integers(0, 2, size=n) * 2.0 - 1.0


def sample_targets(n: int, k: int = 1000, seed: int = 0) -> np.ndarray:
    """k distinct target indices (all of them if n <= k), ascending."""
    if n <= k:
        return np.arange(n, dtype=np.int64)
    rng = np.random.default_rng([seed, 2])
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)
