"""Element-wise parity measures shared by the GPU-vs-oracle tests.

Every measure compares a GPU result with the oracle's value for the SAME
point, box or coefficient, so that an error confined to a few targets (one
leaf's near field, say) or to the high degrees of deep boxes cannot hide
under a norm taken over everything.

  pointwise_phi    max_i |phi_i - phi0_i| / (|phi0_i| + FLOOR * rms(phi0))
  pointwise_field  max_i |E_i - E0_i|_2 / (|E0_i|_2 + FLOOR * rms|E0|)
  box_degree       max over boxes b of
                       max_{n,m} |C_n^m - C0_n^m| s_b^n / max_{n,m} |C0_n^m| s_b^n
                   with s_b = 1 / r_b for multipoles (M_n ~ r^n) and s_b = r_b
                   for locals (L_n ~ r^-n), r_b the box radius: after this
                   scaling every degree of a box has the same size, so the
                   high-degree terms of small boxes are held to the tolerance
                   too; a box whose oracle coefficients are all zero must be
                   zero on the GPU as well.

FLOOR = 0.1: with charges of both signs a potential can pass through zero at
some target, where |phi0_i| alone would turn rounding into an arbitrarily
large relative error; a tenth of the root-mean-square value keeps the measure
relative everywhere else.

If the environment variable FMM_PARITY_LOG names a file, every check appends
one JSON line (test id, measure, value, tolerance) to it: that is how the
tolerances of the mixed-precision cases were measured.
"""
from __future__ import annotations

import json
import os

import numpy as np

FLOOR = 0.1


def rel_l2(a, b) -> float:
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    d = np.linalg.norm(a - b)
    return float(d / nb) if nb > 0 else float(d)


def pointwise_phi(g, o) -> float:
    g, o = np.asarray(g, np.float64).ravel(), np.asarray(o, np.float64).ravel()
    rms = np.sqrt(np.mean(o * o)) if o.size else 0.0
    den = np.abs(o) + FLOOR * rms
    if rms == 0.0:
        return float(np.abs(g - o).max(initial=0.0))
    return float((np.abs(g - o) / den).max(initial=0.0))


def pointwise_field(g, o) -> float:
    g, o = np.asarray(g, np.float64).reshape(-1, 3), np.asarray(o, np.float64).reshape(-1, 3)
    mag = np.linalg.norm(o, axis=1)
    rms = np.sqrt(np.mean(mag * mag)) if mag.size else 0.0
    err = np.linalg.norm(g - o, axis=1)
    if rms == 0.0:
        return float(err.max(initial=0.0))
    return float((err / (mag + FLOOR * rms)).max(initial=0.0))


def degree_of_coef(p: int) -> np.ndarray:
    """Degree n of each stored coefficient (n, m), 0 <= m <= n <= p, packed
    at n(n+1)/2 + m."""
    return np.concatenate([np.full(n + 1, n) for n in range(p + 1)])


def box_degree(G, O, radius, p: int, which: str, boxes=None) -> float:
    """Largest per-box relative error after scaling degree n by r^-n (which =
    'M') or r^n (which = 'L'); `boxes` restricts the comparison (default all).
    Boxes of zero radius are compared unscaled."""
    G, O = np.asarray(G), np.asarray(O)
    r = np.asarray(radius, np.float64)
    if boxes is not None:
        G, O, r = G[boxes], O[boxes], r[boxes]
    n = degree_of_coef(p)[None, :]
    rr = np.where(r > 0, r, 1.0)[:, None]
    s = rr ** (-n) if which == "M" else rr ** n
    d = np.abs(G - O) * s
    o = np.abs(O) * s
    scale = o.max(axis=1)
    dmax = d.max(axis=1)
    zero = scale == 0
    if np.any(dmax[zero] != 0):
        return float("inf")
    if np.all(zero):
        return 0.0
    return float((dmax[~zero] / scale[~zero]).max())


def check(test: str, measure: str, value: float, tol: float) -> None:
    """Assert value <= tol, logging both when FMM_PARITY_LOG is set."""
    path = os.environ.get("FMM_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": test, "measure": measure, "value": value, "tol": tol}) + "\n")
    assert value <= tol, f"{test}: {measure} = {value:.3e} > {tol:.3e}"
