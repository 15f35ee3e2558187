"""M2M of the mixed form in double-float arithmetic (two floats per value,
about 44 significant bits; coefficients scaled by the parent's radius while
translated). Pinned against the oracle's FP64 M2M (Alg. 1) applied to the
GPU's own child multipoles: every parent multipole of the levels that M2M
forms must match per box and degree to double-float precision, far below
the mixed form's single-precision stages. Covers the one-launch upward pass
(trees up to 13 levels), the per-level launches (deeper trees), tight boxes,
and empty leaves (children outside their parent's tight box are skipped)."""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2002_04894_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.mark.parametrize("kind,n,B,p,tight", [
    ("plummer", 20000, 10, 12, False),
    ("gmm", 30000, 11, 10, True),
    ("uniform", 300, 10, 8, False),      # empty leaves
    ("gmm", 140000, 14, 8, True),        # per-level launches
])
def test_df_m2m_matches_fp64_m2m(gpu_lib, kind, n, B, p, tight):
    fmm = gpu_lib
    x = inputs.points(kind, n, seed=31)
    q = inputs.charges_uniform(n, seed=31)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), B, p, 0.5, prec=fmm.FMM_PREC_MIXED, tight=tight)
    fmm.fmm_eval(plan, torch.from_numpy(q).cuda())
    M = fmm.fmm_eval_expansions(plan, "M")
    tree = fmm.fmm_plan_tree(plan)
    wl = fmm.fmm_plan_stats(plan)["weak_pairs_level"]
    lw = next((l for l in range(1, B + 1) if wl[l] > 0), B + 1)
    nc = oracle.ncoef(p)
    worst = 0.0
    checked = 0
    for l in range(max(lw, 0), B):
        lo, hi = (1 << l) - 1, (2 << l) - 1
        want = np.zeros((hi - lo, nc), complex)
        for g in range(lo, hi):
            for ch in (2 * g + 1, 2 * g + 2):
                if tree["count"][ch] == 0:
                    continue
                oracle.m2m(M[ch], tree["centre"][ch], tree["centre"][g], p, want[g - lo])
        worst = max(worst, parity.box_degree(M[lo:hi], want, tree["radius"][lo:hi], p, "M"))
        checked += hi - lo
    assert checked > 0
    parity.check(f"df_m2m/{kind}/{n}/{B}/{p}", "box_M_vs_fp64_m2m", worst, TOL)
