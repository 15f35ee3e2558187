"""Mixed-precision form (FMM_PREC_MIXED) vs the FP64 oracle.

P2M, M2L, L2P and P2P run in float with leaf-centred split coordinates,
radius-scaled expansions and Kahan-compensated near-field sums; geometry,
lists, M2M and L2L stay FP64. The tree and lists are identical to the FP64
form (bit-exact). Tolerance on potentials and fields against the oracle's
FMM with the same p and theta: 1e-5 relative L2 -- float unit roundoff
(6e-8) times the ~100-fold growth of the longest reductions (13-term folds
in five chained steps of the rotation M2L, ~16k-term near-field sums
compensated to O(u)), rounded up."""
import numpy as np
import pytest
import torch

import oracle
from paper_2002_04894_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


CASES = [
    ("uniform", 20000, 8, 8, 0.5, np.float64),
    ("plummer", 12000, 8, 10, 0.5, np.float64),
    ("gmm", 9000, 9, 12, 0.5, np.float32),
    ("uniform", 5000, 7, 14, 0.6, np.float64),
    ("plummer", 4000, 7, 16, 0.6, np.float64),   # highest float M2L order: one pair per thread
    ("gmm", 6000, 8, 6, 0.5, np.float64),
    ("plummer", 3000, 6, 7, 0.5, np.float64),    # p without a float M2L instance
    ("uniform", 300, 10, 4, 0.5, np.float64),    # empty leaves
    ("uniform", 1000, 5, 6, 0.0, np.float32),    # theta = 0: near field only
]


@pytest.mark.parametrize("kind,n,levels,p,theta,dt", CASES)
def test_mixed_matches_oracle(gpu_lib, kind, n, levels, p, theta, dt):
    fmm = gpu_lib
    x = inputs.points(kind, n, seed=21).astype(dt)
    q = inputs.charges_uniform(n, seed=21).astype(dt)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), levels, p, theta, prec=fmm.FMM_PREC_MIXED)
    pot, fld = fmm.fmm_eval(plan, torch.from_numpy(q).cuda())
    T = oracle.Tree(x.astype(np.float64), levels, p, theta)
    op, oE = T.eval(q.astype(np.float64))
    np.testing.assert_array_equal(fmm.fmm_plan_tree(plan)["perm"], T.tree()["perm"])
    e_phi = rel(pot.double().cpu().numpy(), op)
    e_E = rel(fld.double().cpu().numpy(), oE)
    assert e_phi <= TOL and e_E <= TOL, (e_phi, e_E)
    gM, oM = fmm.fmm_eval_expansions(plan, "M"), T.expansions("M")
    leaves = slice((1 << levels) - 1, None)
    for g in range((1 << levels) - 1, (2 << levels) - 1):
        s = np.abs(oM[g]).max()
        if s > 0:
            assert np.abs(gM[g] - oM[g]).max() <= TOL * s


def test_close_pairs_keep_relative_precision(gpu_lib):
    """Two points 1e-9 apart inside a unit-size leaf: the split coordinates
    make their difference exact, so their mutual term is not lost."""
    fmm = gpu_lib
    x = inputs.points("uniform", 64, 3)
    x[1] = x[0] + np.array([1e-9, 0.0, 0.0])
    q = np.zeros(64)
    q[1] = 1.0
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), 0, 4, 0.5, prec=fmm.FMM_PREC_MIXED)
    pot, fld = fmm.fmm_eval(plan, torch.from_numpy(q).cuda())
    assert pot[0].item() == pytest.approx(1e9, rel=1e-5)
    assert fld[0, 0].item() == pytest.approx(-1e18, rel=1e-5)


def test_mixed_vs_direct_accuracy(gpu_lib):
    fmm = gpu_lib
    n = 40000
    x = inputs.points("plummer", n, 8)
    q = inputs.charges_uniform(n, 8)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), 9, 12, 0.5, prec=fmm.FMM_PREC_MIXED)
    pot, fld = fmm.fmm_eval(plan, torch.from_numpy(q).cuda())
    t = inputs.sample_targets(n, 400, 8)
    op, oE = oracle.direct(x, q, targets=t)
    assert rel(pot.cpu().numpy()[t], op) < 3e-6


def test_plans_of_different_orders_coexist(gpu_lib):
    """A plan built after another with a smaller order must not shrink the
    shared-memory limit of the kernels the first one launches."""
    fmm = gpu_lib
    n = 20000
    x = torch.from_numpy(inputs.points("plummer", n, 3)).cuda()
    q = torch.from_numpy(inputs.charges_uniform(n, 3)).cuda()
    big = fmm.fmm_plan(x, 8, 16, 0.5, prec=fmm.FMM_PREC_MIXED)
    big64 = fmm.fmm_plan(x, 8, 14, 0.5)
    small = fmm.fmm_plan(x, 8, 2, 0.5, prec=fmm.FMM_PREC_MIXED)
    small64 = fmm.fmm_plan(x, 8, 3, 0.5)
    for plan in (big, big64, small, small64):
        pot, _ = fmm.fmm_eval(plan, q)
        assert torch.isfinite(pot).all()
