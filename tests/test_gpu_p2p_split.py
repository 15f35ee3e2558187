"""Near-field work units cut by source segment: a target leaf whose strong
list holds more than about 65536 source points is processed as several
units, each against a segment of the list, whose partial sums a combine pass
adds in segment order. With theta = 0 every leaf is strongly connected to
every other, so 70,000 points cut every leaf's list in two and the method is
the exact sum of Eq. 2.1; on a clustered set only the leaves of large boxes
in sparse regions are cut. Results are checked against the oracle's direct
sum on sampled targets (FP64 form to rounding, the mixed form at the bounds
measured for clustered sets) and must be the same on a second evaluation."""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2002_04894_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_theta_zero_every_leaf_split_equals_direct(gpu_lib, prec):
    fmm = gpu_lib
    n = 70000
    x = inputs.points("uniform", n, seed=12)
    q = inputs.charges_uniform(n, seed=12)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), 8, 4, 0.0, prec=prec)
    st = fmm.fmm_plan_stats(plan)
    assert st["weak_pairs"] == 0
    assert st["p2p_partial_slots"] == 2 * n         # every leaf: two segments
    pot, fld = fmm.fmm_eval(plan, torch.from_numpy(q).cuda())
    pot2, fld2 = fmm.fmm_eval(plan, torch.from_numpy(q).cuda())
    assert torch.equal(pot, pot2) and torch.equal(fld, fld2)   # fixed combine order
    t = inputs.sample_targets(n, 1000, 12)
    op, oE = oracle.direct(x, q, targets=t)
    g, e = pot.cpu().numpy()[t], fld.cpu().numpy()[t]
    if prec == 0:
        assert parity.rel_l2(g, op) <= 1e-13 and parity.rel_l2(e, oE) <= 1e-13
        parity.check("split_fp64_theta0", "point_phi", parity.pointwise_phi(g, op), 1e-12)
    else:
        parity.check("split_mixed_theta0", "l2_phi", parity.rel_l2(g, op), 1e-6)
        parity.check("split_mixed_theta0", "l2_field", parity.rel_l2(e, oE), 1e-6)
        parity.check("split_mixed_theta0", "point_phi", parity.pointwise_phi(g, op), 1e-4)


def test_clustered_set_splits_only_heavy_leaves(gpu_lib):
    fmm = gpu_lib
    n = 400000
    x = inputs.points("gmm", n, seed=6).astype(np.float32)
    q = inputs.charges_pm1(n, seed=6).astype(np.float32)
    xd, qd = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    plan = fmm.fmm_plan(xd, 13, 12, 0.5, prec=fmm.FMM_PREC_MIXED, tight=True)
    st = fmm.fmm_plan_stats(plan)
    assert 0 < st["p2p_partial_slots"] < n
    pot, fld = fmm.fmm_eval(plan, qd)
    pot2, _ = fmm.fmm_eval(plan, qd)
    assert torch.equal(pot, pot2)
    t = inputs.sample_targets(n, 500, 6)
    op, oE = oracle.direct(x.astype(np.float64), q.astype(np.float64), targets=t)
    parity.check("split_mixed_gmm", "l2_phi", parity.rel_l2(pot.cpu().numpy()[t], op), 1e-6)
    parity.check("split_mixed_gmm", "l2_field", parity.rel_l2(fld.cpu().numpy()[t], oE), 1e-6)
    # the FP64 form on the same plan geometry, against the same sums
    p64 = fmm.fmm_plan(xd.double(), 13, 12, 0.5, tight=True)
    assert fmm.fmm_plan_stats(p64)["p2p_partial_slots"] > 0
    g64, _ = fmm.fmm_eval(p64, qd.double())
    parity.check("split_fp64_gmm", "l2_phi", parity.rel_l2(g64.cpu().numpy()[t], op), 1e-6)
