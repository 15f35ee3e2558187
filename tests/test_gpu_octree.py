"""GPU FMM with levels of 2^s children (s bisections per expansion level; s = 3
is the octree of 8 children per box) vs the oracle: lists bit for bit (64
candidate pairs per strong parent pair for the octree), FP64 expansions and
results to 1e-12 relative L2 and element by element (per target, and per box
with every degree scaled to the box's size; bounds twice the largest value
measured on a GB300), and the mixed-precision path against the exact sum."""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2002_04894_gb300 import inputs

pytestmark = pytest.mark.gpu

POINT_TOL = 2e-13
BOX_TOL = 2e-13

CASES = [
    # kind, n, levels (bisections), step
    ("uniform", 20000, 9, 3), ("plummer", 30001, 12, 3), ("gmm", 9000, 9, 3),
    ("plummer", 6000, 8, 2), ("uniform", 300, 6, 3), ("uniform", 5, 3, 3), ("uniform", 700, 0, 3),
]


@pytest.mark.parametrize("kind,n,levels,step", CASES)
@pytest.mark.parametrize("theta", [0.5, 0.0, 0.7])
def test_octree_lists_bit_exact(gpu_lib, kind, n, levels, step, theta):
    fmm = gpu_lib
    x = inputs.points(kind, n, seed=n)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), levels, 3, theta, bisections_per_level=step)
    T = oracle.Tree(x, levels, 3, theta, step=step)
    for l in range(levels + 1):
        for kind_ in ("weak", "strong"):
            gp, gs = fmm.fmm_plan_list(plan, l, kind_)
            op, os_ = T.lists(l, kind_)
            np.testing.assert_array_equal(gp, op, err_msg=f"{kind_} ptr level {l}")
            np.testing.assert_array_equal(gs, os_, err_msg=f"{kind_} src level {l}")
    st = fmm.fmm_plan_stats(plan)
    assert st["weak_pairs"] == sum(len(T.lists(l, "weak")[1]) for l in range(levels + 1))
    t = T.tree()
    sp, ss = T.lists(levels, "strong")
    off = (1 << levels) - 1
    work = sum(int(t["count"][off + a]) * int(t["count"][off + b])
               for a in range(1 << levels) for b in ss[sp[a]:sp[a + 1]])
    assert st["p2p_interactions"] == work


@pytest.mark.parametrize("kind,n,levels,step,p,theta", [
    ("uniform", 20000, 9, 3, 8, 0.5), ("plummer", 8000, 9, 3, 10, 0.5), ("gmm", 6000, 6, 3, 6, 0.6),
    ("plummer", 5000, 8, 2, 8, 0.5), ("uniform", 800, 6, 3, 5, 0.0), ("uniform", 300, 6, 3, 4, 0.5),
])
def test_octree_fmm_matches_oracle(gpu_lib, kind, n, levels, step, p, theta):
    fmm = gpu_lib
    x = inputs.points(kind, n, seed=21)
    q = inputs.charges_uniform(n, seed=21)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), levels, p, theta, bisections_per_level=step)
    pot, fld = fmm.fmm_eval(plan, torch.from_numpy(q).cuda())
    T = oracle.Tree(x, levels, p, theta, step=step)
    op, oE = T.eval(q)
    gM, gL = fmm.fmm_eval_expansions(plan, "M"), fmm.fmm_eval_expansions(plan, "L")
    oM, oL = T.expansions("M"), T.expansions("L")
    wl = fmm.fmm_plan_stats(plan)["weak_pairs_level"]
    lw = next((l for l in range(1, levels + 1) if wl[l] > 0), levels)
    first = (1 << lw) - 1
    assert np.count_nonzero(gM[:first]) == 0
    for l in range(levels + 1):
        if l % step:   # bisection levels inside an expansion level hold nothing
            lvl = slice((1 << l) - 1, (2 << l) - 1)
            assert np.count_nonzero(gM[lvl]) == 0 and np.count_nonzero(gL[lvl]) == 0
    scaleM = max(np.abs(oM[first:]).max(), 1e-300)
    scaleL = max(np.abs(oL).max(), 1e-300)
    assert np.abs(gM[first:] - oM[first:]).max() <= 1e-12 * scaleM
    assert np.abs(gL - oL).max() <= 1e-12 * scaleL
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    g, e = pot.cpu().numpy(), fld.cpu().numpy()
    assert rel(g, op) <= 1e-12
    assert rel(e, oE) <= 1e-12
    tid = f"octree/{kind}/{n}/{levels}/{step}/{p}/{theta}"
    radius = T.tree()["radius"]
    parity.check(tid, "point_phi", parity.pointwise_phi(g, op), POINT_TOL)
    parity.check(tid, "point_field", parity.pointwise_field(e, oE), POINT_TOL)
    parity.check(tid, "box_M", parity.box_degree(gM, oM, radius, p, "M", slice(first, None)), BOX_TOL)
    parity.check(tid, "box_L", parity.box_degree(gL, oL, radius, p, "L"), BOX_TOL)


def test_octree_mixed_accuracy(gpu_lib):
    """The mixed-precision path on octree levels (p = 12, theta = 0.5) keeps
    its error target against the exact sum."""
    fmm = gpu_lib
    n = 200000
    x = inputs.points("plummer", n, seed=4)
    q = inputs.charges_uniform(n, seed=4)
    xd, qd = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    plan = fmm.fmm_plan(xd, 12, 12, 0.5, prec=fmm.FMM_PREC_MIXED, bisections_per_level=3)
    pot, fld = fmm.fmm_eval(plan, qd)
    tgt = inputs.sample_targets(n, 400, 4)
    ref, refE = oracle.direct(x, q, tgt)
    got = pot.cpu().numpy()[tgt]
    gE = fld.cpu().numpy()[tgt]
    # bounds: twice the values measured on a GB300, rounded up
    parity.check("octree_mixed_vs_direct", "l2_phi", parity.rel_l2(got, ref), 6e-7)
    parity.check("octree_mixed_vs_direct", "l2_field", parity.rel_l2(gE, refE), 5e-7)
    parity.check("octree_mixed_vs_direct", "point_phi", parity.pointwise_phi(got, ref), 2e-5)


def test_octree_rejects_levels_not_multiple(gpu_lib):
    fmm = gpu_lib
    x = torch.from_numpy(inputs.points("uniform", 100, seed=1)).cuda()
    with pytest.raises(fmm.FmmError):
        fmm.fmm_plan(x, 7, 3, 0.5, bisections_per_level=3)
