"""GPU FMM evaluation vs the FP64 oracle, stage by stage (Algorithm 1): the
multipole coefficients after P2M/M2M, the local coefficients after M2L/L2L,
and the final potentials and fields (Eq. 2.1 approximated).

Tolerances. Both sides sum the same truncated series in double precision in
a different order, so only rounding differs:
  - relative L2 over all points, potentials and fields: 1e-12;
  - per target (parity.pointwise_*): POINT_TOL;
  - per box, every degree scaled to the box's size (parity.box_degree):
    BOX_TOL.
The per-target and per-box bounds are twice the largest value measured over
these cases on a GB300, rounded up to one significant digit."""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2002_04894_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12
POINT_TOL = 2e-13
BOX_TOL = 2e-13


def rel(a, b):
    d = np.linalg.norm(np.asarray(a) - np.asarray(b))
    nb = np.linalg.norm(b)
    return d / nb if nb > 0 else d


CASES = [
    # kind, n, levels, p, theta
    ("uniform", 20000, 8, 8, 0.5),     # the small uniform configuration
    ("uniform", 20000, 4, 8, 0.5),     # literal 4 levels: pure near field
    ("plummer", 6000, 7, 10, 0.5),
    ("gmm", 5000, 8, 6, 0.4),
    ("uniform", 3001, 7, 12, 0.6),
    ("uniform", 300, 10, 4, 0.5),      # more leaves than points: empty leaves
    ("uniform", 1000, 5, 0, 0.5),      # monopole only
    ("uniform", 800, 6, 5, 0.0),       # theta = 0: no weak pairs
    ("plummer", 500, 0, 3, 0.5),       # no bisection
    ("uniform", 1, 2, 3, 0.5),
]


@pytest.mark.parametrize("kind,n,levels,p,theta", CASES)
def test_fmm_matches_oracle(gpu_lib, kind, n, levels, p, theta):
    fmm = gpu_lib
    x = inputs.points(kind, n, seed=11)
    q = inputs.charges_uniform(n, seed=11)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), levels, p, theta)
    pot, fld = fmm.fmm_eval(plan, torch.from_numpy(q).cuda())
    T = oracle.Tree(x, levels, p, theta)
    op, oE = T.eval(q)
    gM, gL = fmm.fmm_eval_expansions(plan, "M"), fmm.fmm_eval_expansions(plan, "L")
    oM, oL = T.expansions("M"), T.expansions("L")
    # multipoles above the first level with weak pairs are not formed (unused)
    wl = fmm.fmm_plan_stats(plan)["weak_pairs_level"]
    lw = next((l for l in range(1, levels + 1) if wl[l] > 0), levels)
    first = (1 << lw) - 1
    assert np.count_nonzero(gM[:first]) == 0
    scaleM = max(np.abs(oM[first:]).max(), 1e-300)
    scaleL = max(np.abs(oL).max(), 1e-300)
    assert np.abs(gM[first:] - oM[first:]).max() <= TOL * scaleM
    assert np.abs(gL - oL).max() <= TOL * scaleL
    g, e = pot.cpu().numpy(), fld.cpu().numpy()
    assert rel(g, op) <= TOL
    assert rel(e, oE) <= TOL
    tid = f"fp64/{kind}/{n}/{levels}/{p}/{theta}"
    radius = T.tree()["radius"]
    parity.check(tid, "point_phi", parity.pointwise_phi(g, op), POINT_TOL)
    parity.check(tid, "point_field", parity.pointwise_field(e, oE), POINT_TOL)
    parity.check(tid, "box_M", parity.box_degree(gM, oM, radius, p, "M", slice(first, None)), BOX_TOL)
    parity.check(tid, "box_L", parity.box_degree(gL, oL, radius, p, "L"), BOX_TOL)


def test_host_buffers_give_identical_bits(gpu_lib):
    fmm = gpu_lib
    x = inputs.points("plummer", 7000, 2)
    q = inputs.charges_uniform(7000, 2)
    pd = fmm.fmm_plan(torch.from_numpy(x).cuda(), 7, 6, 0.5)
    a, ea = fmm.fmm_eval(pd, torch.from_numpy(q).cuda())
    ph = fmm.fmm_plan(x, 7, 6, 0.5, allocator=None)
    b, eb = fmm.fmm_eval(ph, q)
    np.testing.assert_array_equal(a.cpu().numpy(), b)
    np.testing.assert_array_equal(ea.cpu().numpy(), eb)


def test_library_pool_reuse_and_trim(gpu_lib):
    """Plans without an allocator draw from the library's pool: a plan built
    after another was destroyed (memory kept in the pool), and after the pool
    was trimmed, gives the same results."""
    fmm = gpu_lib
    x = inputs.points("plummer", 6000, 4)
    q = inputs.charges_uniform(6000, 4)
    p1 = fmm.fmm_plan(x, 7, 6, 0.5, allocator=None)
    a, ea = fmm.fmm_eval(p1, q)
    fmm.fmm_destroy(p1)
    p2 = fmm.fmm_plan(x, 7, 6, 0.5, allocator=None)
    b, eb = fmm.fmm_eval(p2, q)
    fmm.fmm_destroy(p2)
    fmm.fmm_pool_trim(torch.cuda.current_device())
    p3 = fmm.fmm_plan(x, 7, 6, 0.5, allocator=None)
    c, ec = fmm.fmm_eval(p3, q)
    fmm.fmm_destroy(p3)
    for u, v in ((a, b), (ea, eb), (a, c), (ea, ec)):
        np.testing.assert_array_equal(u, v)
    with pytest.raises(RuntimeError):
        fmm.fmm_pool_trim(64)


def test_repeated_eval_and_recharge(gpu_lib):
    fmm = gpu_lib
    x = inputs.points("uniform", 4000, 3)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), 6, 6, 0.5)
    q1 = inputs.charges_uniform(4000, 1)
    q2 = inputs.charges_pm1(4000, 2)
    a1, _ = fmm.fmm_eval(plan, torch.from_numpy(q1).cuda())
    a2, _ = fmm.fmm_eval(plan, torch.from_numpy(q2).cuda())
    a3, _ = fmm.fmm_eval(plan, torch.from_numpy(q1).cuda())
    assert torch.equal(a1, a3)
    T = oracle.Tree(x, 6, 6, 0.5)
    assert rel(a2.cpu().numpy(), T.eval(q2, field=False)) <= TOL


def test_zero_charges_give_zero(gpu_lib):
    fmm = gpu_lib
    x = inputs.points("gmm", 3000, 3)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), 6, 5, 0.5)
    pot, fld = fmm.fmm_eval(plan, torch.zeros(3000, dtype=torch.float64, device="cuda"))
    assert torch.count_nonzero(pot).item() == 0 and torch.count_nonzero(fld).item() == 0


def test_direct_matches_oracle(gpu_lib):
    fmm = gpu_lib
    x = inputs.points("plummer", 30000, 5)
    q = inputs.charges_uniform(30000, 5)
    t = inputs.sample_targets(30000, 257, 5)
    gp, gE = fmm.fmm_direct(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(),
                            torch.from_numpy(t).cuda())
    op, oE = oracle.direct(x, q, targets=t)
    assert rel(gp.cpu().numpy(), op) <= 1e-14
    assert rel(gE.cpu().numpy(), oE) <= 1e-14
    hp, hE = fmm.fmm_direct(x, q, t)
    np.testing.assert_array_equal(hp, gp.cpu().numpy())
