"""GPU trees with adaptive splits (Sec. 2.1.2, eta in [0, 1)) vs the oracle,
bit for bit: cut planes eta * median + (1 - eta) * midpoint, children of
data-dependent size (empty ones included), both select/partition regimes,
then the theta-criterion lists and the FP64 evaluation on those trees."""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2002_04894_gb300 import inputs

pytestmark = pytest.mark.gpu

ETAS = [0.0, 0.25, 0.5, 0.75, 0.9]
POINT_TOL = 2e-13
BOX_TOL = 2e-13

CASES = [
    # kind, n, levels: concentrated clouds make the children very unequal
    ("plummer", 30001, 10), ("uniform", 20000, 8), ("gmm", 9000, 9), ("shell", 5000, 8),
    ("plummer", 120000, 12),   # boxes above 4096 points at several levels
    ("uniform", 300, 10),      # most leaves empty
    ("uniform", 5, 3), ("uniform", 1, 3), ("uniform", 2, 1),
]


def ties(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 5, size=(n, 3)).astype(float) - 2.0
    x[::3] *= -1.0
    return x


def make(kind, n):
    return ties(n, n) if kind == "ties" else inputs.points(kind, n, seed=n)


def assert_tree_equal(g, o, levels):
    for k in ("perm", "begin", "count", "lo", "hi", "centre", "radius", "axis"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    internal = (1 << levels) - 1
    np.testing.assert_array_equal(g["plane"][:internal], o["plane"][:internal], err_msg="plane")


@pytest.mark.parametrize("kind,n,levels", CASES + [("ties", 50000, 7), ("ties", 700, 6)])
@pytest.mark.parametrize("eta", ETAS)
def test_tree_eta_bit_exact(gpu_lib, kind, n, levels, eta):
    fmm = gpu_lib
    x = make(kind, n)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), levels, 3, 0.5, eta=eta)
    assert_tree_equal(fmm.fmm_plan_tree(plan), oracle.Tree(x, levels, 3, 0.5, eta=eta).tree(), levels)


def test_eta_one_is_the_median_tree(gpu_lib):
    fmm = gpu_lib
    x = make("plummer", 30001)
    a = fmm.fmm_plan_tree(fmm.fmm_plan(torch.from_numpy(x).cuda(), 10, 3, 0.5))
    b = fmm.fmm_plan_tree(fmm.fmm_plan(torch.from_numpy(x).cuda(), 10, 3, 0.5, eta=1.0))
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_eta_zero_cells_are_bisected_cells(gpu_lib):
    """eta = 0: every cut halves the cell on its longest axis, whatever the
    points, so a concentrated cloud leaves some leaves empty."""
    fmm = gpu_lib
    x = make("plummer", 30001)
    g = fmm.fmm_plan_tree(fmm.fmm_plan(torch.from_numpy(x).cuda(), 9, 3, 0.5, eta=0.0))
    internal = (1 << 9) - 1
    for b in range(internal):
        a = g["axis"][b]
        assert g["plane"][b] == 0.5 * (g["lo"][b, a] + g["hi"][b, a])
    assert np.sum(g["count"][internal:] == 0) > 0


@pytest.mark.parametrize("kind,n,levels", CASES[:6])
@pytest.mark.parametrize("eta", [0.0, 0.5, 0.9])
def test_lists_eta_bit_exact(gpu_lib, kind, n, levels, eta):
    fmm = gpu_lib
    x = make(kind, n)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), levels, 3, 0.5, eta=eta)
    T = oracle.Tree(x, levels, 3, 0.5, eta=eta)
    for l in range(levels + 1):
        for kind_ in ("weak", "strong"):
            gp, gs = fmm.fmm_plan_list(plan, l, kind_)
            op, os_ = T.lists(l, kind_)
            np.testing.assert_array_equal(gp, op, err_msg=f"{kind_} ptr level {l}")
            np.testing.assert_array_equal(gs, os_, err_msg=f"{kind_} src level {l}")


@pytest.mark.parametrize("kind,n,levels,p", [("plummer", 8000, 8, 8), ("gmm", 6000, 8, 10),
                                             ("uniform", 300, 9, 4)])
@pytest.mark.parametrize("eta", [0.0, 0.5])
def test_fmm_eta_matches_oracle(gpu_lib, kind, n, levels, p, eta):
    fmm = gpu_lib
    x = inputs.points(kind, n, seed=5)
    q = inputs.charges_uniform(n, seed=5)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), levels, p, 0.5, eta=eta)
    pot, fld = fmm.fmm_eval(plan, torch.from_numpy(q).cuda())
    T = oracle.Tree(x, levels, p, 0.5, eta=eta)
    op, oE = T.eval(q)
    g, f = pot.cpu().numpy(), fld.cpu().numpy()
    d = np.linalg.norm(g - op) / np.linalg.norm(op)
    e = np.linalg.norm(f - oE) / np.linalg.norm(oE)
    assert d <= 1e-12 and e <= 1e-12
    # element by element (bounds as for the median tree: twice the largest
    # value measured on a GB300)
    tid = f"eta/{kind}/{n}/{levels}/{p}/{eta}"
    gM, oM = fmm.fmm_eval_expansions(plan, "M"), T.expansions("M")
    gL, oL = fmm.fmm_eval_expansions(plan, "L"), T.expansions("L")
    wl = fmm.fmm_plan_stats(plan)["weak_pairs_level"]
    lw = next((l for l in range(1, levels + 1) if wl[l] > 0), levels)
    radius = T.tree()["radius"]
    parity.check(tid, "point_phi", parity.pointwise_phi(g, op), POINT_TOL)
    parity.check(tid, "point_field", parity.pointwise_field(f, oE), POINT_TOL)
    parity.check(tid, "box_M", parity.box_degree(gM, oM, radius, p, "M", slice((1 << lw) - 1, None)), BOX_TOL)
    parity.check(tid, "box_L", parity.box_degree(gL, oL, radius, p, "L"), BOX_TOL)


@pytest.mark.parametrize("eta", [0.0, 0.5])
def test_mixed_eta_accuracy(gpu_lib, eta):
    """The mixed-precision path on unbalanced trees keeps its error target
    against the exact sum (p = 12, theta = 0.5)."""
    fmm = gpu_lib
    n = 60000
    x = inputs.points("plummer", n, seed=9)
    q = inputs.charges_uniform(n, seed=9)
    xd, qd = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    plan = fmm.fmm_plan(xd, 9, 12, 0.5, prec=fmm.FMM_PREC_MIXED, eta=eta)
    pot, _ = fmm.fmm_eval(plan, qd, want_fields=False)
    tgt = inputs.sample_targets(n, 400, 9)
    ref = oracle.direct(x, q, tgt)[0]
    got = pot.cpu().numpy()[tgt]
    # bounds: twice the values measured on a GB300, rounded up
    parity.check(f"eta_mixed_vs_direct/{eta}", "l2_phi", parity.rel_l2(got, ref), 4e-7)
    parity.check(f"eta_mixed_vs_direct/{eta}", "point_phi", parity.pointwise_phi(got, ref),
                 {0.0: 8e-6, 0.5: 7e-6}[eta])
