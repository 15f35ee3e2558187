"""GPU tree and connectivity vs the oracle, bit for bit (Sec. 2.1.2, Eq. 2.2,
Algorithm 2). Both regimes of the select/partition are covered: boxes above
4096 points use the multi-CTA path, smaller ones the one-CTA path."""
import numpy as np
import pytest
import torch

import oracle
from paper_2002_04894_gb300 import inputs

pytestmark = pytest.mark.gpu


def ties(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 5, size=(n, 3)).astype(float) - 2.0
    x[::3] *= -1.0                                          # -0.0 entries
    return x


CASES = [
    ("uniform", 20000, 8), ("uniform", 20000, 4), ("plummer", 30001, 10), ("gmm", 9000, 9),
    ("uniform", 300, 10), ("uniform", 1, 3), ("uniform", 2, 1), ("uniform", 5, 0),
    ("ties", 50000, 7), ("ties", 700, 6), ("shell", 5000, 8), ("helix", 4097, 5),
]


def make(kind, n):
    return ties(n, n) if kind == "ties" else inputs.points(kind, n, seed=n)


@pytest.mark.parametrize("kind,n,levels", CASES)
@pytest.mark.parametrize("dev_input", [True, False])
def test_tree_bit_exact(gpu_lib, kind, n, levels, dev_input):
    fmm = gpu_lib
    x = make(kind, n)
    pts = torch.from_numpy(x).cuda() if dev_input else x
    plan = fmm.fmm_plan(pts, levels, 3, 0.5)
    g = fmm.fmm_plan_tree(plan)
    o = oracle.Tree(x, levels, 3, 0.5).tree()
    np.testing.assert_array_equal(g["perm"], o["perm"])
    np.testing.assert_array_equal(g["begin"], o["begin"])
    np.testing.assert_array_equal(g["count"], o["count"])
    for k in ("lo", "hi", "centre", "radius", "axis"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    internal = (1 << levels) - 1
    np.testing.assert_array_equal(g["plane"][:internal], o["plane"][:internal])


@pytest.mark.parametrize("kind,n,levels", CASES)
@pytest.mark.parametrize("theta", [0.5, 0.0, 0.35, 0.75])
def test_lists_bit_exact(gpu_lib, kind, n, levels, theta):
    fmm = gpu_lib
    x = make(kind, n)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), levels, 3, theta)
    T = oracle.Tree(x, levels, 3, theta)
    for l in range(levels + 1):
        for kind_ in ("weak", "strong"):
            gp, gs = fmm.fmm_plan_list(plan, l, kind_)
            op, os_ = T.lists(l, kind_)
            np.testing.assert_array_equal(gp, op, err_msg=f"{kind_} ptr level {l}")
            np.testing.assert_array_equal(gs, os_, err_msg=f"{kind_} src level {l}")
    st = fmm.fmm_plan_stats(plan)
    t = T.tree()
    sp, ss = T.lists(levels, "strong")
    off = (1 << levels) - 1
    work = sum(t["count"][off + a] * t["count"][off + b]
               for a in range(1 << levels) for b in ss[sp[a]:sp[a + 1]])
    assert st["p2p_interactions"] == work
    assert st["weak_pairs"] == sum(len(T.lists(l, "weak")[1]) for l in range(levels + 1))


def test_float32_points_build_the_same_tree_as_their_float64_image(gpu_lib):
    fmm = gpu_lib
    x32 = inputs.points("gmm", 12000, 4).astype(np.float32)
    plan = fmm.fmm_plan(torch.from_numpy(x32).cuda(), 9, 3, 0.5)
    g = fmm.fmm_plan_tree(plan)
    o = oracle.Tree(x32.astype(np.float64), 9, 3, 0.5).tree()
    np.testing.assert_array_equal(g["perm"], o["perm"])
    np.testing.assert_array_equal(g["lo"], o["lo"])


def test_nonfinite_points_rejected(gpu_lib):
    fmm = gpu_lib
    x = inputs.points("uniform", 1000, 1)
    x[517, 1] = np.nan
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_plan(torch.from_numpy(x).cuda(), 5, 3, 0.5)
    assert e.value.status == -3
    x[517, 1] = np.inf
    with pytest.raises(fmm.FmmError):
        fmm.fmm_plan(x, 5, 3, 0.5)
    # the context is still usable afterwards
    plan = fmm.fmm_plan(torch.from_numpy(inputs.points("uniform", 100, 1)).cuda(), 3, 3, 0.5)
    assert fmm.fmm_plan_stats(plan)["n"] == 100


@pytest.mark.parametrize("kind,n,levels", [("plummer", 30001, 10), ("gmm", 9000, 9)])
def test_gpu_lists_are_symmetric(gpu_lib, kind, n, levels):
    fmm = gpu_lib
    x = make(kind, n)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), levels, 3, 0.5)
    for l in range(levels + 1):
        for kind_ in ("weak", "strong"):
            p, s = fmm.fmm_plan_list(plan, l, kind_)
            a = np.repeat(np.arange(len(p) - 1), np.diff(p))
            fwd = set(zip(a.tolist(), s.tolist()))
            assert fwd == {(b, c) for c, b in fwd}
