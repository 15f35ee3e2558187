"""M2L on the tensor cores (FMM_FLAG_TC_M2L, mixed form, p <= 12; Sec. 2.1.3
rotation form as tcgen05 TF32 products, three per contraction) against the
FP64 oracle and against the default single-precision CUDA-core kernel on the
same plan.

Tolerances: the local expansions and results within 1e-5 of the oracle's
FMM (as for the whole mixed form); tensor-core vs CUDA-core locals within
2e-6 of their scale: both are single-precision evaluations of the same
products, ~3e-7 per product for the split TF32 against 6e-8 for FP32,
grown by the five chained contractions."""
import numpy as np
import pytest
import torch

import oracle
from paper_2002_04894_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


CASES = [
    # kind, n, levels, p, theta
    ("plummer", 12000, 8, 12, 0.5),
    ("uniform", 20000, 8, 8, 0.5),
    ("gmm", 9000, 9, 10, 0.6),
    ("plummer", 6000, 9, 5, 0.5),     # odd p: tensor-core kernel only
    ("uniform", 2000, 8, 1, 0.4),
    ("uniform", 700, 5, 12, 0.7),     # 306 pairs: three tiles, ragged tail
    ("shell", 4000, 9, 11, 0.5),
]


@pytest.mark.parametrize("kind,n,levels,p,theta", CASES)
def test_tc_m2l_matches_oracle(gpu_lib, kind, n, levels, p, theta):
    fmm = gpu_lib
    x = inputs.points(kind, n, seed=31)
    q = inputs.charges_uniform(n, seed=31)
    plan = fmm.fmm_plan(torch.from_numpy(x).cuda(), levels, p, theta, prec=fmm.FMM_PREC_MIXED, tc_m2l=True)
    pot, fld = fmm.fmm_eval(plan, torch.from_numpy(q).cuda())
    fmm.fmm_eval_check(plan)
    T = oracle.Tree(x, levels, p, theta)
    op, oE = T.eval(q)
    gL, oL = fmm.fmm_eval_expansions(plan, "L"), T.expansions("L")
    assert fmm.fmm_plan_stats(plan)["weak_pairs"] > 0
    assert np.abs(gL - oL).max() <= 1e-5 * np.abs(oL).max()
    assert rel(pot.cpu().numpy(), op) <= 1e-5
    assert rel(fld.cpu().numpy(), oE) <= 1e-5


@pytest.mark.parametrize("p", [4, 6, 8, 10, 12])
def test_tc_m2l_matches_cuda_core_kernel(gpu_lib, p):
    fmm = gpu_lib
    n = 30000
    x = inputs.points("plummer", n, seed=p)
    q = inputs.charges_uniform(n, seed=p)
    xd, qd = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    a = fmm.fmm_plan(xd, 10, p, 0.5, prec=fmm.FMM_PREC_MIXED, tc_m2l=True)
    b = fmm.fmm_plan(xd, 10, p, 0.5, prec=fmm.FMM_PREC_MIXED)
    pa, _ = fmm.fmm_eval(a, qd)
    pb, _ = fmm.fmm_eval(b, qd)
    fmm.fmm_eval_check(a)
    La, Lb = fmm.fmm_eval_expansions(a, "L"), fmm.fmm_eval_expansions(b, "L")
    assert np.abs(La - Lb).max() <= 2e-6 * np.abs(Lb).max()
    assert rel(pa.cpu().numpy(), pb.cpu().numpy()) <= 2e-6


def test_tc_m2l_benchmark_accuracy(gpu_lib):
    """p = 12, theta = 0.5 on a Plummer sphere: the solve stays within the
    1e-6 target against the exact sum."""
    fmm = gpu_lib
    n = 100000
    x = inputs.points("plummer", n, seed=2)
    q = inputs.charges_uniform(n, seed=2)
    xd, qd = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    plan = fmm.fmm_plan(xd, 10, 12, 0.5, prec=fmm.FMM_PREC_MIXED, tc_m2l=True)
    pot, fld = fmm.fmm_eval(plan, qd)
    fmm.fmm_eval_check(plan)
    t = inputs.sample_targets(n, 500, 2)
    dp, dE = oracle.direct(x, q, targets=t)
    assert rel(pot.cpu().numpy()[t], dp) <= 1e-6
    assert rel(fld.cpu().numpy()[t], dE) <= 1e-6
