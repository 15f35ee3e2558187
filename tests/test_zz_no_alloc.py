"""The allocation-free entry point, fmm_orb_order_noalloc, against fmm_plan.

Some callers cannot allocate device memory: plug-ins whose host application
owns all device memory, real-time loops. For them the library offers the balanced tree's leaf
order for up to 4096 points with all scratch in a static device array. These
tests call it through the C ABI twice in a row and compare each result, bit
for bit, with the permutation that fmm_plan + fmm_plan_tree report for the
same points. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2002_04894_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [("uniform", 4096, 12), ("plummer", 3000, 7), ("gmm", 1000, 9), ("uniform", 1, 3),
         ("uniform", 2, 1), ("shell", 777, 0), ("uniform", 300, 10)]


@pytest.mark.parametrize("kind,n,levels", CASES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_noalloc_order_matches_plan_twice(gpu_lib, kind, n, levels, dtype):
    fmm = gpu_lib
    lib = fmm.load()
    x = inputs.points(kind, n, seed=n + levels).astype(dtype)
    xd = torch.from_numpy(x).cuda()
    want = fmm.fmm_plan_tree(fmm.fmm_plan(xd, levels, 2, 0.5))["perm"]
    code = 0 if dtype == np.float64 else 1
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        st = lib.fmm_orb_order_noalloc(xd.data_ptr(), n, code, levels, perm.data_ptr(), stream)
        assert st == 0, fmm.fmm_strerror(st)
        np.testing.assert_array_equal(perm.cpu().numpy().astype(np.int64), want)


def test_noalloc_rejects_out_of_range_and_host_pointers(gpu_lib):
    fmm = gpu_lib
    lib = fmm.load()
    big = torch.zeros((fmm.FMM_NOALLOC_MAX_POINTS + 1, 3), dtype=torch.float64, device="cuda")
    perm = torch.empty(fmm.FMM_NOALLOC_MAX_POINTS + 1, dtype=torch.int32, device="cuda")
    assert lib.fmm_orb_order_noalloc(big.data_ptr(), big.shape[0], 0, 4, perm.data_ptr(), None) == -1
    small = big[:10].contiguous()
    assert lib.fmm_orb_order_noalloc(small.data_ptr(), 10, 0, fmm.FMM_NOALLOC_MAX_LEVELS + 1,
                                     perm.data_ptr(), None) == -1
    host = np.zeros((10, 3))
    assert lib.fmm_orb_order_noalloc(host.ctypes.data, 10, 0, 2, perm.data_ptr(), None) == -1
    # a rejected call leaves the next valid call unaffected
    x = torch.from_numpy(inputs.points("uniform", 100, 5)).cuda()
    p = fmm.fmm_orb_order_noalloc(x, 4)
    want = fmm.fmm_plan_tree(fmm.fmm_plan(x, 4, 2, 0.5))["perm"]
    np.testing.assert_array_equal(p.cpu().numpy().astype(np.int64), want)


def test_noalloc_reports_nonfinite_points(gpu_lib):
    fmm = gpu_lib
    x = inputs.points("uniform", 64, 1)
    x[5, 2] = np.nan
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_orb_order_noalloc(torch.from_numpy(x).cuda(), 3)
    assert e.value.status == -3
    x[5, 2] = 0.5                       # the shared scratch is re-cleared by the next call
    p = fmm.fmm_orb_order_noalloc(torch.from_numpy(x).cuda(), 3)
    assert sorted(p.cpu().numpy().tolist()) == list(range(64))
