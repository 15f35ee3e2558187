"""Failure paths of fmm_plan, driven from the host (no GPU fault is made):

  - an allocator that returns NULL on its k-th call, for every k up to the
    number of calls a successful plan makes: fmm_plan returns FMM_ENOMEM,
    hands back no plan, and frees every byte it was given (the callback's
    running balance returns to zero);
  - a connectivity level whose candidate pairs exceed the list capacity
    (lowered through fmm_set_list_capacity): FMM_ECAPACITY, nothing leaked;
  - device-side consistency and non-finite checks keep their own codes.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2002_04894_gb300 import inputs

pytestmark = pytest.mark.gpu


class CountingAllocator:
    """Torch caching-allocator memory, failing on call `fail_at` (1-based;
    0 = never); tracks outstanding bytes and calls."""

    def __init__(self, fmm, fail_at=0):
        self.fail_at, self.calls, self.live = fail_at, 0, {}
        dev = torch.cuda.current_device()

        def alloc(nbytes, ctx, stream):
            self.calls += 1
            if self.fail_at and self.calls == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
            self.live[p] = int(nbytes)
            return p

        def free(ptr, nbytes, ctx, stream):
            assert self.live.pop(ptr) == int(nbytes)
            torch.cuda.caching_allocator_delete(ptr)

        self._cb = (fmm.ALLOC_FN(alloc), fmm.FREE_FN(free))
        self.struct = fmm.fmm_allocator(self._cb[0], self._cb[1], None)

    @property
    def balance(self):
        return sum(self.live.values())


def _plan(fmm, x, alloc, levels=8, p=6, prec=1):
    lib = fmm.load()
    opts = fmm.fmm_opts(levels, p, 0.5, prec, 0, 1.0, 1)
    h = C.c_void_p()
    st = fmm.fmm_plan_raw(lib, x.data_ptr(), x.shape[0], 0, opts, alloc.struct,
                          torch.cuda.current_stream().cuda_stream, h)
    return st, h


@pytest.mark.parametrize("prec", [0, 1])
def test_enomem_at_every_allocator_call_leaks_nothing(gpu_lib, prec):
    fmm = gpu_lib
    x = torch.from_numpy(inputs.points("plummer", 20000, 1)).cuda()
    ok = CountingAllocator(fmm)
    st, h = _plan(fmm, x, ok, prec=prec)
    assert st == 0
    ncalls = ok.calls
    assert ncalls >= 2
    fmm.load().fmm_destroy(h)
    assert ok.balance == 0
    for k in range(1, ncalls + 1):
        a = CountingAllocator(fmm, fail_at=k)
        st, h = _plan(fmm, x, a, prec=prec)
        assert st == -2, (k, st)           # FMM_ENOMEM
        assert not h.value
        assert a.balance == 0, (k, a.live)


def test_ecapacity_from_an_injected_limit(gpu_lib):
    fmm = gpu_lib
    x = torch.from_numpy(inputs.points("uniform", 20000, 2)).cuda()
    prev = fmm.fmm_set_list_capacity(100)
    try:
        a = CountingAllocator(fmm)
        st, h = _plan(fmm, x, a)
        assert st == -4                    # FMM_ECAPACITY
        assert not h.value and a.balance == 0
    finally:
        fmm.fmm_set_list_capacity(prev)
    # the default is back: the same plan now builds
    b = CountingAllocator(fmm)
    st, h = _plan(fmm, x, b)
    assert st == 0
    fmm.load().fmm_destroy(h)
    assert b.balance == 0


def test_capacity_hook_range(gpu_lib):
    fmm = gpu_lib
    prev = fmm.fmm_set_list_capacity(0)      # out of range: default
    assert fmm.fmm_set_list_capacity(prev) == 0x7fffffff


def test_nonfinite_point_is_reported_and_nothing_leaks(gpu_lib):
    fmm = gpu_lib
    xn = inputs.points("uniform", 5000, 3)
    xn[1234, 1] = np.inf
    a = CountingAllocator(fmm)
    st, h = _plan(fmm, torch.from_numpy(xn).cuda(), a)
    assert st == -3 and not h.value and a.balance == 0


def test_downward_wait_that_runs_out_reports_etimedout(gpu_lib):
    """The one-launch downward pass waits (bounded) for each parent's local
    expansion. A box whose completion is withheld (test hook) makes its
    children's waits run out: the evaluation ends, and fmm_eval_check
    reports FMM_ETIMEDOUT. With the limit restored a new plan evaluates as
    before."""
    fmm = gpu_lib
    x = torch.from_numpy(inputs.points("uniform", 20000, 4)).cuda()
    q = torch.from_numpy(inputs.charges_uniform(20000, 4)).cuda()
    B = 8
    good, _ = fmm.fmm_eval(fmm.fmm_plan(x, B, 6, 0.5), q)
    plan = fmm.fmm_plan(x, B, 6, 0.5)
    withheld = (1 << (B - 1)) - 1          # first box of the level above the leaves
    prev = fmm.fmm_set_wait_limit(2000, withheld)
    try:
        fmm.fmm_eval(plan, q)
        with pytest.raises(fmm.FmmError) as e:
            fmm.fmm_eval_check(plan)
        assert e.value.status == -5        # FMM_ETIMEDOUT
    finally:
        fmm.fmm_set_wait_limit(0, -1)
    assert prev > 0
    plan2 = fmm.fmm_plan(x, B, 6, 0.5)
    again, _ = fmm.fmm_eval(plan2, q)
    fmm.fmm_eval_check(plan2)
    assert (torch.linalg.norm(again - good) / torch.linalg.norm(good)).item() <= 1e-13
