"""Parameter autotuner for the balanced-tree FMM.

The paper reports that run time responds convexly to the number of levels L
and to theta when each is varied alone (Sec. 3.2, Table 3.1), suggests a
leaf size of 50-200 points, and bounds the relative error by
C theta^(p+1) / (1 - theta)^2 (Sec. 3.1). The tuner uses all three:

  1. seed: levels for ~100 points per leaf, theta = 0.5, and the smallest
     expansion order p whose bound (C = 1) is below the target error;
  2. coordinate descent on levels, then theta: step in the improving
     direction while the measured time falls (convexity makes the first
     local minimum along a coordinate the minimum on it);
  3. for the chosen (levels, theta), the smallest p among the allowed ones
     whose *measured* error on sampled targets meets the target.

The search logic (`descend`) is independent of the GPU: it takes any cost
function, so it can be exercised on the CPU. `tune` supplies the GPU cost:
one plan + evaluation timed with CUDA events, and the error against the FP64
direct sum on sampled targets. For systems that are evaluated many at a time
(`batch` > 0) the cost is instead the evaluation time per system of a batch
of copies of the system in one launch per stage: alone, a small system's
solve is dominated by per-launch latency, which pushes the search towards
few levels and heavy near fields; in a batch that latency is shared, and the
arithmetic is what counts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field


@dataclass(frozen=True)
class Config:
    levels: int
    p: int
    theta: float


@dataclass
class TuneResult:
    config: Config
    ms: float
    error: float
    trials: list = field(default_factory=list)


def p_from_bound(tol: float, theta: float, allowed=(6, 8, 10, 12, 14, 16)) -> int:
    """Smallest allowed p with theta^(p+1) / (1 - theta)^2 <= tol."""
    need = math.ceil(math.log(tol * (1.0 - theta) ** 2) / math.log(theta)) - 1
    for p in allowed:
        if p >= need:
            return p
    return allowed[-1]


def pick(trials, tol: float):
    """The fastest (config, ms, error) trial whose error meets `tol`; when
    none does, the most accurate one."""
    ok = [t for t in trials if t[2] <= tol]
    return min(ok, key=lambda t: t[1]) if ok else min(trials, key=lambda t: t[2])


def levels_for_leaf(n: int, leaf: float) -> int:
    return max(0, int(round(math.log2(max(n, 1) / leaf))))


def descend(cost, start: int, lo: int, hi: int, step: int = 1):
    """Minimise cost(x) over integers in [lo, hi] from `start`, assuming a
    convex (unimodal) response: probe both neighbours, walk downhill."""
    memo = {}

    def f(x):
        if x not in memo:
            memo[x] = cost(x)
        return memo[x]

    x = min(max(start, lo), hi)
    best = f(x)
    for d in (step, -step):
        moved = False
        while lo <= x + d <= hi and f(x + d) < best:
            x += d
            best = f(x)
            moved = True
        if moved:
            break
    return x, best, memo


def batch_copies(n: int, points: int = 1_000_000, cap: int = 128) -> int:
    """Copies of an n-point system that make a batch of about `points`."""
    return max(1, min(cap, points // max(n, 1)))


def tune(points, charges, tol: float = 1e-6, leaf_range=(32, 256), thetas=(0.4, 0.5, 0.6),
         ps=(6, 8, 10, 12, 14, 16), prec=None, targets: int = 300, seed: int = 0, batch: int = 0) -> TuneResult:
    """Search (levels, theta, p) for the fastest solve meeting `tol` (relative
    L2 potential error against the FP64 direct sum on sampled targets).
    batch > 0: the cost is the evaluation time per system in a batch of
    `batch` copies (one launch per stage)."""
    import numpy as np
    import torch

    from . import (FMM_PREC_MIXED, fmm_batch_create, fmm_batch_destroy, fmm_batch_launch, fmm_destroy,
                   fmm_direct, fmm_eval, fmm_plan)
    from . import inputs as _inputs

    prec = FMM_PREC_MIXED if prec is None else prec
    n = int(points.shape[0])
    xd = points if points.is_cuda else points.cuda()
    qd = charges if charges.is_cuda else charges.cuda()
    tgt = torch.from_numpy(_inputs.sample_targets(n, targets, seed)).cuda()
    ref = fmm_direct(xd, qd, tgt)[0].double().cpu().numpy()
    trials = []

    def run_batch(cfg: Config):
        from .serve import build_plans
        plans = build_plans([xd] * batch, [cfg] * batch, prec=prec)
        pots = [torch.empty(n, dtype=qd.dtype, device=qd.device) for _ in range(batch)]
        b = fmm_batch_create(plans, [qd] * batch, pots)
        times = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fmm_batch_launch(b)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / batch)
        fmm_batch_destroy(b)
        for pl in plans:
            fmm_destroy(pl)
        got = pots[0].double().cpu().numpy()[tgt.cpu().numpy()]
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        trials.append((cfg, min(times), err))
        return min(times), err

    def run(cfg: Config):
        if batch > 0:
            return run_batch(cfg)
        times = []
        for _ in range(2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            plan = fmm_plan(xd, cfg.levels, cfg.p, cfg.theta, prec=prec)
            pot, _ = fmm_eval(plan, qd, want_fields=False)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
            fmm_destroy(plan)
        got = pot.double().cpu().numpy()[tgt.cpu().numpy()]
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        trials.append((cfg, min(times), err))
        return min(times), err

    lmin = levels_for_leaf(n, leaf_range[1])
    lmax = max(lmin, levels_for_leaf(n, leaf_range[0]))
    theta = 0.5
    p = p_from_bound(tol, theta, ps)
    lev, _, _ = descend(lambda L: run(Config(L, p, theta))[0], levels_for_leaf(n, 100), lmin, lmax)
    ti, _, _ = descend(lambda i: run(Config(lev, p, thetas[i]))[0], list(thetas).index(0.5)
                       if 0.5 in thetas else 0, 0, len(thetas) - 1)
    theta = thetas[ti]
    for pp in ps:  # smallest p meeting the target at (lev, theta)
        if run(Config(lev, pp, theta))[1] <= tol:
            break
    # the levels and theta were searched by time alone (a faster theta may
    # miss the target at every allowed p): the fastest trial that meets it
    cfg, ms, err = pick(trials, tol)
    best = TuneResult(cfg, ms, err)
    best.trials = trials
    return best
