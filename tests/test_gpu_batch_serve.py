"""Batched graph evaluation and the continuous-batching server on the GPU:
every result equals the same solve done alone. The only difference allowed
is the order of the double-precision atomic additions in M2L/M2M: 1e-12
relative in the FP64 form; in the mixed form a last-bit change of a double
local coefficient can flip the rounding of its float copy in L2P, so 1e-6."""
import numpy as np
import pytest
import torch

from paper_2002_04894_gb300 import inputs, serve, tune

pytestmark = pytest.mark.gpu
TOL = {0: 1e-12, 1: 1e-6}


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


SYSTEMS = [("uniform", 3000), ("plummer", 12000), ("gmm", 800), ("uniform", 45000),
           ("plummer", 1500), ("shell", 7000), ("helix", 20000), ("uniform", 64)]


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_graph_equals_individual_evals(gpu_lib, prec):
    fmm = gpu_lib
    plans, qs, pots, flds, alone = [], [], [], [], []
    for i, (kind, n) in enumerate(SYSTEMS):
        x = torch.from_numpy(inputs.points(kind, n, seed=i)).cuda()
        q = torch.from_numpy(inputs.charges_uniform(n, seed=i)).cuda()
        plan = fmm.fmm_plan(x, serve.default_levels(n), 8, 0.5, prec=prec)
        a, b = fmm.fmm_eval(plan, q)
        alone.append((a.cpu().numpy(), b.cpu().numpy()))
        plans.append(plan)
        qs.append(q)
        pots.append(torch.zeros(n, dtype=torch.float64, device="cuda"))
        flds.append(torch.zeros((n, 3), dtype=torch.float64, device="cuda"))
    batch = fmm.fmm_batch_create(plans, qs, pots, flds, nstreams=4)
    info = fmm.fmm_batch_info(batch)
    # mixed precision, one order: every system in one launch per stage
    assert info["fused"] == (prec == 1)
    if prec == 1:
        assert info["kernels"] <= 9
    else:
        assert info["kernels"] >= len(SYSTEMS)
    for rep in range(2):                                   # replay: same graph, same buffers
        for p_ in pots:
            p_.zero_()
        fmm.fmm_batch_launch(batch)
        torch.cuda.synchronize()
        for (a, b), p_, f_ in zip(alone, pots, flds):
            assert rel(p_.cpu().numpy(), a) <= TOL[prec]
            assert rel(f_.cpu().numpy(), b) <= TOL[prec]
    # new charges in the same buffers are picked up by the next launch
    qs[1].mul_(-2.0)
    fmm.fmm_batch_launch(batch)
    torch.cuda.synchronize()
    assert rel(pots[1].cpu().numpy(), -2.0 * alone[1][0]) <= TOL[prec]
    fmm.fmm_batch_destroy(batch)


# (kind, n, levels, tight, p): leaves of ~6 to ~25000 points (both near-field
# tile sizes), a single leaf, strong lists long enough to be cut into
# segments, six orders (the order-dependent stages run once per order)
HETERO = [("uniform", 64, 0, False, 8), ("plummer", 5000, 10, False, 12), ("gmm", 300000, 13, True, 10),
          ("uniform", 20000, 5, False, 6), ("helix", 9000, 8, True, 14), ("shell", 2500, 9, False, 16),
          ("plummer", 70000, 9, False, 10), ("uniform", 200000, 3, False, 4)]


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_batched_stages_equal_individual_evals(gpu_lib, dt):
    fmm = gpu_lib
    tt = torch.float64 if dt == np.float64 else torch.float32
    plans, qs, pots, flds, alone = [], [], [], [], []
    tiles, parts = set(), 0
    for i, (kind, n, B, tight, p) in enumerate(HETERO):
        x = torch.from_numpy(inputs.points(kind, n, seed=20 + i).astype(dt)).cuda()
        q = torch.from_numpy(inputs.charges_uniform(n, seed=20 + i).astype(dt)).cuda()
        plan = fmm.fmm_plan(x, B, p, 0.5, prec=1, tight=tight)
        st = fmm.fmm_plan_stats(plan)
        parts += st["p2p_partial_slots"]
        tiles.add(n <= 64 * (1 << B))
        a, b = fmm.fmm_eval(plan, q)
        alone.append((a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)))
        plans.append(plan)
        qs.append(q)
        pots.append(torch.zeros(n, dtype=tt, device="cuda"))
        flds.append(torch.zeros((n, 3), dtype=tt, device="cuda") if i % 3 != 2 else None)
    assert parts > 0 and tiles == {True, False}  # the cases the batched kernels branch on
    batch = fmm.fmm_batch_create(plans, qs, pots, flds)
    info = fmm.fmm_batch_info(batch)
    orders = len({h[4] for h in HETERO})
    assert info["fused"] and info["kernels"] <= 6 + 3 * orders
    tol = 1e-6 if dt == np.float64 else 1e-5
    for rep in range(2):
        for p_ in pots:
            p_.zero_()
        fmm.fmm_batch_launch(batch)
        torch.cuda.synchronize()
        for i, ((a, b), p_, f_) in enumerate(zip(alone, pots, flds)):
            assert rel(p_.cpu().numpy().astype(np.float64), a) <= tol, (i, rep)
            if f_ is not None:
                assert rel(f_.cpu().numpy().astype(np.float64), b) <= tol, (i, rep)
    for plan in plans:
        fmm.fmm_eval_check(plan)
    fmm.fmm_batch_destroy(batch)


@pytest.mark.parametrize("sizes", [[(1, 0)], [(2, 1), (1, 0), (5000, 7)], [(40000, 9)]])
def test_batched_stages_small_and_single_systems(gpu_lib, sizes):
    """Batches of one system, and systems of one or two points (a single leaf,
    no weak pairs, no M2M or L2L), equal the same evaluations alone."""
    fmm = gpu_lib
    plans, qs, pots, flds, alone = [], [], [], [], []
    for i, (n, B) in enumerate(sizes):
        x = torch.from_numpy(inputs.points("plummer", n, seed=60 + i)).cuda()
        q = torch.from_numpy(inputs.charges_uniform(n, seed=60 + i)).cuda()
        plan = fmm.fmm_plan(x, B, 8, 0.5, prec=1)
        a, b = fmm.fmm_eval(plan, q)
        alone.append((a.cpu().numpy(), b.cpu().numpy()))
        plans.append(plan)
        qs.append(q)
        pots.append(torch.zeros(n, dtype=torch.float64, device="cuda"))
        flds.append(torch.zeros((n, 3), dtype=torch.float64, device="cuda"))
    batch = fmm.fmm_batch_create(plans, qs, pots, flds)
    assert fmm.fmm_batch_info(batch)["fused"]
    fmm.fmm_batch_launch(batch)
    torch.cuda.synchronize()
    for (a, b), p_, f_ in zip(alone, pots, flds):
        if np.linalg.norm(a) == 0:
            assert np.array_equal(p_.cpu().numpy(), a)
        else:
            assert rel(p_.cpu().numpy(), a) <= 1e-6
            assert rel(f_.cpu().numpy(), b) <= 1e-6
    fmm.fmm_batch_destroy(batch)


def test_batched_downward_wait_that_runs_out_reports_etimedout(gpu_lib):
    """The batched downward pass waits (bounded) on each parent as the
    single-plan pass does: a withheld box (test hook, in force when the batch
    is made) makes its children's waits run out, and fmm_eval_check reports
    FMM_ETIMEDOUT on every plan deep enough to hold that box."""
    fmm = gpu_lib
    plans, qs, pots = [], [], []
    for i, (n, B) in enumerate([(20000, 8), (3000, 4), (9000, 8)]):
        x = torch.from_numpy(inputs.points("uniform", n, seed=40 + i)).cuda()
        qs.append(torch.from_numpy(inputs.charges_uniform(n, seed=40 + i)).cuda())
        plans.append(fmm.fmm_plan(x, B, 6, 0.5, prec=1))
        pots.append(torch.zeros(n, dtype=torch.float64, device="cuda"))
    withheld = (1 << 7) - 1            # first box of level 7
    fmm.fmm_set_wait_limit(2000, withheld)
    try:
        batch = fmm.fmm_batch_create(plans, qs, pots)
    finally:
        fmm.fmm_set_wait_limit(0, -1)
    assert fmm.fmm_batch_info(batch)["fused"]
    fmm.fmm_batch_launch(batch)
    torch.cuda.synchronize()
    for plan, deep in zip(plans, [True, False, True]):
        if deep:
            with pytest.raises(fmm.FmmError) as e:
                fmm.fmm_eval_check(plan)
            assert e.value.status == -5
        else:
            fmm.fmm_eval_check(plan)
    fmm.fmm_batch_destroy(batch)


def test_server_mix_equals_alone(gpu_lib):
    fmm = gpu_lib
    reqs = []
    for i, (kind, n) in enumerate(SYSTEMS * 2):
        x = inputs.points(kind, n, seed=100 + i)
        q = inputs.charges_uniform(n, seed=100 + i)
        reqs.append(serve.Request(i, x, q, arrival=0.002 * i, p=8 + 2 * (i % 2), prec=i % 2))
    alone = []
    for r in reqs:
        plan = fmm.fmm_plan(r.points, serve.default_levels(len(r.charges)), r.p, r.theta,
                            prec=r.prec, allocator=None)
        a, b = fmm.fmm_eval(plan, r.charges)
        alone.append((a, b, fmm.fmm_plan_tree(plan)["perm"]))
    srv = serve.FmmServer(budget=1 << 30, workers=4)
    res, adm = srv.run(reqs, realtime=True)
    assert adm.in_use == 0
    for r, (a, b, perm) in zip(res, alone):
        tol = TOL[reqs[r.rid].prec]
        assert rel(r.potentials, a) <= tol, r.rid
        assert rel(r.fields, b) <= tol, r.rid
        assert r.done >= r.admitted >= r.arrival - 1e-3
    st = serve.latency_stats(res)
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_server_tight_budget_serialises_but_completes(gpu_lib):
    reqs = [serve.Request(i, inputs.points("plummer", 20000, i), inputs.charges_uniform(20000, i),
                          arrival=0.0, p=8) for i in range(5)]
    need = serve.plan_bytes(20000, serve.default_levels(20000), 8)
    srv = serve.FmmServer(budget=need + 1, workers=4)
    res, adm = srv.run(reqs, realtime=False)
    assert len(res) == 5 and adm.peak <= need + 1


@pytest.mark.parametrize("batch", [0, 8])
def test_tuner_meets_target(gpu_lib, batch):
    x = torch.from_numpy(inputs.points("plummer", 60000, 3)).cuda()
    q = torch.from_numpy(inputs.charges_uniform(60000, 3)).cuda()
    r = tune.tune(x, q, tol=1e-5, ps=(6, 8, 10, 12), batch=batch)
    assert r.error <= 1e-5
    assert 32 <= 60000 / 2 ** r.config.levels <= 256
    assert r.config.theta in (0.4, 0.5, 0.6)


def test_server_resident_plans_equal_fresh_solves(gpu_lib):
    """Requests naming their point set (geom) reuse a resident plan with new
    charges: each result equals a fresh solve of the same points and charges,
    later requests of a point set are served resident, and a plan is never
    used by two requests at once (same key arriving together)."""
    fmm = gpu_lib
    geoms = {g: inputs.points(kind, n, seed=200 + g)
             for g, (kind, n) in enumerate([("plummer", 12000), ("uniform", 3000), ("gmm", 20000)])}
    reqs = []
    for i in range(12):
        g = i % 3
        x = geoms[g]
        q = inputs.charges_uniform(len(x), seed=300 + i)
        reqs.append(serve.Request(i, x, q, arrival=0.0 if i < 6 else 0.05 * i, p=8, prec=1, geom=("set", g)))
    srv = serve.FmmServer(budget=1 << 31, workers=4, cache_bytes=1 << 30)
    res, adm = srv.run(reqs, realtime=True)
    assert srv.hits >= 3 and sum(r.resident for r in res) == srv.hits
    for r in res:
        q = reqs[r.rid]
        plan = fmm.fmm_plan(q.points, serve.default_levels(len(q.charges)), q.p, q.theta, prec=1, allocator=None)
        a, b = fmm.fmm_eval(plan, q.charges)
        assert rel(r.potentials, a) <= TOL[1], r.rid
        assert rel(r.fields, b) <= TOL[1], r.rid
    srv.close()
