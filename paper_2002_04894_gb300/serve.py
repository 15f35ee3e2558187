"""Continuous-batching server for FMM solves.

Requests (points, charges, parameters) arrive over time. The server admits a
request as soon as it has arrived, a worker slot is free, and its estimated
device memory fits in what the budget has left; it never waits to fill a
batch. Each worker owns a CUDA stream, so solves admitted while others are
still running overlap on the device: host-to-device copies, tree, lists,
expansions and near field of different requests interleave. Memory is given
back when a solve completes, which admits the next requests in arrival order.
Latency is measured from arrival to the result on the host.

Resident plans. A request may name its point set (`geom`, any hashable key:
the caller promises that requests with the same key carry the same points and
parameters). The tree, lists and expansion storage of a named point set stay
on the device after its first solve, in a least-recently-used cache bounded
by `cache_bytes` of the budget; a later request with the same key and new
charges runs only the evaluation. A resident plan serves one request at a
time (a plan must not be used from two threads at once): a request that finds
its plan busy builds a transient one.

The admission policy (`Admission`) is plain Python and is unit-tested on the
CPU with a stand-in executor; `FmmServer` runs it against the CUDA library.
"""
from __future__ import annotations

import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    points: object            # host array (n x 3), float64 or float32
    charges: object           # host array (n)
    arrival: float = 0.0      # seconds after the start of the run
    levels: int = -1          # -1: chosen from the leaf-size policy
    p: int = 10
    theta: float = 0.5
    prec: int = 1             # FMM_PREC_MIXED
    fields: bool = True
    geom: object = None       # name of the point set (resident plan), or None


@dataclass
class Result:
    rid: int
    potentials: np.ndarray
    fields: np.ndarray | None
    arrival: float
    admitted: float
    done: float
    levels: int
    bytes_reserved: int
    resident: bool = False    # served by a resident plan (evaluation only)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def default_levels(n: int, leaf: float = 100.0) -> int:
    return max(0, int(round(math.log2(max(n, 1) / leaf))))


def plan_bytes(n: int, levels: int, p: int, mixed: bool = True) -> int:
    """Upper estimate of a plan's device memory while it is built and used:
    points, boxes, lists and expansions (persistent) plus the build's
    temporaries, plus the caller's input and output copies."""
    nbox = (2 << levels) - 1
    nleaf = 1 << levels
    nc = (p + 1) * (p + 2) // 2
    persist = n * (96 + (60 if mixed else 0)) + nbox * (128 + 32 * nc + (24 * nc if mixed else 0))
    lists = nleaf * 3000
    scratch = n * 40 + nbox * 64 + nleaf * 2000
    io = n * 8 * 8
    return int(1.25 * (persist + lists + scratch + io)) + (4 << 20)


class Admission:
    """Arrival-ordered admission under a memory budget and a slot limit.
    A request larger than the whole budget is admitted alone (when nothing
    else is in flight), so it cannot starve."""

    def __init__(self, budget: int, slots: int):
        self.budget, self.slots = int(budget), int(slots)
        self.in_use = 0
        self.active = 0
        self.peak = 0

    def can_admit(self, need: int) -> bool:
        if self.active >= self.slots:
            return False
        return self.in_use + need <= self.budget or self.active == 0

    def admit(self, need: int) -> None:
        self.in_use += need
        self.active += 1
        self.peak = max(self.peak, self.in_use)

    def release(self, need: int) -> None:
        self.in_use -= need
        self.active -= 1


def eval_bytes(n: int) -> int:
    """Device memory of one evaluation on a resident plan: the request's input
    and output copies."""
    return n * 8 * 8 + (1 << 20)


def run_schedule(requests, execute, budget: int, slots: int, realtime: bool = True, clock=time.perf_counter,
                 need_of=None):
    """Admit requests in arrival order as slots and memory free up; `execute`
    (request, t0) -> Result runs on a worker thread; `need_of(request)` gives
    the bytes to reserve (default: a whole plan, plan_bytes). Returns results
    in request order and the admission record."""
    adm = Admission(budget, slots)
    pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
    results = {}
    cv = threading.Condition()
    t0 = clock()
    threads = []
    errors = []

    def worker(req, need, admitted):
        try:
            res = execute(req, t0)
            res.admitted = admitted
            res.bytes_reserved = need
            with cv:
                results[req.rid] = res
        except BaseException as e:  # reported after the run
            errors.append(e)
        finally:
            with cv:
                adm.release(need)
                cv.notify_all()

    i = 0
    while i < len(pending):
        req = pending[i]
        if need_of is not None:
            need = need_of(req)
        else:
            lv = req.levels if req.levels >= 0 else default_levels(len(req.charges))
            need = plan_bytes(len(req.charges), lv, req.p, req.prec == 1)
        with cv:
            while True:
                now = clock() - t0
                if realtime and now < req.arrival:
                    cv.wait(timeout=req.arrival - now)
                    continue
                if adm.can_admit(need):
                    adm.admit(need)
                    break
                cv.wait(timeout=0.05)
        th = threading.Thread(target=worker, args=(req, need, clock() - t0), daemon=True)
        th.start()
        threads.append(th)
        i += 1
    for th in threads:
        th.join()
    if errors:
        raise errors[0]
    return [results[r.rid] for r in requests], adm


class FmmServer:
    """Runs requests through the CUDA library with `workers` concurrent
    solves, each on its own stream, under a device memory budget (bytes), of
    which `cache_bytes` may hold resident plans of named point sets."""

    def __init__(self, budget: int, workers: int = 8, cache_bytes: int = 0):
        import torch

        from . import load
        load()
        self.budget, self.workers = int(budget), int(workers)
        self.cache_bytes = int(min(cache_bytes, budget))
        self._streams = [torch.cuda.Stream() for _ in range(self.workers)]
        self._free = list(range(self.workers))
        self._lock = threading.Lock()
        self._cache = {}      # key -> [plan, bytes, last use, busy]
        self._cached = 0
        self._tick = 0
        self.hits = 0
        self._claims = {}     # rid -> resident plan claimed at admission

    @staticmethod
    def _key(req: Request):
        lv = req.levels if req.levels >= 0 else default_levels(len(req.charges))
        return (req.geom, lv, req.p, req.theta, req.prec)

    def _need(self, req: Request) -> int:
        """Bytes to reserve at admission. An idle resident plan of the
        request's point set is claimed here (so the reservation holds: the
        evaluation's copies only); otherwise a whole transient plan."""
        n = len(req.charges)
        if req.geom is not None:
            with self._lock:
                e = self._cache.get(self._key(req))
                if e is not None and not e[3]:
                    e[3] = True
                    self._tick += 1
                    e[2] = self._tick
                    self.hits += 1
                    self._claims[req.rid] = e[0]
                    return eval_bytes(n)
        lv = req.levels if req.levels >= 0 else default_levels(n)
        return plan_bytes(n, lv, req.p, req.prec == 1)

    def _keep(self, key, plan, nbytes) -> bool:
        """Make `plan` resident (busy: its builder evaluates it next) if it
        fits the cache after evicting idle least-recently-used plans; returns
        False if it does not."""
        from . import fmm_destroy
        if nbytes > self.cache_bytes:
            return False
        with self._lock:
            if key in self._cache:
                return False
            while self._cached + nbytes > self.cache_bytes:
                idle = [(v[2], k) for k, v in self._cache.items() if not v[3]]
                if not idle:
                    return False
                _, k = min(idle)
                fmm_destroy(self._cache.pop(k)[0])
                self._cached = sum(v[1] for v in self._cache.values())
            self._tick += 1
            self._cache[key] = [plan, nbytes, self._tick, True]  # busy: the caller evaluates it now
            self._cached += nbytes
            return True

    def _release(self, key):
        with self._lock:
            if key in self._cache:
                self._cache[key][3] = False

    def _execute(self, req: Request, t0: float) -> Result:
        import torch

        from . import fmm_destroy, fmm_eval, fmm_plan
        with self._lock:
            k = self._free.pop()
        try:
            s = self._streams[k]
            n = len(req.charges)
            lv = req.levels if req.levels >= 0 else default_levels(n)
            # host arrays straight to the library, which stages them through
            # device buffers on the worker's stream (no per-request pinned
            # allocation, which would serialise the workers)
            xh = np.ascontiguousarray(req.points)
            qh = np.ascontiguousarray(req.charges, dtype=xh.dtype)
            ph = np.empty(n, dtype=xh.dtype)
            fh = np.empty((n, 3), dtype=xh.dtype) if req.fields else None
            key = self._key(req) if req.geom is not None else None
            with self._lock:
                plan = self._claims.pop(req.rid, None)
            resident = plan is not None
            with torch.cuda.stream(s):
                if plan is None:
                    plan = fmm_plan(xh, lv, req.p, req.theta, prec=req.prec, stream=s)
                    keep = key is not None and self._keep(key, plan, plan_bytes(n, lv, req.p, req.prec == 1))
                else:
                    keep = True
                try:
                    fmm_eval(plan, qh, ph, fh, stream=s)  # host outputs: returns when complete
                finally:
                    if keep:
                        self._release(key)
                    else:
                        fmm_destroy(plan)
            done = time.perf_counter() - t0
            return Result(req.rid, ph, fh, req.arrival, 0.0, done, lv, 0, resident)
        finally:
            with self._lock:
                self._free.append(k)

    def run(self, requests, realtime: bool = True):
        """Serve `requests` (arrival times relative to now). Returns
        (results in request order, admission record). Resident plans live in
        their own share of the budget (cache_bytes); transient work is
        admitted against the rest."""
        return run_schedule(requests, self._execute, self.budget - self.cache_bytes, self.workers, realtime,
                            need_of=self._need)

    def close(self):
        """Destroy the resident plans."""
        from . import fmm_destroy
        with self._lock:
            for v in self._cache.values():
                fmm_destroy(v[0])
            self._cache.clear()
            self._cached = 0


def build_plans(points, configs, prec: int = 1, workers: int = 8):
    """fmm_plan for many systems at once: `workers` host threads, each with
    its own CUDA stream, so that one plan's host-side steps (level sizes read
    back, allocations) overlap the others' device work. `configs` holds
    objects with levels, p and theta (e.g. tune.Config). Returns the plans in
    input order; their streams are synchronised before returning."""
    import concurrent.futures as cf

    import torch

    from . import fmm_plan
    streams = [torch.cuda.Stream() for _ in range(workers)]

    def one(i):
        s = streams[i % workers]
        c = configs[i]
        with torch.cuda.stream(s):
            return fmm_plan(points[i], c.levels, c.p, c.theta, prec=prec, stream=s)

    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        plans = list(ex.map(one, range(len(points))))
    for s in streams:
        s.synchronize()
    return plans


def latency_stats(results) -> dict:
    lat = np.array([r.latency for r in results])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3)}


def poisson_arrivals(count: int, rate: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: exponential gaps of mean 1/rate."""
    gaps = np.random.default_rng([seed, 3]).exponential(1.0 / rate, size=count)
    return np.cumsum(gaps)
