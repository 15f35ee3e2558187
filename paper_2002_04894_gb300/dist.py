"""One FMM system split over G = 2^g devices: the parallel structure of
Sec. 2.2 and Algorithms 2-4 of Bull & Engblom (arXiv:2002.04894), on the
binary balanced tree of this library.

Ownership. The top g levels of the global tree (the balanced median splits
of all points) hand out subtrees: rank r owns box r of level g and every box
below it, down to the leaves at level B. Level g plays the part of the
paper's local roots. Each rank builds its subtree from its own points, in
ascending original index, with that box's cell as root cell
(FMM_FLAG_ROOT_CELL): the result is the global subtree bit for bit. The boxes
of levels 0..g are known to every rank (the partition step).

Connectivity (Algorithm 2). The lists inside a subtree are the rank's own
plan's lists. Pairs of boxes of two ranks p, q form the halo H_pq: at level
g they are the top tree's pairs between boxes p and q; below, level by level,
rank p sends q the centres and radii of the children of its boxes in strong
pairs with q, receives q's, and theta-tests every child pair (weak pairs go
to M2L, strong ones are refined; at the leaves they are P2P pairs). The
theta-test is symmetric, so H_qp is the transpose of H_pq and both sides
know, without asking, what the other will send.

Exchange (Algorithms 3 and 4). For M2L, rank p sends q the multipoles of its
boxes in weak pairs with q below level g; for P2P, the points and charges of
its leaves in strong leaf pairs with q. Weak pairs at levels 0..g join boxes
that span several ranks: every rank gathers the level-g multipoles and forms
the top levels' expansions itself (the same arithmetic on every rank). Sends
and receives are point-to-point (torch.distributed isend / irecv: NCCL
between GPUs, gloo between CPU processes), into buffers of the receiver.

Arithmetic (theta-tests, expansions, interactions) is delegated to a backend
object; the library's device kernels are the backend on GPUs. This module
holds the bookkeeping only.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def heap(l: int, j) -> np.ndarray:
    """Heap index of box j of level l (box g of level l is 2^l - 1 + j)."""
    return (1 << l) - 1 + np.asarray(j, dtype=np.int64)


def owned(rank: int, g: int, l: int) -> tuple[int, int]:
    """Level-l indices [lo, hi) owned by `rank` (l >= g)."""
    return rank << (l - g), (rank + 1) << (l - g)


def owner(g: int, l: int, j) -> np.ndarray:
    """Rank owning box j of level l >= g."""
    return np.asarray(j, dtype=np.int64) >> (l - g)


@dataclass
class Partition:
    """The top g levels of the global tree: the geometry of boxes 0 ..
    2^(g+1) - 2 (heap order), the cells of the level-g boxes (the ranks'
    root cells) and each rank's points (original indices, ascending)."""
    g: int
    levels: int
    centre: np.ndarray          # (2^(g+1) - 1, 3)
    radius: np.ndarray          # (2^(g+1) - 1,)
    lo: np.ndarray              # (2^g, 3) root cells
    hi: np.ndarray
    points_of: list             # rank -> int64 original indices, ascending

    @classmethod
    def from_tree(cls, tree: dict, g: int, levels: int) -> "Partition":
        """From the tree arrays (perm, begin, count, lo, hi, centre, radius;
        as fmm_plan_tree reports them) of a plan of all points with at least
        g levels and the same geometry options as the ranks' plans."""
        nb = (2 << g) - 1
        first = (1 << g) - 1
        pts = []
        for r in range(1 << g):
            b, c = int(tree["begin"][first + r]), int(tree["count"][first + r])
            pts.append(np.sort(np.asarray(tree["perm"][b:b + c], dtype=np.int64)))
        return cls(g, levels, np.asarray(tree["centre"][:nb], np.float64), np.asarray(tree["radius"][:nb], np.float64),
                   np.asarray(tree["lo"][first:nb], np.float64), np.asarray(tree["hi"][first:nb], np.float64), pts)


@dataclass
class Halo:
    """Rank p's cross-rank pairs: for each peer q and level l (g..B), the
    weak pairs and the strong pairs (level-l indices: i owned by p, j by q).
    `remote` keeps the geometry of q's boxes that p received (level, index)
    -> (centre, radius)."""
    rank: int
    weak: dict = field(default_factory=dict)     # (q, l) -> int64 array (m, 2)
    strong: dict = field(default_factory=dict)   # (q, l) -> int64 array (m, 2)
    remote: dict = field(default_factory=dict)   # (q, l) -> (indices, centre (m, 3), radius (m,))


def top_lists(part: Partition, theta: float, backend):
    """Connectivity of levels 1..g from the top tree (the same on every
    rank): {l: (weak pairs, strong pairs)} as arrays of (a, b) level indices,
    both orientations."""
    out = {}
    strong = np.array([[0, 0]], dtype=np.int64)
    for l in range(1, part.g + 1):
        a = np.repeat(2 * strong[:, 0], 4) + np.tile([0, 0, 1, 1], len(strong))
        b = np.repeat(2 * strong[:, 1], 4) + np.tile([0, 1, 0, 1], len(strong))
        ga, gb = heap(l, a), heap(l, b)
        w = backend.theta_weak(theta, part.centre[ga], part.radius[ga], part.centre[gb], part.radius[gb])
        out[l] = (np.stack([a[w], b[w]], 1), np.stack([a[~w], b[~w]], 1))
        strong = out[l][1]
    return out


def build_halo(rank: int, world: int, part: Partition, theta: float, geo, comm, backend) -> Halo:
    """Algorithm 2 on rank `rank`: the halos with every other rank.
    geo(l) -> (centre (2^(l-g), 3), radius (2^(l-g),)) of the rank's own
    level-l boxes, local order (from its plan's tree)."""
    g, B = part.g, part.levels
    H = Halo(rank)
    top = top_lists(part, theta, backend)
    own_lo = lambda l: owned(rank, g, l)[0]
    # level g: the top tree's pairs between rank boxes
    strong = {}
    if g == 0:
        return H
    wk, st = top[g]
    for q in range(world):
        if q == rank:
            continue
        for kind, pairs in (("weak", wk), ("strong", st)):
            m = pairs[(pairs[:, 0] == rank) & (pairs[:, 1] == q)]
            getattr(H, kind)[(q, g)] = m
        strong[q] = H.strong[(q, g)]
    for l in range(g + 1, B + 1):
        centre, radius = geo(l)
        sends, specs, kids = {}, {}, {}
        for q, S in strong.items():
            if len(S) == 0:
                continue
            mine = np.unique(S[:, 0])
            theirs = np.unique(S[:, 1])
            mk = np.stack([2 * mine, 2 * mine + 1], 1).ravel()
            tk = np.stack([2 * theirs, 2 * theirs + 1], 1).ravel()
            loc = mk - own_lo(l)
            sends[q] = np.concatenate([centre[loc], radius[loc, None]], 1)
            specs[q] = (len(tk), 4)
            kids[q] = tk
        recv = comm.exchange(sends, specs)
        new_strong = {}
        for q, S in strong.items():
            if len(S) == 0:
                new_strong[q] = S
                continue
            tk = kids[q]
            rc = recv[q]
            H.remote[(q, l)] = (tk, rc[:, :3], rc[:, 3])
            a = np.repeat(2 * S[:, 0], 4) + np.tile([0, 0, 1, 1], len(S))
            b = np.repeat(2 * S[:, 1], 4) + np.tile([0, 1, 0, 1], len(S))
            ia = a - own_lo(l)
            jb = np.searchsorted(tk, b)
            w = backend.theta_weak(theta, centre[ia], radius[ia], rc[jb, :3], rc[jb, 3])
            H.weak[(q, l)] = np.stack([a[w], b[w]], 1)
            H.strong[(q, l)] = np.stack([a[~w], b[~w]], 1)
            new_strong[q] = H.strong[(q, l)]
        strong = new_strong
    return H


def m2l_sends(H: Halo, g: int, B: int, world: int) -> dict:
    """(q, l) -> sorted own level-l indices whose multipoles q needs (own
    boxes in weak pairs with q, levels below g: the top levels go by
    gathering)."""
    out = {}
    for (q, l), w in H.weak.items():
        if l > g and len(w):
            out[(q, l)] = np.unique(w[:, 0])
    return out


def m2l_recvs(H: Halo, g: int) -> dict:
    """(q, l) -> sorted level-l indices of q whose multipoles p receives."""
    out = {}
    for (q, l), w in H.weak.items():
        if l > g and len(w):
            out[(q, l)] = np.unique(w[:, 1])
    return out


def p2p_sends(H: Halo, B: int) -> dict:
    """q -> sorted own leaves (level-B indices) whose points q needs."""
    return {q: np.unique(s[:, 0]) for (q, l), s in H.strong.items() if l == B and len(s)}


def p2p_recvs(H: Halo, B: int) -> dict:
    """q -> sorted leaves of q whose points p receives."""
    return {q: np.unique(s[:, 1]) for (q, l), s in H.strong.items() if l == B and len(s)}


class TorchComm:
    """Point-to-point exchange over torch.distributed (NCCL for CUDA tensors,
    gloo for CPU tensors): every send and receive posted at once, then
    waited on. Receive buffers are allocated on `device`."""

    def __init__(self, device="cpu"):
        import torch.distributed as tdist
        self.dist = tdist
        self.rank = tdist.get_rank()
        self.world = tdist.get_world_size()
        self.device = device

    def exchange(self, sends: dict, specs: dict, dtype=None):
        """sends: peer -> array; specs: peer -> shape of what that peer sends
        here. Returns peer -> received array (numpy for numpy input)."""
        import torch
        keys = sorted(set(sends) | set(specs))
        reqs, bufs = [], {}
        for q in keys:   # ordered by peer on both sides
            if q in specs:
                dt = dtype or torch.float64
                bufs[q] = torch.empty(specs[q], dtype=dt, device=self.device)
                reqs.append(self.dist.irecv(bufs[q], src=q))
            if q in sends:
                t = sends[q]
                t = torch.as_tensor(np.ascontiguousarray(t)) if isinstance(t, np.ndarray) else t
                t = t.to(self.device).contiguous()
                reqs.append(self.dist.isend(t, dst=q))
        for r in reqs:
            r.wait()
        return {q: b.cpu().numpy() for q, b in bufs.items()}

    def all_gather(self, x: np.ndarray) -> list:
        import torch
        t = torch.as_tensor(np.ascontiguousarray(x)).to(self.device)
        out = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t)
        return [o.cpu().numpy() for o in out]


class ThreadComm:
    """Ranks as threads of one process (several plans on one device, or CPU
    tests): the same exchange and gather as TorchComm through a shared
    mailbox. Every rank calls exchange/all_gather in the same sequence."""

    class Hub:
        def __init__(self, world):
            import threading
            self.world, self.box, self.cv = world, {}, threading.Condition()

    def __init__(self, hub: "ThreadComm.Hub", rank: int, timeout: float = 120.0):
        self.hub, self.rank, self.world, self.seq, self.timeout = hub, rank, hub.world, 0, timeout

    def _take(self, key):
        with self.hub.cv:
            if not self.hub.cv.wait_for(lambda: key in self.hub.box, timeout=self.timeout):
                raise TimeoutError(f"rank {self.rank}: no message {key}")
            return self.hub.box.pop(key)

    def exchange(self, sends: dict, specs: dict, dtype=None):
        self.seq += 1
        with self.hub.cv:
            for q, a in sends.items():
                self.hub.box[(self.rank, q, self.seq)] = np.array(a, dtype=np.float64, copy=True)
            self.hub.cv.notify_all()
        out = {}
        for q, shape in specs.items():
            a = self._take((q, self.rank, self.seq))
            if a.shape != tuple(shape):
                raise ValueError(f"rank {self.rank}: from {q} got {a.shape}, expected {shape}")
            out[q] = a
        return out

    def all_gather(self, x: np.ndarray) -> list:
        sends = {q: x for q in range(self.world) if q != self.rank}
        got = self.exchange(sends, {q: np.shape(x) for q in sends})
        return [np.array(x, dtype=np.float64) if q == self.rank else got[q] for q in range(self.world)]


def evaluate(rank: int, world: int, part: Partition, H: Halo, plan, charges, theta: float, comm, backend):
    """Algorithms 3 and 4 on rank `rank`: returns the potentials and fields
    at the rank's points (the order its plan was given them)."""
    g, B = part.g, part.levels
    backend.upward(plan, charges)
    # top levels: the level-g multipoles of every rank, then the local
    # expansion their weak pairs give this rank's level-g box
    top = top_lists(part, theta, backend)
    Mg = comm.all_gather(backend.multipoles(plan, 0, np.array([0]))[0].view(np.float64))
    backend.add_local(plan, 0, np.array([0]), [backend.top_local(part, [m.view(complex) for m in Mg], rank, top)])
    # halo M2L: multipoles of the boxes in weak pairs, below level g
    sends, recvs = m2l_sends(H, g, B, world), m2l_recvs(H, g)
    out_s, in_r = {}, {}
    for (q, l), idx in sorted(sends.items()):
        out_s.setdefault(q, []).append(backend.multipoles(plan, l - g, idx - owned(rank, g, l)[0]).view(np.float64))
    for (q, l), idx in sorted(recvs.items()):
        in_r.setdefault(q, []).append((l, idx))
    nc2 = 2 * backend.nc
    got = comm.exchange({q: np.concatenate(v) for q, v in out_s.items()},
                        {q: (sum(len(i) for _, i in v), nc2) for q, v in in_r.items()})
    for q, parts_ in in_r.items():
        arr, o = got[q].view(complex), 0
        for l, idx in parts_:
            w = H.weak[(q, l)]
            rem_idx, rem_c, _ = H.remote[(q, l)]
            M = arr[o:o + len(idx)][np.searchsorted(idx, w[:, 1])]
            backend.m2l_external(plan, l - g, w[:, 0] - owned(rank, g, l)[0], M,
                                 rem_c[np.searchsorted(rem_idx, w[:, 1])])
            o += len(idx)
    # halo P2P: points and charges of the leaves in strong leaf pairs
    ps, pr = p2p_sends(H, B), p2p_recvs(H, B)
    lo = owned(rank, g, B)[0]
    mine = {q: backend.leaf_points(plan, v - lo) for q, v in ps.items()}
    cnts = comm.exchange({q: np.array([len(a) for a in v], np.float64) for q, v in mine.items()},
                         {q: (len(v),) for q, v in pr.items()})
    pts = comm.exchange({q: np.concatenate(v) for q, v in mine.items()},
                        {q: (int(cnts[q].sum()), 4) for q in pr})
    pairs, srcs = [], []
    for (q, l), s in sorted(H.strong.items()):
        if l != B or not len(s):
            continue
        offs = np.concatenate([[0], np.cumsum(cnts[q])]).astype(np.int64)
        for a, b in s:
            k = int(np.searchsorted(pr[q], b))
            pairs.append(int(a - lo))
            srcs.append(pts[q][offs[k]:offs[k + 1]])
    backend.p2p_external(plan, np.array(pairs, np.int64), srcs)
    return backend.downward(plan)


class GpuBackend:
    """The arithmetic of a split system on this rank's GPU, through the
    library's entry points (plain FP64 form): theta-tests (fmm_theta_test),
    the rank's plan (fmm_plan with its root cell), the upward pass
    (fmm_eval_upward), multipoles and leaf points out (fmm_plan_multipoles,
    fmm_plan_leaf_points), the top levels' translations (fmm_translate),
    received multipoles and points in (fmm_plan_add_locals, fmm_m2l_external,
    fmm_p2p_external) and the downward pass (fmm_eval_downward)."""

    def __init__(self, p: int, theta: float, tight: bool = False, device=None, stream=None):
        import torch
        from . import load, ncoef_of
        self.torch, self.lib, self.p, self.theta, self.tight = torch, load(), p, theta, tight
        self.nc = ncoef_of(p)
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.stream = stream

    def _st(self):
        s = self.stream or self.torch.cuda.current_stream(self.device)
        return s.cuda_stream

    def _d(self, a, dtype=None):
        return self.torch.as_tensor(np.ascontiguousarray(a, dtype=dtype)).to(self.device)

    def _ok(self, st, what):
        if st != 0:
            from . import FmmError
            raise FmmError(st, what)

    def theta_weak(self, theta, ca, ra, cb, rb):
        n = len(ra)
        if n == 0:
            return np.zeros(0, bool)
        t = [self._d(v, np.float64) for v in (ca, ra, cb, rb)]
        out = self.torch.empty(n, dtype=self.torch.uint8, device=self.device)
        self._ok(self.lib.fmm_theta_test(float(theta), n, *[v.data_ptr() for v in t], out.data_ptr(), self._st()),
                 "fmm_theta_test")
        return out.cpu().numpy().astype(bool)

    def plan(self, x, levels, root_cell):
        from . import fmm_plan, fmm_plan_tree, FMM_PREC_FP64
        pl = fmm_plan(self._d(x, np.float64), levels, self.p, self.theta, prec=FMM_PREC_FP64, stream=self.stream,
                      tight=self.tight, root_cell=root_cell)
        return {"plan": pl, "t": fmm_plan_tree(pl), "B": levels, "n": len(x)}

    def geo(self, P, l):
        sl = slice((1 << l) - 1, (2 << l) - 1)
        return P["t"]["centre"][sl], P["t"]["radius"][sl]

    def upward(self, P, q):
        P["q"] = self._d(q, np.float64)
        self._ok(self.lib.fmm_eval_upward(P["plan"].handle, P["q"].data_ptr(), self._st()), "fmm_eval_upward")

    def multipoles(self, P, l, idx):
        idx = self._d(idx, np.int32)
        out = self.torch.empty((len(idx), self.nc, 2), dtype=self.torch.float64, device=self.device)
        self._ok(self.lib.fmm_plan_multipoles(P["plan"].handle, int(l), len(idx), idx.data_ptr(), out.data_ptr(),
                                              self._st()), "fmm_plan_multipoles")
        return out.cpu().numpy().reshape(len(idx), 2 * self.nc).view(complex)

    def _translate(self, kind, src, cs, cd):
        src = np.ascontiguousarray(np.asarray(src, complex).reshape(-1, self.nc))
        s, a, b = self._d(src.view(np.float64)), self._d(cs, np.float64), self._d(cd, np.float64)
        out = self.torch.zeros_like(s)
        self._ok(self.lib.fmm_translate(kind, self.p, len(src), s.data_ptr(), a.data_ptr(), b.data_ptr(),
                                        out.data_ptr(), self._st()), "fmm_translate")
        return out.cpu().numpy().view(complex).reshape(-1, self.nc)

    def top_local(self, part, Mg, rank, top):
        """Local expansion at the rank's level-g box from the weak pairs of
        levels 1..g: the top boxes' multipoles by M2M from the gathered
        level-g ones, M2L into the rank's ancestors, L2L down to its box."""
        g = part.g
        M = {((1 << g) - 1) + r: Mg[r] for r in range(1 << g)}
        for l in range(g - 1, -1, -1):
            for j in range(1 << l):
                h = (1 << l) - 1 + j
                kids = [2 * h + 1, 2 * h + 2]
                t = self._translate(0, [M[c] for c in kids], part.centre[kids], part.centre[[h, h]])
                M[h] = t.sum(0)
        L = np.zeros(self.nc, complex)
        for l in range(1, g + 1):
            a = rank >> (g - l)
            ha = (1 << l) - 1 + a
            bs = [int(b) for aa, b in top[l][0] if aa == a]
            if not bs:
                continue
            hb = [(1 << l) - 1 + b for b in bs]
            cur = self._translate(1, [M[h] for h in hb], part.centre[hb], part.centre[[ha] * len(hb)]).sum(0)
            for ll in range(l + 1, g + 1):
                hc = (1 << ll) - 1 + (rank >> (g - ll))
                cur = self._translate(2, [cur], part.centre[[ha]], part.centre[[hc]])[0]
                ha = hc
            L += cur
        return L

    def add_local(self, P, l, idx, Ls):
        idx = self._d(idx, np.int32)
        Lv = self._d(np.asarray(Ls, complex).reshape(-1, self.nc).view(np.float64))
        self._ok(self.lib.fmm_plan_add_locals(P["plan"].handle, int(l), len(idx), idx.data_ptr(), Lv.data_ptr(),
                                              self._st()), "fmm_plan_add_locals")

    def m2l_external(self, P, l, tgt, M, centres):
        t = self._d(tgt, np.int32)
        Mv = self._d(np.ascontiguousarray(np.asarray(M, complex)).view(np.float64))
        c = self._d(centres, np.float64)
        self._ok(self.lib.fmm_m2l_external(P["plan"].handle, int(l), len(t), t.data_ptr(), Mv.data_ptr(),
                                           c.data_ptr(), self._st()), "fmm_m2l_external")

    def leaf_points(self, P, idx):
        tr, B = P["t"], P["B"]
        cnt = tr["count"][(1 << B) - 1 + np.asarray(idx, np.int64)]
        off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
        out = self.torch.empty((int(off[-1]), 4), dtype=self.torch.float64, device=self.device)
        li, lo = self._d(idx, np.int32), self._d(off, np.int64)
        self._ok(self.lib.fmm_plan_leaf_points(P["plan"].handle, len(idx), li.data_ptr(), lo.data_ptr(),
                                               out.data_ptr(), self._st()), "fmm_plan_leaf_points")
        h = out.cpu().numpy()
        return [h[off[k]:off[k + 1]] for k in range(len(idx))]

    def p2p_external(self, P, tgt, srcs):
        if len(tgt) == 0:
            return
        off = np.concatenate([[0], np.cumsum([len(s) for s in srcs])]).astype(np.int64)
        src = np.concatenate(srcs) if off[-1] else np.zeros((1, 4))
        t, o, s = self._d(tgt, np.int32), self._d(off, np.int64), self._d(src, np.float64)
        self._ok(self.lib.fmm_p2p_external(P["plan"].handle, len(t), t.data_ptr(), o.data_ptr(), s.data_ptr(),
                                           self._st()), "fmm_p2p_external")

    def downward(self, P):
        n = P["n"]
        pot = self.torch.empty(n, dtype=self.torch.float64, device=self.device)
        fld = self.torch.empty((n, 3), dtype=self.torch.float64, device=self.device)
        self._ok(self.lib.fmm_eval_downward(P["plan"].handle, pot.data_ptr(), fld.data_ptr(), self._st()),
                 "fmm_eval_downward")
        return pot.cpu().numpy(), fld.cpu().numpy()
