"""One system split over G = 2 and 4 ranks (paper Sec. 2.2, Algorithms 2-4),
run as gloo processes on the CPU: the bookkeeping of paper_2002_04894_gb300.dist
with an oracle-based backend standing in for the device kernels.

Checks, per rank and gathered on rank 0:
  - a rank's subtree, built from its own points with its root cell, is the
    global subtree (oracle trees);
  - the union over ranks of the local lists and the halos is the single-rank
    oracle's connectivity, bit for bit, at every level;
  - every halo equals the brute-force cross-rank weak/strong pairs (child
    pairs of strongly connected parents, theta-tested);
  - the multipoles and leaf points each rank receives are exactly its peers'
    boxes and leaves in the halo;
  - the distributed evaluation (upward pass per rank, gathered top levels,
    halo M2L from received multipoles, halo P2P from received points) gives
    the single-rank oracle's potentials and fields.
"""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


class OracleBackend:
    """The arithmetic of the split, done with the oracle's operators on the
    CPU (test only). A 'plan' is a dict over an oracle tree of the rank's
    points."""

    def __init__(self, p, theta, tight):
        import oracle
        self.o, self.p, self.theta, self.tight = oracle, p, theta, tight
        self.nc = oracle.ncoef(p)

    def theta_weak(self, theta, ca, ra, cb, rb):
        return np.array([self.o.theta_weak(theta, ca[i], ra[i], cb[i], rb[i]) for i in range(len(ra))], bool)

    def plan(self, x, levels, root_cell):
        T = self.o.Tree(x, levels, self.p, self.theta, root_cell=root_cell, tight=self.tight)
        t = T.tree()
        nb = len(t["radius"])
        return {"T": T, "t": t, "x": np.asarray(x, np.float64), "B": levels,
                "M": np.zeros((nb, self.nc), complex), "L": np.zeros((nb, self.nc), complex),
                "phi": np.zeros(len(x)), "E": np.zeros((len(x), 3))}

    def geo(self, P, l):
        sl = slice((1 << l) - 1, (2 << l) - 1)
        return P["t"]["centre"][sl], P["t"]["radius"][sl]

    def _pts(self, P, g):
        b, c = P["t"]["begin"][g], P["t"]["count"][g]
        return P["t"]["perm"][b:b + c]

    def upward(self, P, q):
        P["q"] = np.asarray(q, np.float64)
        t, B = P["t"], P["B"]
        for j in range(1 << B):
            g = (1 << B) - 1 + j
            idx = self._pts(P, g)
            if len(idx):
                self.o.p2m(P["x"][idx], P["q"][idx], t["centre"][g], self.p, P["M"][g])
        for l in range(B - 1, -1, -1):
            for j in range(1 << l):
                g = (1 << l) - 1 + j
                for c in (2 * g + 1, 2 * g + 2):
                    self.o.m2m(P["M"][c], t["centre"][c], t["centre"][g], self.p, P["M"][g])

    def multipoles(self, P, l_local, idx):
        return P["M"][(1 << l_local) - 1 + np.asarray(idx, np.int64)]

    def top_local(self, part, Mg, rank, top):
        """Local expansion at the rank's level-g box from the top levels."""
        g = part.g
        M = {}
        for r in range(1 << g):
            M[((1 << g) - 1) + r] = Mg[r]
        for l in range(g - 1, -1, -1):
            for j in range(1 << l):
                h = (1 << l) - 1 + j
                acc = np.zeros(self.nc, complex)
                for c in (2 * h + 1, 2 * h + 2):
                    self.o.m2m(M[c], part.centre[c], part.centre[h], self.p, acc)
                M[h] = acc
        L = np.zeros(self.nc, complex)
        for l in range(1, g + 1):
            a_own = rank >> (g - l)
            wk, _ = top[l]
            cur = np.zeros(self.nc, complex)
            for a, b in wk:
                if a == a_own:
                    self.o.m2l(M[(1 << l) - 1 + b], part.centre[(1 << l) - 1 + b],
                               part.centre[(1 << l) - 1 + a], self.p, cur)
            # shift down to the rank's level-g box
            h = (1 << l) - 1 + a_own
            for ll in range(l + 1, g + 1):
                child = (1 << ll) - 1 + (rank >> (g - ll))
                nxt = np.zeros(self.nc, complex)
                self.o.l2l(cur, part.centre[h], part.centre[child], self.p, nxt)
                cur, h = nxt, child
            L += cur
        return L

    def add_local(self, P, l_local, idx, Ls):
        for i, Lv in zip(idx, Ls):
            P["L"][(1 << l_local) - 1 + i] += Lv

    def m2l_external(self, P, l_local, tgt, Ms, cs):
        for i, Mv, c in zip(tgt, Ms, cs):
            g = (1 << l_local) - 1 + i
            self.o.m2l(Mv, c, P["t"]["centre"][g], self.p, P["L"][g])

    def leaf_points(self, P, idx):
        out = []
        for j in idx:
            k = self._pts(P, (1 << P["B"]) - 1 + j)
            out.append(np.concatenate([P["x"][k], P["q"][k, None]], 1))
        return out

    def _p2p(self, P, j, src):
        """Direct sum of sources src (m, 4) at the points of leaf j."""
        k = self._pts(P, (1 << P["B"]) - 1 + j)
        if not len(k) or not len(src):
            return
        xx = np.concatenate([P["x"][k], src[:, :3]])
        qq = np.concatenate([np.zeros(len(k)), src[:, 3]])
        f, E = self.o.direct(xx, qq, targets=np.arange(len(k)))
        P["phi"][k] += f
        P["E"][k] += E

    def p2p_external(self, P, tgt, srcs):
        for i, s in zip(tgt, srcs):
            self._p2p(P, int(i), s)

    def downward(self, P):
        t, B, T = P["t"], P["B"], P["T"]
        for l in range(1, B + 1):
            wp, ws = T.lists(l, "weak")
            for a in range(1 << l):
                ga = (1 << l) - 1 + a
                for b in ws[wp[a]:wp[a + 1]]:
                    gb = (1 << l) - 1 + b
                    self.o.m2l(P["M"][gb], t["centre"][gb], t["centre"][ga], self.p, P["L"][ga])
        for l in range(1, B + 1):
            for j in range(1 << l):
                g = (1 << l) - 1 + j
                par = (g - 1) // 2
                self.o.l2l(P["L"][par], t["centre"][par], t["centre"][g], self.p, P["L"][g])
        sp, ss = T.lists(B, "strong")
        for j in range(1 << B):
            g = (1 << B) - 1 + j
            k = self._pts(P, g)
            for i in k:
                f, E = self.o.l2p(P["L"][g], t["centre"][g], self.p, P["x"][i])
                P["phi"][i] += f
                P["E"][i] += E
            for s in ss[sp[j]:sp[j + 1]]:
                ks = self._pts(P, (1 << B) - 1 + s)
                src = np.concatenate([P["x"][ks], P["q"][ks, None]], 1)
                if s == j:   # self pair: the direct sum over the leaf skips i == j itself
                    if len(k):
                        f, E = self.o.direct(P["x"][k], P["q"][k])
                        P["phi"][k] += f
                        P["E"][k] += E
                else:
                    self._p2p(P, j, src)
        return P["phi"], P["E"]


def _worker(rank, world, port, cfg, out):
    os.environ["OMP_NUM_THREADS"] = "1"  # many tiny oracle calls: no thread team each time
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as tdist
    import oracle
    from paper_2002_04894_gb300 import dist, inputs
    tdist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        kind, n, B, p, theta, tight = cfg
        g = world.bit_length() - 1
        x = inputs.points(kind, n, seed=3)
        q = inputs.charges_uniform(n, seed=3)
        G = oracle.Tree(x, B, p, theta, tight=tight)           # single-rank reference
        gt = G.tree()
        part = dist.Partition.from_tree(gt, g, B)
        be = OracleBackend(p, theta, tight)
        comm = dist.TorchComm("cpu")
        mine = part.points_of[rank]
        P = be.plan(x[mine], B - g, (part.lo[rank], part.hi[rank]))
        res = {}
        # the rank's subtree is the global subtree
        lo0 = dist.owned(rank, g, g)[0]
        for l in range(g, B + 1):
            c, r = be.geo(P, l - g)
            a, b = dist.owned(rank, g, l)
            hs = dist.heap(l, np.arange(a, b))
            assert np.array_equal(c, gt["centre"][hs]) and np.array_equal(r, gt["radius"][hs]), l
        # halos (Algorithm 2)
        H = dist.build_halo(rank, world, part, theta, lambda l: be.geo(P, l - g), comm, be)
        # lists: local (shifted to global indices) + halos, per level, as sets
        mylists = {}
        for l in range(g, B + 1):
            a0 = dist.owned(rank, g, l)[0]
            for kind_ in ("weak", "strong"):
                pp, ss = P["T"].lists(l - g, kind_)
                rows = np.repeat(np.arange(len(pp) - 1), np.diff(pp)) + a0
                pairs = set(zip(rows.tolist(), (ss + a0).tolist()))
                for qq in range(world):
                    if qq != rank and (qq, l) in getattr(H, kind_):
                        pairs |= set(map(tuple, getattr(H, kind_)[(qq, l)].tolist()))
                mylists[(l, kind_)] = pairs
        res["lists"] = mylists
        res["halo"] = {k: v.tolist() for k, v in H.weak.items()}, {k: v.tolist() for k, v in H.strong.items()}
        # evaluation (Algorithms 3 and 4), with the received data checked:
        # every multipole is the oracle's multipole of the box with that
        # centre, every block of points is one peer leaf's points and charges
        G.eval(q)
        GM = G.expansions("M")
        box_of = {tuple(gt["centre"][h]): h for h in range(len(gt["radius"]))}
        leaf_of = {}
        for j in range(1 << B):
            h = dist.heap(B, j)
            k = np.sort(gt["perm"][gt["begin"][h]:gt["begin"][h] + gt["count"][h]])
            if len(k):
                leaf_of[tuple(x[k[0]])] = k
        seen = {"M": 0, "P": 0}
        m2l0, p2p0 = be.m2l_external, be.p2p_external

        def m2l_checked(P_, l, tgt, M, cs):
            for Mv, c in zip(M, cs):
                h = box_of[tuple(c)]
                assert dist.owner(g, l + g, h - ((1 << (l + g)) - 1)) != rank
                assert np.allclose(Mv, GM[h], rtol=1e-12, atol=1e-13 * np.abs(GM[h]).max())
            seen["M"] += len(tgt)
            return m2l0(P_, l, tgt, M, cs)

        def p2p_checked(P_, tgt, srcs):
            for src in srcs:
                k = leaf_of[tuple(src[0, :3])]
                np.testing.assert_array_equal(src[:, :3], x[k])
                np.testing.assert_array_equal(src[:, 3], q[k])
            seen["P"] += len(tgt)
            return p2p0(P_, tgt, srcs)

        be.m2l_external, be.p2p_external = m2l_checked, p2p_checked
        phi, E = dist.evaluate(rank, world, part, H, P, q[mine], theta, comm, be)
        res["halo_m2l_pairs"], res["halo_p2p_pairs"] = seen["M"], seen["P"]
        ophi, oE = G.eval(q)
        res["err_phi"] = float(np.abs(phi - ophi[mine]).max() / np.abs(ophi).max())
        res["err_E"] = float(np.abs(E - oE[mine]).max() / np.abs(oE).max())
        res["n_local"] = len(mine)
        out.put((rank, res))
    finally:
        tdist.destroy_process_group()


def _run(world, cfg):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, cfg, out)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = dict(out.get(timeout=600) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    return res


@pytest.mark.parametrize("world,cfg", [
    (2, ("plummer", 3000, 7, 4, 0.5, False)),
    (2, ("gmm", 2000, 7, 4, 0.5, True)),
    (4, ("uniform", 2000, 7, 3, 0.6, False)),
])
def test_split_matches_single_rank(world, cfg):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2002_04894_gb300 import dist, inputs
    res = _run(world, cfg)
    kind, n, B, p, theta, tight = cfg
    g = world.bit_length() - 1
    x = inputs.points(kind, n, seed=3)
    G = oracle.Tree(x, B, p, theta, tight=tight)
    gt = G.tree()
    assert sum(r["n_local"] for r in res.values()) == n
    # union of per-rank lists (targets owned by each rank) == global lists
    for l in range(g, B + 1):
        for kind_ in ("weak", "strong"):
            pp, ss = G.lists(l, kind_)
            rows = np.repeat(np.arange(len(pp) - 1), np.diff(pp))
            want = set(zip(rows.tolist(), ss.tolist()))
            got = set().union(*[r["lists"][(l, kind_)] for r in res.values()])
            assert got == want, (l, kind_)
    # each halo is the brute-force cross-rank pair set
    for rank, r in res.items():
        wk, st = r["halo"]
        for l in range(g, B + 1):
            pp, ss = G.lists(l, "weak")
            rows = np.repeat(np.arange(len(pp) - 1), np.diff(pp))
            for q in range(world):
                if q == rank:
                    continue
                sel = (dist.owner(g, l, rows) == rank) & (dist.owner(g, l, ss) == q)
                want_w = set(zip(rows[sel].tolist(), ss[sel].tolist()))
                assert set(map(tuple, wk.get((q, l), []))) == want_w, (rank, q, l)
                sp_, sss = G.lists(l, "strong")
                rows_s = np.repeat(np.arange(len(sp_) - 1), np.diff(sp_))
                sel = (dist.owner(g, l, rows_s) == rank) & (dist.owner(g, l, sss) == q)
                want_s = set(zip(rows_s[sel].tolist(), sss[sel].tolist()))
                assert set(map(tuple, st.get((q, l), []))) == want_s, (rank, q, l)
    # the halos carried work (cross-rank M2L and P2P both exercised)
    assert sum(r["halo_m2l_pairs"] for r in res.values()) > 0
    assert sum(r["halo_p2p_pairs"] for r in res.values()) > 0
    # distributed evaluation == single-rank oracle evaluation
    for r in res.values():
        assert r["err_phi"] < 1e-12 and r["err_E"] < 1e-12, r
