"""Pins for the oracle's balanced tree (Sec. 2.1.2, eta = 1 median splits;
Algorithm 2) and connectivity (Eq. 2.2 and the inheritance rule of Sec. 2.1.1):
invariants, a second independent implementation, and brute force."""
import numpy as np
import pytest

import oracle
from paper_2002_04894_gb300 import inputs


def naive_tree(x, levels, eta=1.0):
    """Second, independent implementation of the same reading: full sort of
    each box on its longest cell axis, floor(n/2) smallest keys to the left;
    for eta < 1 the plane moves to eta*median + (1-eta)*midpoint and the left
    child takes the points strictly below it."""
    x = np.asarray(x, float) + 0.0
    nb = (2 << levels) - 1
    lo = np.zeros((nb, 3)); hi = np.zeros((nb, 3)); plane = np.zeros(nb)
    members = [None] * nb
    members[0] = np.arange(len(x))
    lo[0], hi[0] = x.min(0), x.max(0)
    for l in range(levels):
        for j in range(1 << l):
            g = (1 << l) - 1 + j
            idx = members[g]
            ext = hi[g] - lo[g]
            ax = int(np.argmax(ext))           # first maximum: x before y before z
            order = sorted(idx, key=lambda i: (x[i, ax], i))
            k = len(idx) // 2
            left = set(order[:k])
            if len(idx) >= 2:
                s = 0.5 * (x[order[k - 1], ax] + x[order[k], ax])
            elif len(idx) == 1:
                s = x[order[0], ax]
            else:
                s = 0.5 * (lo[g, ax] + hi[g, ax])
            if eta < 1.0:
                s = eta * s + (1.0 - eta) * (0.5 * (lo[g, ax] + hi[g, ax]))
                left = {i for i in idx if x[i, ax] < s}
            plane[g] = s
            a, b = 2 * g + 1, 2 * g + 2
            members[a] = np.array([i for i in idx if i in left], int)
            members[b] = np.array([i for i in idx if i not in left], int)
            lo[a], hi[a], lo[b], hi[b] = lo[g], hi[g].copy(), lo[g].copy(), hi[g]
            hi[a, ax] = s
            lo[b, ax] = s
    first_leaf = (1 << levels) - 1
    perm = np.concatenate([members[g] for g in range(first_leaf, nb)])
    return perm, lo, hi, plane


CASES = [("uniform", 1000, 5), ("uniform", 777, 6), ("plummer", 1500, 6), ("gmm", 1200, 7),
         ("uniform", 20, 6), ("uniform", 1, 3), ("uniform", 2, 2)]


@pytest.mark.parametrize("kind,n,levels", CASES)
def test_tree_matches_independent_implementation(kind, n, levels):
    x = inputs.points(kind, n, seed=n)
    t = oracle.Tree(x, levels, 2, 0.5).tree()
    perm, lo, hi, plane = naive_tree(x, levels)
    np.testing.assert_array_equal(t["perm"], perm)
    np.testing.assert_array_equal(t["lo"], lo)
    np.testing.assert_array_equal(t["hi"], hi)
    internal = (1 << levels) - 1
    np.testing.assert_array_equal(t["plane"][:internal], plane[:internal])


def test_tree_with_ties_and_negative_zero():
    rng = np.random.default_rng(1)
    x = rng.integers(0, 3, size=(300, 3)).astype(float) - 1.0
    x[::7] *= -1.0                         # produces -0.0 entries
    t = oracle.Tree(x, 5, 2, 0.5).tree()
    perm, lo, hi, _ = naive_tree(x, 5)
    np.testing.assert_array_equal(t["perm"], perm)
    np.testing.assert_array_equal(t["lo"], lo)


@pytest.mark.parametrize("kind,n,levels", CASES[:4])
def test_tree_invariants(kind, n, levels):
    x = inputs.points(kind, n, seed=3) + 0.0
    t = oracle.Tree(x, levels, 2, 0.5).tree()
    assert sorted(t["perm"]) == list(range(n))                    # bijection
    for l in range(levels + 1):
        for j in range(1 << l):
            g = (1 << l) - 1 + j
            cnt = t["count"][g]
            assert cnt in (n >> l, -((-n) >> l))                  # balanced (Sec. 1)
            pts = t["perm"][t["begin"][g]:t["begin"][g] + cnt]
            if l == levels:
                assert np.all(np.diff(pts) > 0)                   # stable: ascending index
            assert np.all(x[pts] >= t["lo"][g]) and np.all(x[pts] <= t["hi"][g])
            np.testing.assert_array_equal(t["centre"][g], 0.5 * (t["lo"][g] + t["hi"][g]))
            if l < levels:
                ax = t["axis"][g]
                ext = t["hi"][g] - t["lo"][g]
                assert ext[ax] == ext.max() and np.argmax(ext) == ax
                a, b = 2 * g + 1, 2 * g + 2
                assert t["count"][a] == cnt // 2
                la = x[t["perm"][t["begin"][a]:t["begin"][a] + t["count"][a]], ax]
                rb = x[t["perm"][t["begin"][b]:t["begin"][b] + t["count"][b]], ax]
                if len(la) and len(rb):
                    assert la.max() <= t["plane"][g] <= rb.min()


def ancestors_weak(t, theta, l, a, b):
    while l > 0:
        l -= 1
        a //= 2
        b //= 2
        ga, gb = (1 << l) - 1 + a, (1 << l) - 1 + b
        if oracle.theta_weak(theta, t["centre"][ga], t["radius"][ga], t["centre"][gb], t["radius"][gb]):
            return True
    return False


@pytest.mark.parametrize("theta", [0.0, 0.35, 0.5, 0.8])
def test_lists_brute_force(theta):
    x = inputs.points("plummer", 300, seed=4)
    levels = 5
    T = oracle.Tree(x, levels, 2, theta)
    t = T.tree()
    for l in range(1, levels + 1):
        wp, ws = T.lists(l, "weak")
        sp, ss = T.lists(l, "strong")
        for a in range(1 << l):
            want_w, want_s = [], []
            for b in range(1 << l):
                if ancestors_weak(t, theta, l, a, b):
                    continue
                ga, gb = (1 << l) - 1 + a, (1 << l) - 1 + b
                if oracle.theta_weak(theta, t["centre"][ga], t["radius"][ga], t["centre"][gb], t["radius"][gb]):
                    want_w.append(b)
                else:
                    want_s.append(b)
            assert list(ws[wp[a]:wp[a + 1]]) == want_w
            assert list(ss[sp[a]:sp[a + 1]]) == want_s


def test_theta_criterion_formula_and_edges():
    c0, c1 = np.zeros(3), np.array([3.0, 0, 0])
    # R + theta r <= theta d at equality is weak: r = R = 1, theta = 0.5, d = 3
    assert oracle.theta_weak(0.5, c0, 1.0, c1, 1.0)
    assert not oracle.theta_weak(0.5, c0, 1.0, c1, 1.0 + 1e-12)
    assert not oracle.theta_weak(0.0, c0, 0.0, c1, 0.0)          # theta = 0: never weak
    assert not oracle.theta_weak(0.5, c0, 0.0, c0, 0.0)          # d = 0: never weak
    assert oracle.theta_weak(0.5, c0, 0.0, c1, 0.0)


@pytest.mark.parametrize("kind,theta", [("uniform", 0.5), ("plummer", 0.4), ("gmm", 0.6)])
def test_every_source_counted_once(kind, theta):
    """For every target leaf, sources reached through weak lists at all levels
    (their whole subtrees) plus strong leaves cover all N points exactly once."""
    n, levels = 800, 6
    x = inputs.points(kind, n, seed=2)
    T = oracle.Tree(x, levels, 2, theta)
    t = T.tree()
    lists = {l: T.lists(l, "weak") for l in range(1, levels + 1)}
    sp, ss = T.lists(levels, "strong")
    for leaf in range(1 << levels):
        total = 0
        for l in range(1, levels + 1):
            a = leaf >> (levels - l)
            wp, ws = lists[l]
            total += sum(t["count"][(1 << l) - 1 + b] for b in ws[wp[a]:wp[a + 1]])
        total += sum(t["count"][(1 << levels) - 1 + b] for b in ss[sp[leaf]:sp[leaf + 1]])
        assert total == n


def test_list_counts_follow_cost_model_directions():
    """M2L work rises and P2P work falls with theta and with levels (Sec. 3.2)."""
    x = inputs.points("uniform", 4000, seed=0)

    def counts(levels, theta):
        T = oracle.Tree(x, levels, 2, theta)
        w = sum(len(T.lists(l, "weak")[1]) for l in range(1, levels + 1))
        return w, len(T.lists(levels, "strong")[1])
    w1, s1 = counts(7, 0.4)
    w2, s2 = counts(7, 0.6)
    assert w2 > w1 and s2 < s1
    w3, s3 = counts(8, 0.5)
    w4, s4 = counts(6, 0.5)
    assert w3 > w4
    assert s3 * (4000 / 256) ** 2 < s4 * (4000 / 64) ** 2


@pytest.mark.parametrize("kind,n", [("uniform", 999), ("plummer", 1200), ("gmm", 64)])
def test_single_box_bisection_matches_tree(kind, n):
    """The one-box bisection agrees with the tree's own splits of every box."""
    x = inputs.points(kind, n, seed=6) + 0.0
    t = oracle.Tree(x, 4, 2, 0.5).tree()
    for g in range(15):
        pts = np.sort(t["perm"][t["begin"][g]:t["begin"][g] + t["count"][g]])
        ax, left, plane = oracle.bisect_box(x[pts], t["lo"][g], t["hi"][g])
        assert ax == t["axis"][g] and plane == t["plane"][g]
        a = 2 * g + 1
        want = set(t["perm"][t["begin"][a]:t["begin"][a] + t["count"][a]])
        assert set(pts[left]) == want


@pytest.mark.parametrize("eta", [0.0, 0.25, 0.5, 0.75])
@pytest.mark.parametrize("kind,n,levels", [("plummer", 900, 6), ("gmm", 700, 7), ("uniform", 50, 5)])
def test_eta_tree_matches_independent_implementation(kind, n, levels, eta):
    x = inputs.points(kind, n, seed=n + 1)
    t = oracle.Tree(x, levels, 2, 0.5, eta=eta).tree()
    perm, lo, hi, plane = naive_tree(x, levels, eta)
    np.testing.assert_array_equal(t["perm"], perm)
    np.testing.assert_array_equal(t["lo"], lo)
    np.testing.assert_array_equal(t["hi"], hi)


def test_eta_zero_is_the_fixed_geometric_tree():
    """eta = 0: every split at the cell midpoint, so at level l each cell is
    the root cell halved along its longest axes -- sizes independent of the
    points (Sec. 2.1.2)."""
    x = inputs.points("plummer", 2000, 5)
    t = oracle.Tree(x, 6, 2, 0.5, eta=0.0).tree()
    for g in range(63):
        ax = t["axis"][g]
        assert t["plane"][g] == 0.5 * (t["lo"][g, ax] + t["hi"][g, ax])
    ext = t["hi"][63:] - t["lo"][63:]
    assert np.allclose(ext, ext[0])                 # all leaves the same shape


def test_eta_one_keeps_median_balance():
    x = inputs.points("gmm", 3000, 2)
    a = oracle.Tree(x, 6, 2, 0.5, eta=1.0).tree()
    b = oracle.Tree(x, 6, 2, 0.5).tree()
    np.testing.assert_array_equal(a["perm"], b["perm"])


@pytest.mark.parametrize("eta", [0.0, 0.5])
def test_eta_fmm_accuracy(eta):
    """The expansions do not depend on how boxes were split: accuracy holds."""
    x = inputs.points("plummer", 4000, 9)
    q = inputs.charges_uniform(4000, 9)
    phi = oracle.Tree(x, 6, 10, 0.5, eta=eta).eval(q, field=False)
    p0 = oracle.direct(x, q, field=False)
    assert np.linalg.norm(phi - p0) / np.linalg.norm(p0) < 1e-5


# ---------------------------------------------------------------------------
# Octree levels: 3 bisections per FMM level (8 children per box)
# ---------------------------------------------------------------------------
def ancestors_weak_step(t, theta, l, a, b, step):
    while l > step:
        l -= step
        a >>= step
        b >>= step
        ga, gb = (1 << l) - 1 + a, (1 << l) - 1 + b
        if oracle.theta_weak(theta, t["centre"][ga], t["radius"][ga], t["centre"][gb], t["radius"][gb]):
            return True
    return False


@pytest.mark.parametrize("step,levels", [(3, 6), (2, 6), (3, 3)])
@pytest.mark.parametrize("theta", [0.35, 0.5, 0.8])
def test_octree_lists_brute_force(step, levels, theta):
    """Pairs of FMM level l are weak iff the theta-test holds at l and fails
    at every coarser FMM level; bisection levels between FMM levels carry no
    pairs at all."""
    x = inputs.points("plummer", 400, seed=6)
    T = oracle.Tree(x, levels, 2, theta, step=step)
    t = T.tree()
    for l in range(1, levels + 1):
        wp, ws = T.lists(l, "weak")
        sp, ss = T.lists(l, "strong")
        if l % step:
            assert wp[-1] == 0 and sp[-1] == 0
            continue
        for a in range(1 << l):
            want_w, want_s = [], []
            for b in range(1 << l):
                if ancestors_weak_step(t, theta, l, a, b, step):
                    continue
                ga, gb = (1 << l) - 1 + a, (1 << l) - 1 + b
                if oracle.theta_weak(theta, t["centre"][ga], t["radius"][ga], t["centre"][gb], t["radius"][gb]):
                    want_w.append(b)
                else:
                    want_s.append(b)
            assert list(ws[wp[a]:wp[a + 1]]) == want_w
            assert list(ss[sp[a]:sp[a + 1]]) == want_s


def test_octree_candidates_are_64_per_strong_parent_pair():
    x = inputs.points("gmm", 3000, seed=8)
    T = oracle.Tree(x, 9, 2, 0.5, step=3)
    for l in (3, 6, 9):
        nstrong_parent = T.lists(l - 3, "strong")[0][-1]
        assert T.lists(l, "weak")[0][-1] + T.lists(l, "strong")[0][-1] == 64 * nstrong_parent


@pytest.mark.parametrize("kind,theta", [("uniform", 0.5), ("plummer", 0.4)])
def test_octree_every_source_counted_once(kind, theta):
    n, levels, step = 900, 6, 3
    x = inputs.points(kind, n, seed=3)
    T = oracle.Tree(x, levels, 2, theta, step=step)
    t = T.tree()
    lists = {l: T.lists(l, "weak") for l in range(step, levels + 1, step)}
    sp, ss = T.lists(levels, "strong")
    for leaf in range(1 << levels):
        total = 0
        for l, (wp, ws) in lists.items():
            a = leaf >> (levels - l)
            total += sum(t["count"][(1 << l) - 1 + b] for b in ws[wp[a]:wp[a + 1]])
        total += sum(t["count"][(1 << levels) - 1 + b] for b in ss[sp[leaf]:sp[leaf + 1]])
        assert total == n


def test_octree_tree_is_the_binary_tree():
    """The step only changes which bisection levels carry expansions: the
    boxes themselves are the same."""
    x = inputs.points("plummer", 2000, seed=1)
    a = oracle.Tree(x, 6, 2, 0.5).tree()
    b = oracle.Tree(x, 6, 2, 0.5, step=3).tree()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    with pytest.raises(ValueError):
        oracle.Tree(x, 7, 2, 0.5, step=3)


@pytest.mark.parametrize("kind", ["plummer", "uniform"])
@pytest.mark.parametrize("theta,p,tol", [(0.0, 4, 1e-13), (0.5, 6, 1e-4), (0.5, 10, 2e-6),
                                         (0.4, 12, 2e-8)])
def test_octree_fmm_accuracy(kind, theta, p, tol):
    """theta = 0: no weak pairs, so the FMM is the direct sum; otherwise the
    octree FMM (tens of thousands of M2L pairs here) meets the accuracy of
    the binary one (Sec. 3.1 bound)."""
    n = 4000
    x = inputs.points(kind, n, seed=12)
    q = inputs.charges_uniform(n, seed=12)
    T = oracle.Tree(x, 9, p, theta, step=3)
    assert (sum(T.lists(l, "weak")[0][-1] for l in (3, 6, 9)) > 0) == (theta > 0)
    phi, E = T.eval(q)
    d_phi, d_E = oracle.direct(x, q)
    assert np.linalg.norm(phi - d_phi) / np.linalg.norm(d_phi) <= tol
    assert np.linalg.norm(E - d_E) / np.linalg.norm(d_E) <= 3 * tol


@pytest.mark.parametrize("step,levels", [(1, 8), (3, 6)])
@pytest.mark.parametrize("kind", ["plummer", "gmm"])
def test_lists_are_symmetric(kind, step, levels):
    """The theta-criterion is symmetric in the two boxes (Eq. 2.2), so every
    weak or strong pair is stored in both orientations."""
    x = inputs.points(kind, 3000, seed=7)
    T = oracle.Tree(x, levels, 2, 0.5, step=step)
    for l in range(levels + 1):
        for kind_ in ("weak", "strong"):
            p, s = T.lists(l, kind_)
            pairs = {(a, int(b)) for a in range(len(p) - 1) for b in s[p[a]:p[a + 1]]}
            assert pairs == {(b, a) for a, b in pairs}


# ---------------------------------------------------------------------------
# tight box geometry (centre and radius from the box's own points)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,n,levels,eta", [("gmm", 4000, 7, 1.0), ("plummer", 3000, 6, 1.0),
                                               ("uniform", 100, 8, 1.0), ("gmm", 3000, 7, 0.3)])
def test_tight_boxes_hold_their_points_and_keep_the_cells(kind, n, levels, eta):
    x = inputs.points(kind, n, seed=7)
    a = oracle.Tree(x, levels, 2, 0.5, eta=eta).tree()
    b = oracle.Tree(x, levels, 2, 0.5, eta=eta, tight=True).tree()
    for k in ("perm", "begin", "count", "lo", "hi", "axis", "plane"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)   # same splits and cells
    xs = x[b["perm"]]
    for g in range(len(b["count"])):
        c, r = b["centre"][g], b["radius"][g]
        assert r >= a["radius"][g] * 2.0 ** -10
        assert r <= a["radius"][g] * (1 + 1e-15)           # inside the cell
        pts = xs[b["begin"][g]:b["begin"][g] + b["count"][g]]
        if len(pts) == 0:
            np.testing.assert_array_equal(c, a["centre"][g])
            assert r == a["radius"][g] * 2.0 ** -10
            continue
        lo, hi = pts.min(0), pts.max(0)
        np.testing.assert_array_equal(c, 0.5 * (lo + hi))   # brute force, numpy
        assert np.all(np.linalg.norm(pts - c, axis=1) <= r * (1 + 1e-13))  # rounding at a corner
        if len(pts) > 1 and np.any(hi > lo):
            assert np.isclose(r, max(0.5 * np.linalg.norm(hi - lo), a["radius"][g] * 2.0 ** -10), rtol=1e-15)


@pytest.mark.parametrize("theta", [0.35, 0.5, 0.8])
def test_tight_lists_match_brute_force(theta):
    x = inputs.points("gmm", 300, seed=9)
    levels = 5
    T = oracle.Tree(x, levels, 2, theta, tight=True)
    t = T.tree()
    for l in range(1, levels + 1):
        wp, ws = T.lists(l, "weak")
        sp, ss = T.lists(l, "strong")
        for a in range(1 << l):
            want_w, want_s = [], []
            for b in range(1 << l):
                if ancestors_weak(t, theta, l, a, b):
                    continue
                ga, gb = (1 << l) - 1 + a, (1 << l) - 1 + b
                if oracle.theta_weak(theta, t["centre"][ga], t["radius"][ga], t["centre"][gb], t["radius"][gb]):
                    want_w.append(b)
                else:
                    want_s.append(b)
            assert list(ws[wp[a]:wp[a + 1]]) == want_w
            assert list(ss[sp[a]:sp[a + 1]]) == want_s


def test_tight_fmm_converges_to_the_direct_sum():
    n = 3000
    x = inputs.points("gmm", n, seed=2)
    q = inputs.charges_uniform(n, seed=2)
    ref = oracle.direct(x, q, field=False)
    errs = []
    for p in (2, 4, 6, 8, 10):
        phi = oracle.Tree(x, 7, p, 0.5, tight=True).eval(q, field=False)
        errs.append(np.linalg.norm(phi - ref) / np.linalg.norm(ref))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6
    # theta = 0: no weak pairs, so the sum is the direct one
    phi0 = oracle.Tree(x, 7, 3, 0.0, tight=True).eval(q, field=False)
    assert np.linalg.norm(phi0 - ref) / np.linalg.norm(ref) < 1e-14
