"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test pins one oracle function to mathematics or to an independent library:
exact rational arithmetic, brute force over all spanning trees, SciPy's single
linkage, the cut property, hand-built point sets whose merge trees are known, and
the paper's restriction rules worked by hand.  A plausible mistake in the oracle (a
dropped feature, a wrong tie-break, a transposed index, an off-by-one in KL1, a
gate with the wrong inequality) fails at least one of them.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def grid_points(rng, n, d, lim=512):
    """Points on the 1/64 grid with |coordinate| <= lim/64: every squared
    difference and partial sum is exact in binary64."""
    return (rng.integers(-lim, lim + 1, size=(n, d)) / 64.0).astype(np.float32)


def exact_D(x, y):
    return sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(x, y))


# ----------------------------------------------------------------------------------
# Eq. (1): the canonical squared distance
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("d", [1, 5, 8, 25, 32])
def test_dist_exact_on_grid(oracle_mod, d):
    rng = np.random.default_rng(100 + d)
    X = grid_points(rng, 64, d)
    i = rng.integers(0, 64, 300)
    j = rng.integers(0, 64, 300)
    got = oracle_mod.dist_pairs(X, i, j)
    for m in range(300):
        assert got[m] == float(exact_D(X[i[m]], X[j[m]]))


@pytest.mark.parametrize("d", [3, 16, 25])
def test_dist_within_binary64_bound(oracle_mod, d):
    # Random magnitudes over many binades: D must be within the a-priori bound
    # gamma_{d+2} * D of the exact rational value (u = 2^-53).
    rng = np.random.default_rng(7 + d)
    X = (rng.standard_normal((40, d)) * 10.0 ** rng.uniform(-3, 3, (40, d))).astype(np.float32)
    i = rng.integers(0, 40, 200)
    j = rng.integers(0, 40, 200)
    got = oracle_mod.dist_pairs(X, i, j)
    u = Fraction(1, 2 ** 53)
    gamma = (d + 2) * u / (1 - (d + 2) * u)
    for m in range(200):
        ex = exact_D(X[i[m]], X[j[m]])
        assert abs(Fraction(got[m]) - ex) <= gamma * ex
    # symmetric bit for bit, zero on the diagonal
    assert np.array_equal(oracle_mod.dist_pairs(X, i, j), oracle_mod.dist_pairs(X, j, i))
    assert np.all(oracle_mod.dist_pairs(X, i, i) == 0.0)


def test_dist_every_feature_counts(oracle_mod):
    # A difference in any single feature (first, middle, last) shows up in D.
    d = 25
    for k in (0, 12, 24):
        X = np.zeros((2, d), dtype=np.float32)
        X[1, k] = 3.0
        assert oracle_mod.dist_pairs(X, [0], [1])[0] == 9.0


# ----------------------------------------------------------------------------------
# Nearest neighbours
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 4, 9])
def test_knn_matches_sorting_exact_distances(oracle_mod, k):
    rng = np.random.default_rng(11)
    X = grid_points(rng, 200, 6, lim=32)   # coarse grid: many exact ties
    X64 = X.astype(np.float64)
    idx, D = oracle_mod.knn(X, k)
    for i in range(200):
        Di = ((X64 - X64[i]) ** 2).sum(1)   # exact on this grid whatever the order
        Di[i] = np.inf
        order = np.lexsort((np.arange(200), Di))[:k]   # by D, then index
        assert np.array_equal(idx[i], order)
        assert np.array_equal(D[i], Di[order])


def test_knn_duplicates_and_subset(oracle_mod):
    X = np.array([[0, 0], [1, 0], [0, 0], [5, 5], [0, 0]], dtype=np.float32)
    idx, D = oracle_mod.knn(X, 3, queries=[0, 3])
    assert idx[0].tolist() == [2, 4, 1] and D[0].tolist() == [0.0, 0.0, 1.0]
    assert idx[1].tolist() == [1, 0, 2] and D[1].tolist() == [41.0, 50.0, 50.0]


# ----------------------------------------------------------------------------------
# The merge tree
# ----------------------------------------------------------------------------------

def edges_list(e):
    return [(int(a), int(b), float(D)) for a, b, D in zip(e["a"], e["b"], e["D"])]


def tree_checks(X, e):
    """Invariants of the single-linkage tree: N-1 edges, spanning, key-sorted."""
    N = X.shape[0]
    assert len(e) == N - 1
    keys = list(zip(e["D"], e["a"], e["b"]))
    assert keys == sorted(keys)
    assert np.all(e["a"] < e["b"])
    parent = list(range(N))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    for a, b in zip(e["a"], e["b"]):
        ra, rb = find(int(a)), find(int(b))
        assert ra != rb, "cycle"
        parent[ra] = rb


def all_methods(o, X):
    N = X.shape[0]
    ref = o.kruskal_allpairs(X)
    outs = {"prim": o.prim(X), "prim1": o.prim(X, threads=1)}
    for P in (1, 7, 64, N):
        outs[f"batched{P}"] = o.nnm_batched(X, P)
    outs["batched_t1"] = o.nnm_batched(X, 13, threads=1)
    return ref, outs


@pytest.mark.parametrize("case", ["gauss", "lattice", "dups", "grid"])
def test_tree_three_routes_agree(oracle_mod, case):
    rng = np.random.default_rng(5)
    if case == "gauss":
        X = rng.standard_normal((300, 7)).astype(np.float32)
    elif case == "lattice":   # all-tie integer lattice: only the tie-break decides
        X = np.array(list(itertools.product(range(5), repeat=3)), dtype=np.float32)
    elif case == "dups":
        X = rng.standard_normal((150, 4)).astype(np.float32)
        X = np.concatenate([X, X[:60], X[:20]])
    else:
        X = grid_points(rng, 250, 5, lim=40)
    ref, outs = all_methods(oracle_mod, X)
    tree_checks(X, ref)
    for name, e in outs.items():
        assert np.array_equal(e, ref), name


def test_tree_is_min_over_all_spanning_trees(oracle_mod):
    # Brute force: for N <= 7 enumerate every labelled tree (Pruefer codes).  Weigh
    # each pair by the rank of its key: distinct integer weights, so the minimum-sum
    # tree is unique and is the tree under the key order.
    rng = np.random.default_rng(9)
    for trial in range(12):
        N = 5 + trial % 3
        X = (rng.integers(0, 3, size=(N, 2))).astype(np.float32)   # heavy ties
        pairs = sorted((float(exact_D(X[i], X[j])), i, j) for i in range(N) for j in range(i + 1, N))
        rank = {(i, j): r for r, (_, i, j) in enumerate(pairs)}
        best = None
        for code in itertools.product(range(N), repeat=N - 2):
            deg = [1] * N
            for c in code:
                deg[c] += 1
            edges = []
            for c in code:
                leaf = min(v for v in range(N) if deg[v] == 1)
                edges.append((min(leaf, c), max(leaf, c)))
                deg[leaf] -= 1
                deg[c] -= 1
            u, w = [v for v in range(N) if deg[v] == 1]
            edges.append((min(u, w), max(u, w)))
            s = sum(rank[e] for e in edges)
            if best is None or s < best[0]:
                best = (s, sorted(edges))
        got = sorted((int(a), int(b)) for a, b in zip(*[oracle_mod.prim(X)[k] for k in ("a", "b")]))
        assert got == best[1]


def test_tree_heights_match_scipy_single_linkage(oracle_mod):
    from scipy.cluster.hierarchy import linkage
    from scipy.sparse.csgraph import minimum_spanning_tree
    from scipy.spatial.distance import pdist, squareform
    rng = np.random.default_rng(21)
    X = (rng.standard_normal((400, 9)) + rng.integers(0, 4, (400, 1)) * 6).astype(np.float32)
    e = oracle_mod.prim(X)
    h = np.sqrt(e["D"])
    Z = linkage(X.astype(np.float64), method="single")
    assert np.allclose(np.sort(Z[:, 2]), h, rtol=1e-12, atol=0)
    T = minimum_spanning_tree(squareform(pdist(X.astype(np.float64))))
    assert abs(T.sum() - h.sum()) <= 1e-10 * h.sum()


def test_tree_hand_built_collinear(oracle_mod):
    X = np.array([[0.0], [1.0], [3.0], [6.0], [10.0]], dtype=np.float32)
    for e in (oracle_mod.prim(X), oracle_mod.nnm_batched(X, 2)):
        assert edges_list(e) == [(0, 1, 1.0), (1, 2, 4.0), (2, 3, 9.0), (3, 4, 16.0)]


def test_tree_hand_built_two_blobs(oracle_mod):
    rng = np.random.default_rng(3)
    A = rng.uniform(0, 1, (30, 3))
    B = rng.uniform(0, 1, (30, 3)) + np.array([100.0, 0, 0])
    X = np.concatenate([A, B]).astype(np.float32)
    e = oracle_mod.prim(X)
    X64 = X.astype(np.float64)
    gap = min(((X64[i] - X64[j]) ** 2).sum() for i in range(30) for j in range(30, 60))
    last = e[-1]
    assert (last["a"] < 30) != (last["b"] < 30)      # the last merge joins the blobs
    assert abs(last["D"] - gap) <= 1e-12 * gap
    assert np.all(e["D"][:-1] < last["D"])


def test_tree_duplicates_zero_first_by_index(oracle_mod):
    X = np.array([[2, 2], [0, 0], [2, 2], [0, 0], [2, 2]], dtype=np.float32)
    e = edges_list(oracle_mod.prim(X))
    assert e[:3] == [(0, 2, 0.0), (0, 4, 0.0), (1, 3, 0.0)]
    assert e[3] == (0, 1, 8.0)


def test_tree_cut_property_and_nn_edges(oracle_mod):
    rng = np.random.default_rng(31)
    X = grid_points(rng, 120, 4, lim=64)
    e = oracle_mod.prim(X)
    N = X.shape[0]
    X64 = X.astype(np.float64)
    D = ((X64[:, None, :] - X64[None, :, :]) ** 2).sum(-1)   # exact on the grid
    tree = set(zip(e["a"].tolist(), e["b"].tolist()))
    # every row's nearest neighbour edge (by (D, j)) is a tree edge
    for i in range(N):
        Di = D[i].copy()
        Di[i] = np.inf
        j = int(np.lexsort((np.arange(N), Di))[0])
        assert (min(i, j), max(i, j)) in tree
    # cut property: removing a tree edge splits the rows; it is the smallest crossing key
    adj = {v: [] for v in range(N)}
    for a, b in tree:
        adj[a].append(b)
        adj[b].append(a)
    for q in rng.choice(N - 1, 25, replace=False):
        a, b = int(e["a"][q]), int(e["b"][q])
        side = {a}
        stack = [a]
        while stack:
            v = stack.pop()
            for w in adj[v]:
                if {v, w} == {a, b} or w in side:
                    continue
                side.add(w)
                stack.append(w)
        S = np.zeros(N, bool)
        S[list(side)] = True
        ii, jj = np.nonzero(S[:, None] & ~S[None, :])
        keys = sorted(zip(D[ii, jj], np.minimum(ii, jj), np.maximum(ii, jj)))
        assert keys[0] == (e["D"][q], a, b)


# ----------------------------------------------------------------------------------
# Restrictions ("Problem statement", "Problem settings")
# ----------------------------------------------------------------------------------

def merges_list(m):
    return [(int(a), int(b), float(D), int(s)) for a, b, D, s in zip(m["a"], m["b"], m["D"], m["new_size"])]


LINE = np.array([[0.0], [1.0], [3.0], [6.0], [10.0]], dtype=np.float32)   # gaps 1, 2, 3, 4


def restrict(o, X, **r):
    return merges_list(o.restrict_tree(o.prim(X), X.shape[0], r))


def test_restrict_none_is_whole_tree(oracle_mod):
    m = restrict(oracle_mod, LINE)
    assert m == [(0, 1, 1.0, 2), (1, 2, 4.0, 3), (2, 3, 9.0, 4), (3, 4, 16.0, 5)]
    mg = oracle_mod.restrict_tree(oracle_mod.prim(LINE), 5, {})
    assert mg["dist"].tolist() == [1.0, 2.0, 3.0, 4.0]


def test_restrict_max_join_distance(oracle_mod):
    assert restrict(oracle_mod, LINE, max_join_dist=2.5) == [(0, 1, 1.0, 2), (1, 2, 4.0, 3)]
    # only a distance above the cap blocks: an equal distance joins
    assert restrict(oracle_mod, LINE, max_join_dist=2.0) == [(0, 1, 1.0, 2), (1, 2, 4.0, 3)]
    assert restrict(oracle_mod, LINE, max_join_dist=1.999) == [(0, 1, 1.0, 2)]


def test_restrict_kl1_stops_at_count(oracle_mod):
    # 5 clusters; KL1 = 3 leaves exactly 3 clusters
    assert restrict(oracle_mod, LINE, kl1_stop_clusters=3) == [(0, 1, 1.0, 2), (1, 2, 4.0, 3)]
    assert len(restrict(oracle_mod, LINE, kl1_stop_clusters=1)) == 4
    assert restrict(oracle_mod, LINE, kl1_stop_clusters=5) == []


def test_restrict_kl2_pre_sizes(oracle_mod):
    # KL2 = 2: a cluster of 3 may still exist (overshoot), but joins no further
    m = restrict(oracle_mod, LINE, kl2_max_pre_size=2)
    assert m == [(0, 1, 1.0, 2), (1, 2, 4.0, 3), (3, 4, 16.0, 2)]
    X = np.array([[0.0], [1.0], [10.0], [11.0], [30.0]], dtype=np.float32)
    # pairs (0,1), (2,3) join; (1,2) at 81 joins two clusters of size 2 -> 4; (3,4) blocked
    assert restrict(oracle_mod, X, kl2_max_pre_size=2) == [(0, 1, 1.0, 2), (2, 3, 1.0, 2), (1, 2, 81.0, 4)]


def test_restrict_kl3_total_size(oracle_mod):
    X = np.array([[0.0], [1.0], [10.0], [11.0], [30.0]], dtype=np.float32)
    # (1,2) would make 4 > 3: blocked; (3,4) makes 3: allowed
    assert restrict(oracle_mod, X, kl3_max_size=3) == [(0, 1, 1.0, 2), (2, 3, 1.0, 2), (3, 4, 361.0, 3)]


def test_restrict_kl4_priority(oracle_mod):
    # Points: a pair at gap 1 (0,1), another pair at gap 1 (2,3) far away, and a
    # singleton 4 at gap 5 from row 3.  Tree in key order: (0,1)=1, (2,3)=1,
    # (3,4)=25, (1,2)=400.  KL4 = 2: joins touching a cluster of size < 2 first.
    X = np.array([[0.0], [1.0], [21.0], [22.0], [27.0]], dtype=np.float32)
    plain = restrict(oracle_mod, X, kl1_stop_clusters=2)
    assert plain == [(0, 1, 1.0, 2), (2, 3, 1.0, 2), (3, 4, 25.0, 3)]
    # With KL4 = 3 every pair met touches a cluster smaller than 3, so the order
    # is unchanged; with KL4 = 2 the pair (1,2) (sizes 2 and 3) waits for the
    # second walk, which it would reach last anyway.
    assert restrict(oracle_mod, X, kl1_stop_clusters=2, kl4_min_size=3) == plain
    assert restrict(oracle_mod, X, kl4_min_size=2) == [
        (0, 1, 1.0, 2), (2, 3, 1.0, 2), (3, 4, 25.0, 3), (1, 2, 400.0, 5)]


def test_restrict_kl4_reorders(oracle_mod):
    # Key order: (0,1)=1, (2,3)=1, (1,2)=4, (4,5)=100, then (3,4).  KL4 = 2 makes the
    # join of singletons 4,5 go before the join of two pairs (1,2).
    X = np.array([[0.0], [1.0], [3.0], [4.0], [30.0], [40.0]], dtype=np.float32)
    assert restrict(oracle_mod, X) == [
        (0, 1, 1.0, 2), (2, 3, 1.0, 2), (1, 2, 4.0, 4), (4, 5, 100.0, 2), (3, 4, 676.0, 6)]
    assert restrict(oracle_mod, X, kl4_min_size=2) == [
        (0, 1, 1.0, 2), (2, 3, 1.0, 2), (4, 5, 100.0, 2), (1, 2, 4.0, 4), (3, 4, 676.0, 6)]
    # with KL1 = 3 the priority decides which clusters survive
    assert restrict(oracle_mod, X, kl4_min_size=2, kl1_stop_clusters=3) == [
        (0, 1, 1.0, 2), (2, 3, 1.0, 2), (4, 5, 100.0, 2)]


def test_restrict_tree_vs_literal_counterexample(oracle_mod):
    # U (row 0) and V (row 6) are singletons either side of a 5-row cluster M.
    # KL3 = 5 blocks U-M and M-V.  The tree semantics never joins U and V; the
    # literal all-pairs reading joins them through the longer U-V pair.
    X = np.array([[0.0], [10.0], [11.0], [12.0], [13.0], [14.0], [24.0]], dtype=np.float32)
    tree = merges_list(oracle_mod.restrict_tree(oracle_mod.prim(X), 7, {"kl3_max_size": 5}))
    lit = merges_list(oracle_mod.restrict_literal(X, {"kl3_max_size": 5}))
    assert [(a, b) for a, b, _, _ in tree] == [(1, 2), (2, 3), (3, 4), (4, 5)]
    assert lit == tree + [(0, 6, 576.0, 2)]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_restrict_tree_equals_literal_for_cap_and_kl1(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    X = grid_points(rng, 150, 3, lim=96)
    tree = oracle_mod.prim(X)
    for cap in (0.0, 0.3, 0.7, 1.5):
        for kl1 in (0, 5, 40):
            r = {"max_join_dist": cap, "kl1_stop_clusters": kl1}
            assert np.array_equal(oracle_mod.restrict_tree(tree, 150, r), oracle_mod.restrict_literal(X, r))


@pytest.mark.parametrize("seed", [3, 4])
def test_restrict_invariants(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((400, 5)).astype(np.float32)
    tree = oracle_mod.prim(X)
    N = 400
    for r in ({"max_join_dist": 0.8, "kl3_max_size": 20},
              {"kl2_max_pre_size": 8, "kl1_stop_clusters": 30},
              {"kl4_min_size": 5, "kl3_max_size": 40, "max_join_dist": 1.2},
              {"kl4_min_size": 3, "kl1_stop_clusters": 50}):
        m = oracle_mod.restrict_tree(tree, N, r)
        cap = r.get("max_join_dist", 0)
        if cap:
            assert np.all(m["D"] <= cap * cap)
        parent = list(range(N))
        size = [1] * N

        def find(x):
            while parent[x] != x:
                x = parent[x]
            return x
        for a, b, s in zip(m["a"], m["b"], m["new_size"]):
            ra, rb = find(int(a)), find(int(b))
            assert ra != rb
            if r.get("kl2_max_pre_size"):
                assert size[ra] <= r["kl2_max_pre_size"] and size[rb] <= r["kl2_max_pre_size"]
            if r.get("kl3_max_size"):
                assert size[ra] + size[rb] <= r["kl3_max_size"]
            parent[ra] = rb
            size[rb] += size[ra]
            assert s == size[rb]
        assert N - len(m) >= r.get("kl1_stop_clusters", 0)
        tree_set = set(zip(tree["a"].tolist(), tree["b"].tolist()))
        assert all((int(a), int(b)) in tree_set for a, b in zip(m["a"], m["b"]))
        if not r.get("kl4_min_size"):
            assert np.all(np.diff(m["D"]) >= 0)


# ----------------------------------------------------------------------------------
# Labels
# ----------------------------------------------------------------------------------

def test_labels_partition_and_order(oracle_mod):
    rng = np.random.default_rng(8)
    X = rng.standard_normal((300, 3)).astype(np.float32)
    m = oracle_mod.restrict_tree(oracle_mod.prim(X), 300, {"max_join_dist": 0.35})
    lab, K = oracle_mod.labels(m, 300)
    # BFS over the accepted joins gives the same partition
    adj = {v: [] for v in range(300)}
    for a, b in zip(m["a"], m["b"]):
        adj[int(a)].append(int(b))
        adj[int(b)].append(int(a))
    seen = -np.ones(300, int)
    comps = 0
    for s in range(300):
        if seen[s] >= 0:
            continue
        stack = [s]
        seen[s] = comps
        while stack:
            v = stack.pop()
            for w in adj[v]:
                if seen[w] < 0:
                    seen[w] = comps
                    stack.append(w)
        comps += 1
    assert K == comps == 300 - len(m)
    assert np.array_equal(lab, seen)   # BFS from increasing seeds numbers clusters by smallest member
    first = [int(np.nonzero(lab == c)[0][0]) for c in range(K)]
    assert first == sorted(first)


# ----------------------------------------------------------------------------------
# other metrics (Eq. 1 is Euclidean; the paper allows another metric where a task needs one)
# ----------------------------------------------------------------------------------

def metric_by_hand(x, y, metric):
    """Python floats (binary64), feature order: the definitions written out."""
    s = 0.0
    for a, b in zip(x.tolist(), y.tolist()):
        e = float(a) - float(b)
        if metric == "manhattan":
            s = s + abs(e)
        else:
            s = max(s, abs(e))
    return s


def test_metric_values_by_hand(oracle_mod):
    # (0,0), (3,4), (1,-2): |3|+|4| = 7, |1|+|2| = 3, |2|+|6| = 8; max: 4, 2, 6
    X = np.array([[0, 0], [3, 4], [1, -2]], np.float32)
    i, j = [0, 0, 1], [1, 2, 2]
    assert oracle_mod.dist_pairs(X, i, j, metric="manhattan").tolist() == [7.0, 3.0, 8.0]
    assert oracle_mod.dist_pairs(X, i, j, metric="chebyshev").tolist() == [4.0, 2.0, 6.0]
    assert oracle_mod.dist_pairs(X, i, j).tolist() == [25.0, 5.0, 40.0]   # Euclidean unchanged


@pytest.mark.parametrize("metric", ["manhattan", "chebyshev"])
def test_metric_matches_definition_and_norm_order(oracle_mod, metric):
    rng = np.random.default_rng(21)
    X = (rng.standard_normal((60, 13)) * rng.uniform(0.1, 50, 13)).astype(np.float32)
    i, j = np.triu_indices(60, 1)
    D = oracle_mod.dist_pairs(X, i, j, metric=metric)
    want = [metric_by_hand(X[a], X[b], metric) for a, b in zip(i, j)]
    assert D.tolist() == want
    # |v|_inf <= |v|_2 <= |v|_1 <= sqrt(d) |v|_2 (a dropped term or sign would break one)
    L2 = np.sqrt(oracle_mod.dist_pairs(X, i, j))
    tol = 1e-12 * L2
    if metric == "manhattan":
        assert np.all(D >= L2 - tol) and np.all(D <= np.sqrt(13) * L2 + tol)
    else:
        assert np.all(D <= L2 + tol) and np.all(D >= L2 / np.sqrt(13) - tol)


@pytest.mark.parametrize("metric", ["manhattan", "chebyshev"])
def test_metric_knn_and_trees(oracle_mod, metric):
    rng = np.random.default_rng(22)
    X = grid_points(rng, 200, 4, lim=20)   # many equal distances: the tie-break decides
    idx, D = oracle_mod.knn(X, 5, metric=metric)
    for r in range(0, 200, 17):
        cand = sorted((metric_by_hand(X[r], X[c], metric), c) for c in range(200) if c != r)[:5]
        assert [c for _, c in cand] == idx[r].tolist()
        assert [v for v, _ in cand] == D[r].tolist()
    ref = oracle_mod.kruskal_allpairs(X, metric=metric)
    tree_checks(X, ref)
    for e in (oracle_mod.prim(X, metric=metric), oracle_mod.nnm_batched(X, 7, metric=metric)):
        assert np.array_equal(e, ref)
    # the lightest pair at every row is a tree edge (cut property under any metric)
    keys = set(zip(ref["a"].tolist(), ref["b"].tolist()))
    for r in range(200):
        c = int(idx[r, 0])
        assert (min(r, c), max(r, c)) in keys


def test_metric_cap_and_reported_length(oracle_mod):
    # three points on a line, 1.0 apart: D = 1 under every metric (squared: 1 as well),
    # but the cap compares D with c itself for L1/Linf and with c^2 for Euclidean
    X = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [1.0, 3.0]], np.float32)
    for metric in ("manhattan", "chebyshev"):
        tree = oracle_mod.kruskal_allpairs(X, metric=metric)
        m = oracle_mod.restrict_tree(tree, 4, {"max_join_dist": 1.0}, metric=metric)
        assert len(m) == 2 and np.all(m["dist"] == m["D"])   # length = D itself
        m2 = oracle_mod.restrict_tree(tree, 4, {"max_join_dist": 2.0}, metric=metric)
        assert len(m2) == 3   # the last pair is 2.0 away: D <= 2.0 admits it
    tree = oracle_mod.kruskal_allpairs(X)
    m = oracle_mod.restrict_tree(tree, 4, {"max_join_dist": 2.0})
    assert len(m) == 3 and m["D"][-1] == 4.0 and m["dist"][-1] == 2.0   # D <= 2.0^2
