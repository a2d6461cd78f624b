"""KL4 ("Problem settings": joins that touch a cluster smaller than KL4 take precedence)
pinned against a plain priority selector written here.

The oracle implements KL4 as two walks in key order: the first joins only pairs that
touch a cluster below KL4 and defers the others, the second walks the deferred pairs.
The rule itself is a priority: after every join, the next join is the smallest-key
admissible pair that touches a cluster below KL4, and only when there is none the
smallest-key admissible pair of any kind; the cap, KL1, KL2 and KL3 apply throughout.
The two agree because sizes only grow: a pair whose clusters are both at least KL4
stays so, and a pair a gate blocks stays blocked.  The selector below re-evaluates
every pending pair after every join (no walk, no deferral list), so a deferral taken
with stale sizes, a KL1 stop checked in the wrong place or a dropped second walk in
the oracle would make them differ.  Random small trees with ties, and every pair of
small point sets (the all-pairs reading), with every gate combination.
"""
import math

import numpy as np
import pytest

import oracle


def priority_selector(edges, N, r, euclidean=True):
    """Accepted merges (a, b, D, dist, new_size) under the priority reading of KL4,
    re-deciding from scratch after every join; ``edges`` in key order."""
    cap = r.get("max_join_dist", 0.0)
    cap2 = (cap * cap if euclidean else cap) if cap > 0 and math.isfinite(cap) else math.inf
    kl1, kl2, kl3, kl4 = (r.get(k, 0) for k in ("kl1_stop_clusters", "kl2_max_pre_size", "kl3_max_size",
                                               "kl4_min_size"))
    parent = list(range(N))
    size = [1] * N

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    def admissible(e):
        a, b, D = int(e["a"]), int(e["b"]), float(e["D"])
        ra, rb = find(a), find(b)
        if ra == rb or not D <= cap2:
            return None
        if kl2 > 0 and (size[ra] > kl2 or size[rb] > kl2):
            return None
        if kl3 > 0 and size[ra] + size[rb] > kl3:
            return None
        return ra, rb

    pending = list(range(len(edges)))
    K = N
    out = []
    while True:
        chosen = None
        if kl4 > 0:
            for q in pending:
                roots = admissible(edges[q])
                if roots and min(size[roots[0]], size[roots[1]]) < kl4:
                    chosen = (q, roots)
                    break
        if chosen is None:
            for q in pending:
                roots = admissible(edges[q])
                if roots:
                    chosen = (q, roots)
                    break
        if chosen is None:
            break
        if kl1 > 0 and K <= kl1:
            break
        q, (ra, rb) = chosen
        pending.remove(q)
        parent[rb] = ra
        size[ra] += size[rb]
        K -= 1
        e = edges[q]
        D = float(e["D"])
        out.append((int(e["a"]), int(e["b"]), D, math.sqrt(D) if euclidean else D, size[ra]))
    return out


def as_tuples(merges):
    return [(int(m["a"]), int(m["b"]), float(m["D"]), float(m["dist"]), int(m["new_size"])) for m in merges]


def random_tree(rng, N):
    """A random labelled tree with keys drawn from a few values (many ties), key-sorted."""
    e = np.zeros(N - 1, dtype=oracle.EDGE_DTYPE)
    order = rng.permutation(N)
    for q in range(1, N):
        u, v = int(order[q]), int(order[rng.integers(0, q)])
        e[q - 1] = (min(u, v), max(u, v), float(rng.integers(1, 6)) * 0.25)
    idx = np.lexsort((e["b"], e["a"], e["D"]))
    return e[idx]


def random_restrictions(rng, N):
    r = {}
    if rng.random() < 0.5:
        r["max_join_dist"] = float(rng.choice([0.6, 0.9, 1.1]))
    if rng.random() < 0.4:
        r["kl1_stop_clusters"] = int(rng.integers(1, max(2, N // 2)))
    if rng.random() < 0.4:
        r["kl2_max_pre_size"] = int(rng.integers(1, max(2, N // 3)))
    if rng.random() < 0.5:
        lo = r.get("kl2_max_pre_size", 0) + 1
        r["kl3_max_size"] = int(rng.integers(lo + 1, lo + max(3, N // 2)))
    r["kl4_min_size"] = int(rng.integers(2, 9)) if rng.random() < 0.85 else 0
    return r


def test_kl4_priority_on_random_trees():
    rng = np.random.default_rng(1402)
    differing_order = 0
    for _ in range(400):
        N = int(rng.integers(2, 40))
        tree = random_tree(rng, N)
        r = random_restrictions(rng, N)
        got = as_tuples(oracle.restrict_tree(tree, N, r))
        want = priority_selector(tree, N, r)
        assert got == want, (N, r)
        if r.get("kl4_min_size") and want != priority_selector(tree, N, {**r, "kl4_min_size": 0}):
            differing_order += 1
    # the cases exercise KL4: it changes the result in many of them
    assert differing_order > 50


def test_kl4_priority_on_all_pairs():
    """The all-pairs reading: the same rule with every pair as a candidate."""
    rng = np.random.default_rng(3789)
    for _ in range(60):
        N = int(rng.integers(2, 30))
        d = int(rng.integers(1, 4))
        X = (np.round(rng.uniform(0.0, 3.0, size=(N, d)) * 4.0) / 4.0).astype(np.float32)
        i, j = np.triu_indices(N, 1)
        D = oracle.dist_pairs(X, i, j)
        pairs = np.zeros(i.shape[0], dtype=oracle.EDGE_DTYPE)
        pairs["a"], pairs["b"], pairs["D"] = i, j, D
        pairs = pairs[np.lexsort((pairs["b"], pairs["a"], pairs["D"]))]
        r = random_restrictions(rng, N)
        assert as_tuples(oracle.restrict_literal(X, r)) == priority_selector(pairs, N, r), (N, r)


@pytest.mark.parametrize("metric", ["manhattan", "chebyshev"])
def test_kl4_priority_other_metrics(metric):
    rng = np.random.default_rng(7)
    for _ in range(40):
        N = int(rng.integers(2, 25))
        X = rng.uniform(0.0, 2.0, size=(N, 3)).astype(np.float32)
        tree = oracle.prim(X, metric=metric)
        r = random_restrictions(rng, N)
        got = as_tuples(oracle.restrict_tree(tree, N, r, metric=metric))
        assert got == priority_selector(tree, N, r, euclidean=False), (N, r)
