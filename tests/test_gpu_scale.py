"""GPU parity at the workloads' full sizes, in the launch configuration bench.py times.

The oracle cannot build a 2M-row dendrogram here, so at full size the checks are:
- sampled rows: exact k nearest neighbours (indices and binary64 distances) against the
  oracle's brute force on the same rows;
- the tree: N-1 edges in strictly increasing key order forming one spanning tree (one
  component, hence no cycle), sampled edges' D equal to the oracle's canonical D, and
  each sampled row's 1-NN edge in the tree (the lightest edge at a vertex belongs to the
  unique minimum spanning tree);
- the restrictions and labels: the oracle's restriction walk and labels on the GPU's
  tree equal the GPU's merges and labels element by element.
The 262,144-row workload also gets the full oracle dendrogram (dense Prim on the host
cores, about a minute), and a subset of the batched workload's instances spanning its
size range (up to 65,482 rows, d from 4 to 25) is clustered in one batched context and
compared instance by instance with the full oracle.
"""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nnm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_3789_gb300 import build, nnm as binding
    build.build()
    binding.load_library()
    return binding


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def dev(X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()


def spanning(tree, N):
    """True iff the edges form one spanning tree of the N rows: N-1 edges joining all rows
    into one component (then no edge closes a cycle)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    if tree.shape[0] != N - 1:
        return False
    g = coo_matrix((np.ones(N - 1), (tree["a"].astype(np.int64), tree["b"].astype(np.int64))), shape=(N, N))
    return connected_components(g, directed=False)[0] == 1


def key_order_ok(tree):
    a, b, D = tree["a"].astype(np.int64), tree["b"].astype(np.int64), tree["D"]
    nxt = (D[1:] > D[:-1]) | ((D[1:] == D[:-1]) & ((a[1:] > a[:-1]) | ((a[1:] == a[:-1]) & (b[1:] > b[:-1]))))
    return bool(np.all(a < b)) and bool(np.all(nxt))


@pytest.mark.parametrize("workload,precisions", [
    ("nnm_n262144_d16", ["bf16x3", "fp32"]),
    ("nnm_n2097152_d25", ["bf16x3"]),
    ("nnm_n1048576_d25_ties", ["bf16x3", "fp16"]),
])
def test_full_size_sampled_rows_tree_and_restrictions(nnm, orc, workload, precisions):
    from paper_1402_3789_gb300.inputs import WORKLOADS, make
    w = WORKLOADS[workload]
    X = make(workload)
    N = X.shape[0]
    Xd = dev(X)
    rng = np.random.default_rng(123)
    # 10,000 sampled rows at the paper-scale sizes (the oracle's brute force on the host
    # cores takes about 20 s at N = 2M), 2,000 at the smaller one
    rows = np.sort(rng.choice(N, size=10_000 if N >= 1_000_000 else 2_000, replace=False))
    oi, oD = orc.knn(X, 8, queries=rows)
    trees = []
    for p in precisions:
        ctx = nnm.nnm_create(Xd, precision=p)
        try:
            idx, D = nnm.nnm_nearest(ctx, 8)
            idx = idx.cpu().numpy().view(np.uint32)[rows]
            D = D.cpu().numpy()[rows]
            assert np.array_equal(idx, oi), p
            assert np.array_equal(D, oD), p
            res = nnm.nnm_cluster(ctx, dict(w.restrictions))
            tree = nnm.nnm_get_tree(ctx)
            merges = res.merges()
            lab = res.labels.cpu().numpy()
        finally:
            nnm.nnm_destroy(ctx)
        assert tree.shape[0] == N - 1
        assert key_order_ok(tree)
        assert spanning(tree, N), p
        sel = rng.choice(N - 1, size=2000, replace=False)
        assert np.array_equal(tree["D"][sel], orc.dist_pairs(X, tree["a"][sel], tree["b"][sel]))
        keys = set(zip(tree["a"].tolist(), tree["b"].tolist()))
        for i, j in zip(rows.tolist(), oi[:, 0].tolist()):
            assert (min(i, j), max(i, j)) in keys
        om = orc.restrict_tree(tree, N, w.restrictions)
        olab, oK = orc.labels(om, N)
        assert np.array_equal(merges, om), p
        assert np.array_equal(lab, olab) and res.n_clusters == oK, p
        trees.append(tree)
    for t in trees[1:]:
        assert np.array_equal(t, trees[0])   # every precision gives the same tree


def test_batched_instances_full_oracle(nnm, orc):
    from paper_1402_3789_gb300.inputs import batched_instances
    inst = [x for x in batched_instances() if x.shape[0] <= 12000][:6]
    assert len(inst) == 6
    for X in inst:
        otree, om, olab, oK = orc.cluster(X, {})
        for p in ("bf16x3", "fp32"):
            ctx = nnm.nnm_create(dev(X), precision=p)
            try:
                res = nnm.nnm_cluster(ctx, {})
                tree = nnm.nnm_get_tree(ctx)
                assert np.array_equal(tree, otree), (p, X.shape)
                assert np.array_equal(res.merges(), om)
                assert np.array_equal(res.labels.cpu().numpy(), olab) and res.n_clusters == oK
            finally:
                nnm.nnm_destroy(ctx)


def test_n262144_full_oracle_dendrogram(nnm, orc):
    """The 262,144-row workload against the oracle's own dendrogram: tree, merges,
    labels and cluster count element by element, FP32 and split-BF16 candidates."""
    from paper_1402_3789_gb300.inputs import WORKLOADS, make
    w = WORKLOADS["nnm_n262144_d16"]
    X = make("nnm_n262144_d16")
    N = X.shape[0]
    otree, om, olab, oK = orc.cluster(X, dict(w.restrictions))
    assert spanning(otree, N)
    Xd = dev(X)
    for p in ("bf16x3", "fp32"):
        ctx = nnm.nnm_create(Xd, precision=p)
        try:
            res = nnm.nnm_cluster(ctx, dict(w.restrictions))
            tree = nnm.nnm_get_tree(ctx)
            assert np.array_equal(tree, otree), p
            assert np.array_equal(res.merges(), om), p
            assert np.array_equal(res.labels.cpu().numpy(), olab) and res.n_clusters == oK, p
        finally:
            nnm.nnm_destroy(ctx)


def batched_subset():
    """A seeded subset of the batched workload's 512 instances that spans its range: the
    three largest (64-65k rows), the largest with d = 25 above 30,000 rows, the first with
    d = 4 and with d = 25, the two smallest, and four more drawn at random; kept in the
    workload's order."""
    from paper_1402_3789_gb300.inputs import batched_instances
    xs = batched_instances()
    n = np.array([x.shape[0] for x in xs])
    d = np.array([x.shape[1] for x in xs])
    pick = set(np.argsort(-n)[:3].tolist())
    pick.add(int(np.argmax(np.where(d == 25, n, 0))))
    pick.add(int(np.where(d == 4)[0][0]))
    pick.add(int(np.where(d == 25)[0][0]))
    pick.update(np.argsort(n)[:2].tolist())
    rng = np.random.default_rng(2024)
    rest = [i for i in range(len(xs)) if i not in pick]
    pick.update(rng.choice(rest, size=4, replace=False).tolist())
    idx = sorted(pick)
    return [xs[i] for i in idx]


def test_batched_context_at_the_workload_sizes(nnm, orc):
    """One batched context holding instances of 1k to 65k rows and d = 4..25: every
    instance's tree, merges and labels equal the full oracle's (labels of instance b are
    the oracle's plus the clusters of the instances before it)."""
    inst = batched_subset()
    assert max(x.shape[0] for x in inst) > 60000 and min(x.shape[0] for x in inst) < 1100
    assert {4, 25} <= {x.shape[1] for x in inst}
    otrees = [orc.prim(x) for x in inst]
    for p in ("bf16x3", "fp32"):
        for restr in ({}, {"max_join_dist": 0.8, "kl1_stop_clusters": 10},
                      {"kl4_min_size": 5, "kl3_max_size": 5000}):
            ctx = nnm.nnm_create_batched([dev(x) for x in inst], precision=p)
            try:
                off = ctx.offsets
                res = nnm.nnm_cluster(ctx, restr)
                tree = nnm.nnm_get_tree(ctx)
                merges = res.merges()
                lab = res.labels.cpu().numpy()
            finally:
                nnm.nnm_destroy(ctx)
            assert tree.shape[0] == off[-1] - len(inst)
            inst_of = np.searchsorted(np.array(off), np.arange(off[-1]), side="right") - 1
            k_before = 0
            for b, X in enumerate(inst):
                lo = off[b]
                om = orc.restrict_tree(otrees[b], X.shape[0], restr)
                olab, oK = orc.labels(om, X.shape[0])
                t = tree[inst_of[tree["a"]] == b].copy()
                t["a"] -= lo
                t["b"] -= lo
                assert np.array_equal(t, otrees[b]), (p, b, X.shape)
                m = merges[inst_of[merges["a"]] == b].copy()
                m["a"] -= lo
                m["b"] -= lo
                assert np.array_equal(m, om), (p, restr, b)
                assert np.array_equal(lab[lo:off[b + 1]], olab + k_before), (p, restr, b)
                k_before += oK
            assert res.n_clusters == k_before
