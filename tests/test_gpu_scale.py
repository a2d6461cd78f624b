"""GPU parity at the workloads' full sizes, in the launch configuration bench.py times.

The oracle cannot build a 2M-row dendrogram here, so at full size the checks are:
- sampled rows: exact k nearest neighbours (indices and binary64 distances) against the
  oracle's brute force on the same rows;
- the tree: N-1 edges in strictly increasing key order, sampled edges' D equal to the
  oracle's canonical D, and each sampled row's 1-NN edge in the tree (the lightest edge
  at a vertex belongs to the unique minimum spanning tree);
- the restrictions and labels: the oracle's restriction walk and labels on the GPU's
  tree equal the GPU's merges and labels element by element.
Smaller instances of the batched workload get the full oracle dendrogram.
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
