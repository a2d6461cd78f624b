"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Exact results (indices, binary64 distances, merge tree, merges, labels) must be equal
element by element: every decision of the method is taken on the canonical binary64
squared distance with the (D, min, max) tie-break, which both sides compute the same
way.  Inputs are the seeded mixtures of paper_1402_3789_gb300.inputs at sizes that span
several row tiles (256 rows) and column tiles, with ragged tails.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PRECISIONS = ["fp32", "bf16", "fp16", "bf16x3"]


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


def make(name, n, seed=None):
    from paper_1402_3789_gb300.inputs import make as mk
    return mk(name, n=n, seed=seed)


def dev(X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()


def run_nearest(nnm, X, k, precision, **opt):
    ctx = nnm.nnm_create(dev(X), precision=precision, **opt)
    try:
        idx, D = nnm.nnm_nearest(ctx, k)
        return idx.cpu().numpy().view(np.uint32), D.cpu().numpy(), nnm.nnm_get_stats(ctx)
    finally:
        nnm.nnm_destroy(ctx)


def run_cluster(nnm, X, restr, precision, **opt):
    ctx = nnm.nnm_create(dev(X), precision=precision, **opt)
    try:
        res = nnm.nnm_cluster(ctx, restr)
        tree = nnm.nnm_get_tree(ctx)
        return tree, res.merges(), res.labels.cpu().numpy(), res.n_clusters, nnm.nnm_get_stats(ctx)
    finally:
        nnm.nnm_destroy(ctx)


# ----------------------------------------------------------------------------------
# nearest neighbours
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n,d,k", [(4096, 8, 1), (4096, 8, 8), (3001, 25, 5), (777, 3, 16), (300, 32, 2),
                                   (1000, 1, 4), (5000, 16, 12)])
def test_nearest_matches_oracle(nnm, orc, precision, n, d, k):
    if precision == "bf16x3" and d > 30:
        pytest.skip("the split form takes d <= 30")
    rng = np.random.default_rng(n + d)
    X = (rng.standard_normal((n, d)) * rng.uniform(0.5, 3, d) + rng.integers(0, 5, (n, 1))).astype(np.float32)
    idx, D, st = run_nearest(nnm, X, k, precision)
    oi, oD = orc.knn(X, k)
    assert np.array_equal(idx, oi)
    assert np.array_equal(D, oD)
    if precision == "fp32":
        assert st["max_rel_err"] <= (d + 2) * 2.0 ** -24 * 1.01


@pytest.mark.parametrize("precision", PRECISIONS)
def test_nearest_paper_mixture_small(nnm, orc, precision):
    X = make("nnm_n4096_d8", 4096)
    idx, D, _ = run_nearest(nnm, X, 4, precision)
    oi, oD = orc.knn(X, 4)
    assert np.array_equal(idx, oi) and np.array_equal(D, oD)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_nearest_ties_and_duplicates(nnm, orc, precision):
    # the tie-stress recipe (1/64 grid, 2% duplicates) at a small size: many equal D
    X = make("nnm_n1048576_d25_ties", 6000)
    idx, D, st = run_nearest(nnm, X, 6, precision)
    oi, oD = orc.knn(X, 6)
    assert np.array_equal(idx, oi) and np.array_equal(D, oD)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_nearest_all_identical_rows(nnm, orc, precision):
    X = np.ones((700, 5), dtype=np.float32) * 3.25
    idx, D, _ = run_nearest(nnm, X, 3, precision)
    oi, oD = orc.knn(X, 3)
    assert np.array_equal(idx, oi) and np.array_equal(D, oD)


@pytest.mark.parametrize("precision", ["bf16", "fp16", "bf16x3"])
def test_nearest_large_offset_and_spread(nnm, orc, precision):
    # large common offset (removed by centring) and features of very different scale:
    # the rounding radii are large, so the completeness test does real work
    rng = np.random.default_rng(3)
    X = (1000.0 + rng.standard_normal((3000, 12)) * np.geomspace(1e-3, 30, 12)).astype(np.float32)
    idx, D, st = run_nearest(nnm, X, 5, precision)
    oi, oD = orc.knn(X, 5)
    assert np.array_equal(idx, oi) and np.array_equal(D, oD)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_nearest_forced_column_splits(nnm, orc, precision):
    X = make("nnm_n262144_d16", 9000)
    for s in (1, 3, 7):
        idx, D, _ = run_nearest(nnm, X, 3, precision, col_split=s)
        oi, oD = orc.knn(X, 3)
        assert np.array_equal(idx, oi) and np.array_equal(D, oD)


# ----------------------------------------------------------------------------------
# merge tree, restrictions, labels
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("precision", PRECISIONS)
def test_cluster_full_tree_n4096(nnm, orc, precision):
    X = make("nnm_n4096_d8", 4096)
    tree, merges, labels, K, st = run_cluster(nnm, X, None, precision)
    otree, omerges, olabels, oK = orc.cluster(X, None)
    assert np.array_equal(tree, otree)
    assert np.array_equal(merges, omerges)
    assert K == oK == 1
    assert np.array_equal(labels, olabels)


RESTRICTIONS = [
    {"max_join_dist": 0.8},
    {"kl1_stop_clusters": 37},
    {"max_join_dist": 1.0, "kl1_stop_clusters": 20},
    {"kl2_max_pre_size": 40},
    {"kl3_max_size": 100, "max_join_dist": 1.3},
    {"kl4_min_size": 6, "kl3_max_size": 200},
    {"kl4_min_size": 12, "kl1_stop_clusters": 50, "kl2_max_pre_size": 30, "kl3_max_size": 90},
]


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("restr", RESTRICTIONS, ids=[str(i) for i in range(len(RESTRICTIONS))])
def test_cluster_restrictions(nnm, orc, precision, restr):
    X = make("nnm_n4096_d8", 5000, seed=11)
    tree, merges, labels, K, _ = run_cluster(nnm, X, restr, precision)
    otree, omerges, olabels, oK = orc.cluster(X, restr)
    assert np.array_equal(tree, otree)
    assert np.array_equal(merges, omerges)
    assert K == oK
    assert np.array_equal(labels, olabels)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_cluster_ties_tree(nnm, orc, precision):
    X = make("nnm_n1048576_d25_ties", 3000)
    tree, merges, labels, K, _ = run_cluster(nnm, X, {"max_join_dist": 0.5}, precision)
    otree, omerges, olabels, oK = orc.cluster(X, {"max_join_dist": 0.5})
    assert np.array_equal(tree, otree)
    assert np.array_equal(merges, omerges) and K == oK and np.array_equal(labels, olabels)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_cluster_ragged_and_tiny(nnm, orc, precision):
    rng = np.random.default_rng(5)
    for n, d in ((2, 3), (3, 1), (257, 7), (1023, 25), (2049, 2)):
        X = rng.standard_normal((n, d)).astype(np.float32)
        tree, merges, labels, K, _ = run_cluster(nnm, X, None, precision)
        otree, omerges, olabels, oK = orc.cluster(X, None)
        assert np.array_equal(tree, otree), (n, d)
        assert np.array_equal(merges, omerges) and K == oK and np.array_equal(labels, olabels)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_cluster_cut_chains_and_extremes(nnm, orc, precision):
    """The cap/KL1-only restriction step (a cut plus new sizes by halving rank ranges)
    on the shapes that make a dendrogram deep: rows on a line with growing gaps (each
    join adds one row to one cluster: new sizes 2..N), a growing spiral, all rows equal,
    and restrictions that admit nothing, everything, or stop at KL1 = N - 1."""
    rng = np.random.default_rng(17)
    n = 3000
    line = np.zeros((n, 3), np.float32)
    line[:, 0] = np.cumsum(np.linspace(0.01, 1.0, n)).astype(np.float32)
    line = line[rng.permutation(n)]
    t = np.linspace(0, 40, 2500)
    spiral = np.stack([t * np.cos(t), t * np.sin(t), 0.1 * t], 1).astype(np.float32)
    same = np.ones((700, 5), np.float32)
    cases = [(line, None), (line, {"kl1_stop_clusters": 100}), (line, {"max_join_dist": 1e-9}),
             (line, {"kl1_stop_clusters": n - 1}), (line, {"kl1_stop_clusters": n + 5}),
             (spiral, None), (spiral, {"max_join_dist": 0.5, "kl1_stop_clusters": 3}),
             (same, None), (same, {"kl1_stop_clusters": 2})]
    for i, (X, restr) in enumerate(cases):
        tree, merges, labels, K, _ = run_cluster(nnm, X, restr, precision)
        otree, omerges, olabels, oK = orc.cluster(X, restr)
        assert np.array_equal(tree, otree), i
        assert np.array_equal(merges, omerges), i
        assert K == oK and np.array_equal(labels, olabels), i
    # the line's dendrogram is one chain: every join grows the same cluster
    _, merges, _, _, _ = run_cluster(nnm, line, None, precision)
    assert np.array_equal(np.sort(merges["new_size"]), np.arange(2, n + 1))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_cluster_freeze_at_cap_keeps_the_restricted_result(nnm, orc, precision):
    X = make("nnm_n262144_d16", 8000)
    restr = {"max_join_dist": 1.5, "kl1_stop_clusters": 200}
    tree, merges, labels, K, _ = run_cluster(nnm, X, restr, precision, freeze_at_cap=True)
    otree, omerges, olabels, oK = orc.cluster(X, restr)
    assert np.array_equal(merges, omerges) and K == oK and np.array_equal(labels, olabels)
    cut = otree[otree["D"] <= 1.5 * 1.5]
    assert np.array_equal(np.sort(tree[tree["D"] <= 2.25], order=["D", "a", "b"]), cut)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_cluster_mixture_n20000(nnm, orc, precision):
    X = make("nnm_n262144_d16", 20000)
    restr = {"max_join_dist": 1.5, "kl1_stop_clusters": 200}
    tree, merges, labels, K, st = run_cluster(nnm, X, restr, precision)
    otree, omerges, olabels, oK = orc.cluster(X, restr)
    assert np.array_equal(tree, otree)
    assert np.array_equal(merges, omerges) and K == oK and np.array_equal(labels, olabels)


# ----------------------------------------------------------------------------------
# errors
# ----------------------------------------------------------------------------------

def test_errors(nnm):
    X = np.random.default_rng(0).standard_normal((100, 4)).astype(np.float32)
    with pytest.raises(nnm.NNMError) as e:
        nnm.nnm_create(dev(np.zeros((10, 31), np.float32)), precision="bf16x3")
    assert e.value.status == nnm.NNM_EUNSUPPORTED
    Xbad = X.copy()
    Xbad[7, 2] = np.nan
    with pytest.raises(nnm.NNMError) as e:
        nnm.nnm_create(dev(Xbad))
    assert e.value.status == nnm.NNM_ENONFINITE
    Xbad[7, 2] = np.inf
    with pytest.raises(nnm.NNMError):
        nnm.nnm_create(dev(Xbad))
    ctx = nnm.nnm_create(dev(X))
    try:
        for k in (0, 17, 100):
            with pytest.raises(nnm.NNMError) as e:
                nnm.nnm_nearest(ctx, k)
            assert e.value.status == nnm.NNM_EINVAL
        with pytest.raises(nnm.NNMError) as e:
            nnm.nnm_cluster(ctx, {"kl2_max_pre_size": 10, "kl3_max_size": 10})
        assert e.value.status == nnm.NNM_EINVAL
        with pytest.raises(nnm.NNMError) as e:
            nnm.nnm_cluster(ctx, {"kl1_stop_clusters": -1})
        assert e.value.status == nnm.NNM_EINVAL
        with pytest.raises(nnm.NNMError) as e:
            nnm.nnm_cluster(ctx, {"semantics": 3})
        assert e.value.status == nnm.NNM_EINVAL
        # the context stays usable after rejected calls
        idx, D = nnm.nnm_nearest(ctx, 2)
        assert idx.shape == (100, 2)
    finally:
        nnm.nnm_destroy(ctx)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_candidates_are_tight(nnm, precision):
    # The exact re-rank would repair any candidate list (through the collect pass), so
    # check separately that the sweep's values are close: few re-ranked pairs per row,
    # no overflowing row, and a candidate error of the size the arithmetic predicts.
    X = make("nnm_n4096_d8", 4096)
    _, _, st = run_nearest(nnm, X, 4, precision)
    assert st["rows_overflowed"] == 0
    assert st["rerank_pairs"] <= 12 * 4096
    bound = {"fp32": 10 * 2.0 ** -24, "fp16": 0.05, "bf16": 0.25, "bf16x3": 0.01}[precision]
    assert st["max_rel_err"] <= bound


@pytest.mark.parametrize("precision", PRECISIONS)
def test_tile_pruning_skips_far_tiles_and_changes_nothing(nnm, orc, precision):
    # Well separated blobs: the bounding-sphere bound must skip most column tiles,
    # and the exact results must equal both the unpruned run and the oracle.
    rng = np.random.default_rng(17)
    centres = rng.uniform(0, 400, (24, 6))
    X = (centres[rng.integers(0, 24, 9000)] + rng.standard_normal((9000, 6))).astype(np.float32)
    idx_p, D_p, st_p = run_nearest(nnm, X, 4, precision)
    idx_u, D_u, st_u = run_nearest(nnm, X, 4, precision, tile_pruning=False)
    # one column range per row tile: the skip count then depends little on timing
    idx_1, D_1, st_1 = run_nearest(nnm, X, 4, precision, col_split=1)
    oi, oD = orc.knn(X, 4)
    assert np.array_equal(idx_p, oi) and np.array_equal(D_p, oD)
    assert np.array_equal(idx_u, oi) and np.array_equal(D_u, oD)
    assert np.array_equal(idx_1, oi) and np.array_equal(D_1, oD)
    assert st_u["tiles_skipped"] == 0
    assert st_p["tiles_skipped"] > 0
    assert st_1["tiles_skipped"] > 0.4 * (st_1["tiles_skipped"] + st_1["tiles_swept"])
    tree_p, m_p, lab_p, K_p, _ = run_cluster(nnm, X, {"max_join_dist": 3.0}, precision)
    otree, om, olab, oK = orc.cluster(X, {"max_join_dist": 3.0})
    assert np.array_equal(tree_p, otree) and np.array_equal(m_p, om) and np.array_equal(lab_p, olab)


# ----------------------------------------------------------------------------------
# batched contexts: many independent instances in one context
# ----------------------------------------------------------------------------------

def batched_cases():
    from paper_1402_3789_gb300.inputs import batched_instances
    inst = [x for x in batched_instances(count=40, seed=11, n_lo=300, n_hi=3000)][:9]
    rng = np.random.default_rng(5)
    inst.insert(3, rng.standard_normal((2, 5)).astype(np.float32))     # two rows
    inst.insert(6, rng.standard_normal((3, 12)).astype(np.float32))    # three rows
    inst.append(np.round(rng.standard_normal((700, 6)) * 4).astype(np.float32) / 4)   # ties
    return inst


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("restr", [{}, {"max_join_dist": 1.2}, {"kl1_stop_clusters": 4},
                                   {"kl4_min_size": 5, "kl3_max_size": 400},
                                   {"kl1_stop_clusters": 3, "kl2_max_pre_size": 150}],
                         ids=["none", "cap", "kl1", "kl4kl3", "kl1kl2"])
def test_batched_context_equals_each_instance_alone(nnm, orc, precision, restr):
    inst = batched_cases()
    ctx = nnm.nnm_create_batched([dev(x) for x in inst], precision=precision)
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
    total_k = 0
    for b, X in enumerate(inst):
        lo = off[b]
        otree, om, olab, oK = orc.cluster(X, restr)
        t = tree[inst_of[tree["a"]] == b].copy()
        t["a"] -= lo
        t["b"] -= lo
        assert np.array_equal(t, otree), b
        m = merges[inst_of[merges["a"]] == b].copy()
        m["a"] -= lo
        m["b"] -= lo
        assert np.array_equal(m, om), b
        # labels: the same partition, numbered in the same order of smallest members
        lb = lab[lo:off[b + 1]]
        _, dense = np.unique(lb, return_inverse=True)
        first = {}
        relabel = np.array([first.setdefault(v, len(first)) for v in dense])
        assert np.array_equal(relabel, olab), b
        total_k += oK
    assert res.n_clusters == total_k


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_batched_nearest_stays_inside_instances(nnm, orc, precision):
    inst = [x for x in batched_cases() if x.shape[0] > 8]
    ctx = nnm.nnm_create_batched([dev(x) for x in inst], precision=precision)
    try:
        off = ctx.offsets
        idx, D = nnm.nnm_nearest(ctx, 4)
        idx = idx.cpu().numpy().view(np.uint32)
        D = D.cpu().numpy()
        with pytest.raises(nnm.NNMError):
            nnm.nnm_nearest(ctx, min(x.shape[0] for x in inst))   # k must be < the smallest instance
    finally:
        nnm.nnm_destroy(ctx)
    for b, X in enumerate(inst):
        oi, oD = orc.knn(X, 4)
        assert np.array_equal(idx[off[b]:off[b + 1]] - off[b], oi), b
        assert np.array_equal(D[off[b]:off[b + 1]], oD), b


# ----------------------------------------------------------------------------------
# other metrics: Manhattan and Chebyshev on the FP32 direct path
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("metric", ["manhattan", "chebyshev"])
@pytest.mark.parametrize("case", ["mixture", "grid_ties", "wide_offsets"])
def test_other_metrics_nearest_and_tree(nnm, orc, metric, case):
    rng = np.random.default_rng(31)
    if case == "mixture":
        X = make("nnm_n4096_d8", 3001, seed=7)
    elif case == "grid_ties":
        X = (rng.integers(0, 6, (2500, 5)) / 4.0).astype(np.float32)   # many equal distances
    else:
        X = (rng.standard_normal((1800, 11)) * rng.uniform(0.01, 300, 11) + 1000).astype(np.float32)
    ctx = nnm.nnm_create(dev(X), precision="fp32", metric=metric)
    try:
        idx, D = nnm.nnm_nearest(ctx, 6)
        idx = idx.cpu().numpy().view(np.uint32)
        D = D.cpu().numpy()
        restr = {"max_join_dist": 2.5, "kl4_min_size": 4}
        res = nnm.nnm_cluster(ctx, restr)
        tree = nnm.nnm_get_tree(ctx)
        merges = res.merges()
        lab = res.labels.cpu().numpy()
    finally:
        nnm.nnm_destroy(ctx)
    oi, oD = orc.knn(X, 6, metric=metric)
    assert np.array_equal(idx, oi) and np.array_equal(D, oD)
    otree, om, olab, oK = orc.cluster(X, restr, metric=metric)
    assert np.array_equal(tree, otree)
    assert np.array_equal(merges, om)
    assert np.array_equal(lab, olab) and res.n_clusters == oK


@pytest.mark.parametrize("metric", ["manhattan", "chebyshev"])
def test_other_metrics_batched_and_pruning(nnm, orc, metric):
    rng = np.random.default_rng(32)
    inst = [make("nnm_n4096_d8", 900, seed=s) for s in range(3)] + [rng.standard_normal((5, 8)).astype(np.float32)]
    ctx = nnm.nnm_create_batched([dev(x) for x in inst], precision="fp32", metric=metric)
    try:
        off = ctx.offsets
        nnm.nnm_cluster(ctx, {})
        tree = nnm.nnm_get_tree(ctx)
    finally:
        nnm.nnm_destroy(ctx)
    inst_of = np.searchsorted(np.array(off), np.arange(off[-1]), side="right") - 1
    for b, X in enumerate(inst):
        t = tree[inst_of[tree["a"]] == b].copy()
        t["a"] -= off[b]
        t["b"] -= off[b]
        assert np.array_equal(t, orc.prim(X, metric=metric)), b
    # well separated blobs: the Euclidean sphere bound prunes for these metrics too
    centres = rng.uniform(0, 400, (16, 6))
    X = (centres[rng.integers(0, 16, 6000)] + rng.standard_normal((6000, 6))).astype(np.float32)
    ctx = nnm.nnm_create(dev(X), precision="fp32", metric=metric, col_split=1)
    try:
        idx, D = nnm.nnm_nearest(ctx, 3)
        st = nnm.nnm_get_stats(ctx)
    finally:
        nnm.nnm_destroy(ctx)
    oi, oD = orc.knn(X, 3, metric=metric)
    assert np.array_equal(idx.cpu().numpy().view(np.uint32), oi) and np.array_equal(D.cpu().numpy(), oD)
    assert st["tiles_skipped"] > 0.4 * (st["tiles_skipped"] + st["tiles_swept"])


def test_other_metrics_need_the_fp32_path(nnm):
    X = dev(np.zeros((64, 4), np.float32))
    for p in ("bf16", "fp16", "bf16x3"):
        with pytest.raises(nnm.NNMError):
            nnm.nnm_create(X, precision=p, metric="manhattan")


# ----------------------------------------------------------------------------------
# KL2 / KL3 without KL4: safe edges joined in parallel, the walk over the others only
# ----------------------------------------------------------------------------------

def _chain(n):
    """Rows on a line with growing gaps: one long chain in the merge tree (every join
    adds one row to the big cluster), the case where most edges are unsafe."""
    x = np.cumsum(np.linspace(0.01, 1.0, n)).astype(np.float32)
    return np.stack([x, np.zeros_like(x)], axis=1)


@pytest.mark.parametrize("restr", [
    {"kl3_max_size": 700}, {"kl2_max_pre_size": 300}, {"kl3_max_size": 900, "kl2_max_pre_size": 250},
    {"kl3_max_size": 500, "kl1_stop_clusters": 30}, {"kl3_max_size": 800, "max_join_dist": 1.3},
    {"kl2_max_pre_size": 1, "kl3_max_size": 2}, {"kl3_max_size": 100000},
], ids=["kl3", "kl2", "kl2kl3", "kl3kl1", "kl3cap", "tiny", "kl3large"])
@pytest.mark.parametrize("data", ["mixture", "chain", "ties"])
def test_size_gates_without_kl4_match_the_oracle(nnm, orc, restr, data):
    if data == "mixture":
        from paper_1402_3789_gb300.inputs import make
        X = make("nnm_n4096_d8", n=30000, seed=77)
    elif data == "chain":
        X = _chain(5000)
    else:
        rng = np.random.default_rng(3)
        X = (np.round(rng.uniform(0, 6, size=(8000, 3)) * 4) / 4).astype(np.float32)
    N = X.shape[0]
    ctx = nnm.nnm_create(dev(X), precision="fp32")
    try:
        res = nnm.nnm_cluster(ctx, restr)
        tree = nnm.nnm_get_tree(ctx)
    finally:
        nnm.nnm_destroy(ctx)
    om = orc.restrict_tree(tree, N, restr)
    olab, oK = orc.labels(om, N)
    assert np.array_equal(res.merges(), om)
    assert np.array_equal(res.labels.cpu().numpy(), olab) and res.n_clusters == oK


@pytest.mark.parametrize("restr", [{}, {"max_join_dist": 1.0}, {"kl1_stop_clusters": 5},
                                   {"max_join_dist": 1.4, "kl1_stop_clusters": 9}], ids=["none", "cap", "kl1", "capkl1"])
def test_batched_many_small_instances_walk_each_instance(nnm, orc, restr):
    """64 instances, the largest under 1/32 of the rows: the restriction step walks each
    instance in its own CTA instead of cutting the whole batch."""
    from paper_1402_3789_gb300.inputs import batched_instances
    inst = batched_instances(count=64, seed=29, n_lo=150, n_hi=480, d_lo=3, d_hi=20)
    assert max(x.shape[0] for x in inst) * 32 < sum(x.shape[0] for x in inst)
    ctx = nnm.nnm_create_batched([dev(x) for x in inst], precision="bf16x3")
    try:
        off = ctx.offsets
        res = nnm.nnm_cluster(ctx, restr)
        merges = res.merges()
        lab = res.labels.cpu().numpy()
    finally:
        nnm.nnm_destroy(ctx)
    inst_of = np.searchsorted(np.array(off), np.arange(off[-1]), side="right") - 1
    k_before = 0
    for b, X in enumerate(inst):
        lo = off[b]
        _, om, olab, oK = orc.cluster(X, restr)
        m = merges[inst_of[merges["a"]] == b].copy()
        m["a"] -= lo
        m["b"] -= lo
        assert np.array_equal(m, om), b
        assert np.array_equal(lab[lo:off[b + 1]], olab + k_before), b
        k_before += oK
    assert res.n_clusters == k_before
