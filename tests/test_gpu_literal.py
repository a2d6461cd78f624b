"""GPU parity of the restrictions in the paper's all-pairs reading (semantics = 1): the
gates act on every pair in key order, as the paper's batched procedure walks its P
minimal pairs.  The GPU's batches (pairs that cross two clusters and pass every gate at
the batch start, cut by FP32 value, kept by binary64 D, walked in key order) must give
the oracle's or_restrict_literal merges and labels element by element: the U-M-V case
where the all-pairs reading joins two clusters through a pair outside the tree, cap and
KL1 alone (where both readings agree), every size gate, KL4's two phases, KL1 stops,
ties, the Manhattan metric, and one 20,000-row case.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

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


def literal_gpu(nnm, X, restr, precision="fp32", metric="euclidean"):
    ctx = nnm.nnm_create(torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda(), precision=precision,
                         metric=metric)
    try:
        res = nnm.nnm_cluster(ctx, {**restr, "semantics": 1})
        return res.merges(), res.labels.cpu().numpy(), res.n_clusters
    finally:
        nnm.nnm_destroy(ctx)


def check(nnm, orc, X, restr, precision="fp32", metric="euclidean"):
    om = orc.restrict_literal(X, restr, metric=metric)
    olab, oK = orc.labels(om, X.shape[0])
    m, lab, K = literal_gpu(nnm, X, restr, precision, metric)
    assert np.array_equal(m, om), restr
    assert np.array_equal(lab, olab) and K == oK, restr
    return om


def test_literal_counterexample_joins_outside_the_tree(nnm, orc):
    X = np.array([[0.0], [10.0], [11.0], [12.0], [13.0], [14.0], [24.0]], dtype=np.float32)
    om = check(nnm, orc, X, {"kl3_max_size": 5})
    assert [(int(a), int(b)) for a, b in zip(om["a"], om["b"])] == [(1, 2), (2, 3), (3, 4), (4, 5), (0, 6)]


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_literal_equals_tree_for_cap_and_kl1(nnm, orc, precision):
    from paper_1402_3789_gb300.inputs import make
    X = make("nnm_n4096_d8", n=4000, seed=31)
    for r in ({"max_join_dist": 0.9}, {"max_join_dist": 1.4, "kl1_stop_clusters": 40}, {"kl1_stop_clusters": 7}):
        om = check(nnm, orc, X, r, precision)
        tree = orc.prim(X)
        assert np.array_equal(om, orc.restrict_tree(tree, X.shape[0], r))


@pytest.mark.parametrize("restr", [
    {"kl3_max_size": 150},
    {"kl2_max_pre_size": 40},
    {"kl2_max_pre_size": 60, "kl3_max_size": 200, "max_join_dist": 2.0},
    {"kl4_min_size": 6},
    {"kl4_min_size": 8, "kl3_max_size": 300},
    {"kl4_min_size": 5, "kl2_max_pre_size": 80, "kl1_stop_clusters": 25},
    {"kl4_min_size": 1, "kl3_max_size": 90},
    {"kl3_max_size": 120, "kl1_stop_clusters": 30, "max_join_dist": 1.5},
], ids=["kl3", "kl2", "kl2kl3cap", "kl4", "kl4kl3", "kl4kl2kl1", "kl4is1", "kl3kl1cap"])
def test_literal_gates_on_a_mixture(nnm, orc, restr):
    from paper_1402_3789_gb300.inputs import make
    X = make("nnm_n4096_d8", n=3000, seed=17)
    check(nnm, orc, X, restr)


def test_literal_ties_and_duplicates(nnm, orc):
    rng = np.random.default_rng(9)
    X = (np.round(rng.uniform(0.0, 3.0, size=(2500, 3)) * 4.0) / 4.0).astype(np.float32)
    X[100:140] = X[5]   # exact duplicates: many pairs at D = 0
    for r in ({"kl3_max_size": 60}, {"kl4_min_size": 4, "kl2_max_pre_size": 30}, {"kl1_stop_clusters": 50}):
        check(nnm, orc, X, r)


def test_literal_manhattan(nnm, orc):
    from paper_1402_3789_gb300.inputs import make
    X = make("nnm_n4096_d8", n=2500, seed=23)
    check(nnm, orc, X, {"kl3_max_size": 100, "kl4_min_size": 4, "max_join_dist": 3.0}, metric="manhattan")


@pytest.mark.slow
def test_literal_at_20000_rows(nnm, orc):
    from paper_1402_3789_gb300.inputs import make
    X = make("nnm_n262144_d16", n=20000, seed=41)
    check(nnm, orc, X, {"kl4_min_size": 10, "kl3_max_size": 600, "kl1_stop_clusters": 20})


def test_literal_rejects_what_it_does_not_cover(nnm):
    from paper_1402_3789_gb300.inputs import make
    parts = [torch.from_numpy(make("nnm_n4096_d8", n=n, seed=s)).cuda() for n, s in ((300, 1), (400, 2))]
    ctx = nnm.nnm_create_batched(parts)
    try:
        with pytest.raises(nnm.NNMError) as ei:
            nnm.nnm_cluster(ctx, {"semantics": 1})
        assert ei.value.status == nnm.NNM_EUNSUPPORTED
        with pytest.raises(nnm.NNMError) as ei:
            nnm.nnm_cluster(ctx, {"semantics": 2})
        assert ei.value.status == nnm.NNM_EINVAL
    finally:
        nnm.nnm_destroy(ctx)
