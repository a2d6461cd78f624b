"""GPU tests of the failure path and of the host-memory entry point, through the C ABI.

Failure detection: every device-side wait of the tensor-core sweep is bounded; when a
wait runs out the kernel raises its error flag, lets its own copies and MMAs land,
frees its TMEM and exits, and the call returns NNM_ETIMEOUT.  The test makes the waits
run out with a 1 ns limit (no fault, no endless loop: every wait gives up and returns)
and then runs the same context with the default limit, which must give the oracle's
result.  nnm_cluster_host is checked against the oracle from host memory.
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


def dev(X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()


@pytest.mark.parametrize("precision", ["bf16x3", "fp16"])
def test_wait_limit_times_out_and_the_context_recovers(nnm, orc, precision):
    from paper_1402_3789_gb300.inputs import make
    X = make("nnm_n4096_d8", n=20000, seed=9)
    restr = {"max_join_dist": 1.0, "kl3_max_size": 900, "kl4_min_size": 4}
    otree, om, olab, oK = orc.cluster(X, restr)
    oi, oD = orc.knn(X, 4)
    ctx = nnm.nnm_create(dev(X), precision=precision, wait_limit_ns=1)
    try:
        with pytest.raises(nnm.NNMError) as ei:
            nnm.nnm_cluster(ctx, restr)
        assert ei.value.status == nnm.NNM_ETIMEOUT
        with pytest.raises(nnm.NNMError) as ei:
            nnm.nnm_nearest(ctx, 4)
        assert ei.value.status == nnm.NNM_ETIMEOUT
        nnm.nnm_set_wait_limit(ctx, 0)          # back to the default: the same context works
        idx, D = nnm.nnm_nearest(ctx, 4)
        assert np.array_equal(idx.cpu().numpy().view(np.uint32), oi) and np.array_equal(D.cpu().numpy(), oD)
        res = nnm.nnm_cluster(ctx, restr)
        assert np.array_equal(nnm.nnm_get_tree(ctx), otree)
        assert np.array_equal(res.merges(), om)
        assert np.array_equal(res.labels.cpu().numpy(), olab) and res.n_clusters == oK
    finally:
        nnm.nnm_destroy(ctx)


def test_wait_limit_rejects_negative_values(nnm):
    X = torch.zeros((64, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(nnm.NNMError) as ei:
        nnm.nnm_create(X, precision="bf16", wait_limit_ns=-1)
    assert ei.value.status == nnm.NNM_EINVAL
    ctx = nnm.nnm_create(X + torch.arange(64, device="cuda", dtype=torch.float32)[:, None], precision="bf16")
    try:
        with pytest.raises(nnm.NNMError) as ei:
            nnm.nnm_set_wait_limit(ctx, -5)
        assert ei.value.status == nnm.NNM_EINVAL
    finally:
        nnm.nnm_destroy(ctx)


@pytest.mark.parametrize("precision,metric", [("bf16x3", "euclidean"), ("fp32", "manhattan")])
def test_cluster_host_matches_the_oracle(nnm, orc, precision, metric):
    from paper_1402_3789_gb300.inputs import make
    X = make("nnm_n4096_d8", n=5000, seed=12)
    restr = {"max_join_dist": 1.2, "kl1_stop_clusters": 20}
    _, om, olab, oK = orc.cluster(X, restr, metric=metric)
    Xh = torch.from_numpy(X).pin_memory()
    merges, labels, K = nnm.cluster_host(Xh, restr, precision=precision, metric=metric)
    assert np.array_equal(merges, om)
    assert np.array_equal(labels, olab) and K == oK
    # pageable host memory works too
    merges, labels, K = nnm.cluster_host(X, restr, precision=precision, metric=metric)
    assert np.array_equal(merges, om) and np.array_equal(labels, olab) and K == oK
