"""nnm_restrict_static: the restriction walk and labels without any device allocation
inside the library (its scratch is a fixed device array), for callers whose device
memory is owned by a pool or fixed at start-up.

Checked through the C ABI against the existing entry point: nnm_cluster's merges and
labels must equal what nnm_restrict_static produces from nnm_cluster's own tree, on two
calls in a row (the second call reuses the fixed array left by the first), for the
Euclidean and the Manhattan metric (the cap's units and the reported lengths follow the
metric), and once at a size close to the array's row limit.  Trees the walk must not
index with (an endpoint at N, a == b, keys out of order, a batched context's tree
grouped by instance) are refused with NNM_EINVAL.  This file is collected last so that
a failure here stops a run only after every other test.
"""
import ctypes

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


def _static_call(nnm, tree_dev, n_edges, N, restr, metric="euclidean"):
    """Call the C symbol directly (ctypes), with output buffers made here."""
    lib = nnm.load_library()
    merges = torch.empty(max(N - 1, 1) * nnm.MERGE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    labels = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    r = nnm._restrictions(restr)
    n_m, n_c = ctypes.c_int64(-1), ctypes.c_int64(-1)
    st = lib.nnm_restrict_static(ctypes.c_void_p(tree_dev.data_ptr()), n_edges, N, nnm.METRICS[metric],
                                 ctypes.byref(r), ctypes.c_void_p(merges.data_ptr()), ctypes.byref(n_m),
                                 ctypes.c_void_p(labels.data_ptr()), ctypes.byref(n_c),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, merges, n_m.value, labels, n_c.value


def _reference(nnm, X, restr, metric="euclidean", precision="fp32", batched=None):
    if batched:
        ctx = nnm.nnm_create_batched([torch.from_numpy(x).cuda() for x in batched], precision=precision,
                                     metric=metric)
    else:
        ctx = nnm.nnm_create(torch.from_numpy(X).cuda(), precision=precision, metric=metric)
    try:
        ref = nnm.nnm_cluster(ctx, restr)
        tree = nnm.nnm_get_tree(ctx)
    finally:
        nnm.nnm_destroy(ctx)
    return ref, tree


def _check_twice(nnm, X, restr, metric, precision="fp32"):
    ref, tree = _reference(nnm, X, restr, metric, precision)
    ref_merges = ref.merges()
    ref_labels = ref.labels.cpu().numpy()
    tree_dev = torch.from_numpy(tree.view(np.uint8).copy()).cuda()
    for _ in range(2):
        st, merges, n_m, labels, n_c = _static_call(nnm, tree_dev, tree.shape[0], X.shape[0], restr, metric)
        assert st == nnm.NNM_OK
        got = merges[: n_m * nnm.MERGE_DTYPE.itemsize].cpu().numpy().view(nnm.MERGE_DTYPE)
        assert n_m == ref.n_merges and np.array_equal(got, ref_merges)
        assert n_c == ref.n_clusters and np.array_equal(labels.cpu().numpy(), ref_labels)


@pytest.mark.parametrize("metric", ["euclidean", "manhattan"])
@pytest.mark.parametrize("restr", [
    {"max_join_dist": 1.1, "kl1_stop_clusters": 30},
    {"max_join_dist": 2.5, "kl4_min_size": 8, "kl3_max_size": 150, "kl2_max_pre_size": 60},
])
def test_static_entry_point_matches_nnm_cluster(nnm, restr, metric):
    from paper_1402_3789_gb300.inputs import make
    X = make("nnm_n4096_d8", n=6000, seed=21)
    _check_twice(nnm, X, restr, metric)


def test_static_entry_point_near_its_row_limit(nnm):
    from paper_1402_3789_gb300.inputs import make
    X = make("nnm_n4096_d8", n=nnm.STATIC_MAX_ROWS - 3, seed=5)
    _check_twice(nnm, X, {"max_join_dist": 0.6, "kl3_max_size": 400, "kl4_min_size": 5}, "euclidean")


def test_static_entry_point_rejects_sizes_beyond_its_array(nnm):
    tree_dev = torch.zeros(16, dtype=torch.uint8, device="cuda")
    st, *_ = _static_call(nnm, tree_dev, 1, nnm.STATIC_MAX_ROWS + 1, None)
    assert st == nnm.NNM_EUNSUPPORTED
    st, *_ = _static_call(nnm, tree_dev, 5, 3, None)      # more edges than N-1
    assert st == nnm.NNM_EINVAL
    st, *_ = _static_call(nnm, tree_dev, 0, 3, None)
    assert st == nnm.NNM_OK
    lib = nnm.load_library()
    r = nnm._restrictions(None)
    n_m, n_c = ctypes.c_int64(), ctypes.c_int64()
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    st = lib.nnm_restrict_static(ctypes.c_void_p(tree_dev.data_ptr()), 1, 3, 7, ctypes.byref(r),
                                 ctypes.c_void_p(buf.data_ptr()), ctypes.byref(n_m), ctypes.c_void_p(buf.data_ptr()),
                                 ctypes.byref(n_c), None)
    assert st == nnm.NNM_EINVAL   # unknown metric


def test_static_entry_point_rejects_bad_trees(nnm):
    from paper_1402_3789_gb300.inputs import make
    X = make("nnm_n4096_d8", n=3000, seed=8)
    N = X.shape[0]
    _, tree = _reference(nnm, X, None)
    restr = {"kl3_max_size": 200}

    def call(t):
        return _static_call(nnm, torch.from_numpy(np.ascontiguousarray(t).view(np.uint8).copy()).cuda(),
                            t.shape[0], N, restr)[0]

    assert call(tree) == nnm.NNM_OK
    bad = tree.copy()
    bad["b"][100] = N               # an endpoint one past the last row (still inside the array)
    assert call(bad) == nnm.NNM_EINVAL
    bad = tree.copy()
    bad["a"][7] = bad["b"][7]       # a self pair
    assert call(bad) == nnm.NNM_EINVAL
    bad = tree.copy()
    bad[[10, 11]] = bad[[11, 10]]   # two edges out of key order
    assert call(bad) == nnm.NNM_EINVAL
    bad = tree.copy()
    bad["D"][0] = np.nan
    assert call(bad) == nnm.NNM_EINVAL
    # the array still serves a good tree after the refusals
    assert call(tree) == nnm.NNM_OK


def test_static_entry_point_rejects_a_batched_tree(nnm):
    from paper_1402_3789_gb300.inputs import make
    parts = [make("nnm_n4096_d8", n=n, seed=s) for n, s in ((900, 1), (1300, 2), (700, 3))]
    _, tree = _reference(nnm, None, None, batched=parts)
    N = sum(p.shape[0] for p in parts)
    assert tree.shape[0] == N - len(parts)
    tree_dev = torch.from_numpy(tree.view(np.uint8).copy()).cuda()
    st, *_ = _static_call(nnm, tree_dev, tree.shape[0], N, {"kl3_max_size": 100})
    assert st == nnm.NNM_EINVAL
