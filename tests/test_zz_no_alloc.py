"""nnm_restrict_static: the restriction walk and labels without any device allocation
inside the library (its scratch is a fixed device array), for callers whose device
memory is owned by a pool or fixed at start-up.

Checked through the C ABI against the existing entry point: nnm_cluster's merges and
labels must equal what nnm_restrict_static produces from nnm_cluster's own tree, on two
calls in a row (the second call reuses the fixed array left by the first).  This file
is collected last so that a failure here stops a run only after every other test.
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


def _static_call(nnm, tree_dev, n_edges, N, restr):
    """Call the C symbol directly (ctypes), with output buffers made here."""
    lib = nnm.load_library()
    merges = torch.empty(max(N - 1, 1) * nnm.MERGE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    labels = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    r = nnm._restrictions(restr)
    n_m, n_c = ctypes.c_int64(-1), ctypes.c_int64(-1)
    st = lib.nnm_restrict_static(ctypes.c_void_p(tree_dev.data_ptr()), n_edges, N, ctypes.byref(r),
                                 ctypes.c_void_p(merges.data_ptr()), ctypes.byref(n_m),
                                 ctypes.c_void_p(labels.data_ptr()), ctypes.byref(n_c),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, merges, n_m.value, labels, n_c.value


@pytest.mark.parametrize("restr", [
    {"max_join_dist": 1.1, "kl1_stop_clusters": 30},
    {"kl4_min_size": 8, "kl3_max_size": 150, "kl2_max_pre_size": 60},
])
def test_static_entry_point_matches_nnm_cluster(nnm, restr):
    from paper_1402_3789_gb300.inputs import make
    X = make("nnm_n4096_d8", n=6000, seed=21)
    ctx = nnm.nnm_create(torch.from_numpy(X).cuda(), precision="fp32")
    try:
        ref = nnm.nnm_cluster(ctx, restr)
        tree = nnm.nnm_get_tree(ctx)
    finally:
        nnm.nnm_destroy(ctx)
    ref_merges = ref.merges()
    ref_labels = ref.labels.cpu().numpy()
    tree_dev = torch.from_numpy(tree.view(np.uint8).copy()).cuda()
    for _ in range(2):
        st, merges, n_m, labels, n_c = _static_call(nnm, tree_dev, tree.shape[0], X.shape[0], restr)
        assert st == nnm.NNM_OK
        got = merges[: n_m * nnm.MERGE_DTYPE.itemsize].cpu().numpy().view(nnm.MERGE_DTYPE)
        assert n_m == ref.n_merges and np.array_equal(got, ref_merges)
        assert n_c == ref.n_clusters and np.array_equal(labels.cpu().numpy(), ref_labels)


def test_static_entry_point_rejects_sizes_beyond_its_array(nnm):
    tree_dev = torch.zeros(16, dtype=torch.uint8, device="cuda")
    st, *_ = _static_call(nnm, tree_dev, 1, nnm.STATIC_MAX_ROWS + 1, None)
    assert st == nnm.NNM_EUNSUPPORTED
    st, *_ = _static_call(nnm, tree_dev, 5, 3, None)      # more edges than N-1
    assert st == nnm.NNM_EINVAL
