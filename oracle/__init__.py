"""CPU oracle for nearest-neighbour-method (NNM) single-linkage clustering.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; the product path never imports it.  It is a
thin ctypes layer over ``nnm_oracle.c`` (plain C, IEEE binary64, no FMA), which
shares no code with the CUDA library.

Functions (paper: Litvinenko, arXiv:1402.3789); each takes metric= "euclidean" (Eq. (1),
D its square), "manhattan" or "chebyshev" (the paper leaves other metrics open):
  dist_pairs        D in the canonical feature order
  knn               exact k nearest neighbours by brute force, order (D, j)
  nnm_batched       the paper's P-minimal-pairs procedure ("General description of
                    the algorithm for constructing the set of minimum distances")
  prim, kruskal_allpairs
                    independent routes to the same unique merge tree
  restrict_tree     restrictions of "Problem statement"/"Problem settings" (KL1-KL4,
                    max joining distance) on the key-ordered tree
  restrict_literal  the same gates applied to every pair (small N)
  labels            dense labels ordered by each cluster's smallest member
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build, library_path

EDGE_DTYPE = np.dtype([("a", "<u4"), ("b", "<u4"), ("D", "<f8")])
MERGE_DTYPE = np.dtype([("a", "<u4"), ("b", "<u4"), ("D", "<f8"), ("dist", "<f8"),
                        ("new_size", "<i8")])


class _Restr(ctypes.Structure):
    _fields_ = [("max_join_dist", ctypes.c_double), ("kl1_stop_clusters", ctypes.c_int64),
                ("kl2_max_pre_size", ctypes.c_int64), ("kl3_max_size", ctypes.c_int64),
                ("kl4_min_size", ctypes.c_int64)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        lib.or_dist_pairs.argtypes = [P, i32, P, P, i64, P]
        lib.or_dist_pairs.restype = None
        lib.or_knn.argtypes = [P, i64, i32, P, i64, i32, i32, P, P]
        lib.or_knn.restype = ctypes.c_int
        lib.or_nnm_batched.argtypes = [P, i64, i32, i64, i32, P]
        lib.or_nnm_batched.restype = i64
        lib.or_prim.argtypes = [P, i64, i32, i32, P]
        lib.or_prim.restype = i64
        lib.or_kruskal_allpairs.argtypes = [P, i64, i32, P]
        lib.or_kruskal_allpairs.restype = i64
        lib.or_restrict_tree.argtypes = [P, i64, i64, ctypes.POINTER(_Restr), P]
        lib.or_restrict_tree.restype = i64
        lib.or_restrict_literal.argtypes = [P, i64, i32, ctypes.POINTER(_Restr), P]
        lib.or_restrict_literal.restype = i64
        lib.or_labels.argtypes = [P, i64, i64, P]
        lib.or_labels.restype = i64
        lib.or_sort_edges.argtypes = [P, i64]
        lib.or_sort_edges.restype = None
        lib.or_set_metric.argtypes = [i32]
        lib.or_set_metric.restype = None
        _LIB = lib
    return _LIB


def _rows(X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    assert X.ndim == 2
    return X, X.shape[0], X.shape[1]


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


METRICS = {"euclidean": 0, "manhattan": 1, "chebyshev": 2}


class _metric:
    """Select the oracle's metric for one call (back to Euclidean afterwards)."""

    def __init__(self, metric):
        self.code = METRICS[metric] if isinstance(metric, str) else int(metric)

    def __enter__(self):
        _lib().or_set_metric(self.code)

    def __exit__(self, *exc):
        _lib().or_set_metric(0)


def dist_pairs(X, i, j, metric="euclidean"):
    """D(i[m], j[m]) for every m: Eq. (1) squared in the canonical order."""
    X, N, d = _rows(X)
    i = np.ascontiguousarray(i, dtype=np.int64)
    j = np.ascontiguousarray(j, dtype=np.int64)
    out = np.empty(i.shape[0], dtype=np.float64)
    with _metric(metric):
        _lib().or_dist_pairs(_ptr(X), d, _ptr(i), _ptr(j), i.shape[0], _ptr(out))
    return out


def knn(X, k, queries=None, threads=0, metric="euclidean"):
    """Exact k nearest neighbours (self excluded) of each query row, order (D, j)."""
    X, N, d = _rows(X)
    q = np.arange(N, dtype=np.int64) if queries is None else np.ascontiguousarray(queries, np.int64)
    idx = np.empty((q.shape[0], k), dtype=np.uint32)
    D = np.empty((q.shape[0], k), dtype=np.float64)
    with _metric(metric):
        rc = _lib().or_knn(_ptr(X), N, d, _ptr(q), q.shape[0], k, threads, _ptr(idx), _ptr(D))
    if rc != 0:
        raise ValueError("or_knn: bad arguments")
    return idx, D


def _edges_call(fn, X, *extra, metric="euclidean"):
    X, N, d = _rows(X)
    out = np.zeros(max(N - 1, 1), dtype=EDGE_DTYPE)
    with _metric(metric):
        m = fn(_ptr(X), N, d, *extra, _ptr(out))
    if m < 0:
        raise ValueError(f"{fn.__name__}: bad arguments")
    return out[:m]


def nnm_batched(X, P, threads=0, metric="euclidean"):
    """Merge tree by the paper's batched P-minimal-pairs passes; edges in key order."""
    return _edges_call(_lib().or_nnm_batched, X, P, threads, metric=metric)


def prim(X, threads=0, metric="euclidean"):
    """Merge tree by dense Prim; edges in key order."""
    return _edges_call(_lib().or_prim, X, threads, metric=metric)


def kruskal_allpairs(X, metric="euclidean"):
    """Merge tree by Kruskal over all pairs (N <= 20000); edges in key order."""
    return _edges_call(_lib().or_kruskal_allpairs, X, metric=metric)


def _restr(r):
    r = dict(r or {})
    return _Restr(float(r.get("max_join_dist", 0.0)), int(r.get("kl1_stop_clusters", 0)),
                  int(r.get("kl2_max_pre_size", 0)), int(r.get("kl3_max_size", 0)),
                  int(r.get("kl4_min_size", 0)))


def restrict_tree(edges, N, restrictions=None, metric="euclidean"):
    """Accepted merges (acceptance order) of the key-ordered tree under the restrictions."""
    edges = np.ascontiguousarray(edges, dtype=EDGE_DTYPE)
    out = np.zeros(max(N - 1, 1), dtype=MERGE_DTYPE)
    r = _restr(restrictions)
    with _metric(metric):
        m = _lib().or_restrict_tree(_ptr(edges), edges.shape[0], N, ctypes.byref(r), _ptr(out))
    return out[:m]


def restrict_literal(X, restrictions=None, metric="euclidean"):
    """Accepted merges when the gates act on every pair in key order (N <= 20000)."""
    X, N, d = _rows(X)
    out = np.zeros(max(N - 1, 1), dtype=MERGE_DTYPE)
    r = _restr(restrictions)
    with _metric(metric):
        m = _lib().or_restrict_literal(_ptr(X), N, d, ctypes.byref(r), _ptr(out))
    if m < 0:
        raise ValueError("or_restrict_literal: bad arguments")
    return out[:m]


def labels(merges, N):
    """(labels int32[N], K): dense labels ordered by each cluster's smallest member."""
    merges = np.ascontiguousarray(merges, dtype=MERGE_DTYPE)
    lab = np.empty(N, dtype=np.int32)
    K = _lib().or_labels(_ptr(merges), merges.shape[0], N, _ptr(lab))
    return lab, int(K)


def cluster(X, restrictions=None, threads=0, method="prim", P=None, metric="euclidean"):
    """Full oracle: merge tree, restrictions, labels -> (tree, merges, labels, K)."""
    X, N, d = _rows(X)
    if method == "prim":
        tree = prim(X, threads, metric=metric)
    elif method == "batched":
        tree = nnm_batched(X, P if P else N, threads, metric=metric)
    else:
        tree = kruskal_allpairs(X, metric=metric)
    merges = restrict_tree(tree, N, restrictions, metric=metric)
    lab, K = labels(merges, N)
    return tree, merges, lab, K
