"""Thin ctypes binding over ``libnnm.so`` (include/nnm.h): argument marshalling only.

Every step of the computation runs in the library's sm_103a kernels.  PyTorch only
supplies device memory and the CUDA stream.  The functions keep the C names:

    ctx = nnm_create(X_cuda_float32, precision="bf16")
    idx, D = nnm_nearest(ctx, k)
    res = nnm_cluster(ctx, {"max_join_dist": 2.0, "kl3_max_size": 50000})
    tree = nnm_get_tree(ctx)
    stats = nnm_get_stats(ctx)
    nnm_destroy(ctx)

If the compiled library is missing the first call raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

NNM_OK, NNM_EINVAL, NNM_ENONFINITE, NNM_ENOMEM, NNM_ECUDA, NNM_ETIMEOUT, NNM_EUNSUPPORTED = range(7)
PRECISIONS = {"fp32": 0, "bf16": 1, "fp16": 2, "bf16x3": 3}

EDGE_DTYPE = np.dtype([("a", "<u4"), ("b", "<u4"), ("D", "<f8")])
MERGE_DTYPE = np.dtype([("a", "<u4"), ("b", "<u4"), ("D", "<f8"), ("dist", "<f8"), ("new_size", "<i8")])


class NNMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


class nnm_options(ctypes.Structure):
    _fields_ = [("cache_k", ctypes.c_int32), ("freeze_at_cap", ctypes.c_int32),
                ("col_split", ctypes.c_int32), ("no_tile_pruning", ctypes.c_int32),
                ("wait_limit_ns", ctypes.c_int64)]


class nnm_restrictions(ctypes.Structure):
    _fields_ = [("max_join_dist", ctypes.c_double), ("kl1_stop_clusters", ctypes.c_int64),
                ("kl2_max_pre_size", ctypes.c_int64), ("kl3_max_size", ctypes.c_int64),
                ("kl4_min_size", ctypes.c_int64), ("semantics", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class nnm_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("ms_prep", "ms_sweep", "ms_rerank", "ms_rounds", "ms_sort",
                                               "ms_restrict", "ms_labels", "ms_total")] + \
               [(n, ctypes.c_int64) for n in ("rounds", "sweep_launches", "pairs_evaluated", "rows_rescanned",
                                              "rows_overflowed", "rerank_pairs", "max_candidates")] + \
               [("max_abs_err", ctypes.c_double), ("max_rel_err", ctypes.c_double),
                ("sweep_ms_per_launch_full", ctypes.c_double), ("full_sweep_pairs", ctypes.c_int64),
                ("k_pad", ctypes.c_int32), ("cache_k", ctypes.c_int32), ("scale", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("tiles_skipped", ctypes.c_int64),
                ("tiles_swept", ctypes.c_int64), ("full_sweep_pairs_computed", ctypes.c_int64)]


# every symbol include/nnm.h declares
EXPORTS = ("nnm_create", "nnm_create_batched", "nnm_nearest", "nnm_cluster", "nnm_get_tree", "nnm_get_stats",
           "nnm_last_error", "nnm_status_string", "nnm_destroy", "nnm_restrict_static", "nnm_cluster_host",
           "nnm_set_wait_limit")
STATIC_MAX_ROWS = 1 << 20

_LIB = None


def library_path() -> str:
    return _build.library_path()


def load_library(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libnnm.so (raises if it is missing and not built here)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.nnm_create.argtypes = [P, i64, i32, ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(nnm_options),
                               ctypes.POINTER(P)]
    lib.nnm_create.restype = ctypes.c_int
    lib.nnm_create_batched.argtypes = [P, P, i64, i32, ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(nnm_options),
                                       ctypes.POINTER(P)]
    lib.nnm_create_batched.restype = ctypes.c_int
    lib.nnm_nearest.argtypes = [P, i32, P, P]
    lib.nnm_nearest.restype = ctypes.c_int
    lib.nnm_cluster.argtypes = [P, ctypes.POINTER(nnm_restrictions), P, ctypes.POINTER(i64), P,
                                ctypes.POINTER(i64)]
    lib.nnm_cluster.restype = ctypes.c_int
    lib.nnm_get_tree.argtypes = [P, P, ctypes.POINTER(i64)]
    lib.nnm_get_tree.restype = ctypes.c_int
    lib.nnm_get_stats.argtypes = [P, ctypes.POINTER(nnm_stats)]
    lib.nnm_get_stats.restype = ctypes.c_int
    lib.nnm_last_error.argtypes = [P]
    lib.nnm_last_error.restype = ctypes.c_char_p
    lib.nnm_status_string.argtypes = [ctypes.c_int]
    lib.nnm_status_string.restype = ctypes.c_char_p
    lib.nnm_destroy.argtypes = [P]
    lib.nnm_destroy.restype = None
    lib.nnm_restrict_static.argtypes = [P, i64, i64, ctypes.c_int, ctypes.POINTER(nnm_restrictions), P,
                                        ctypes.POINTER(i64), P, ctypes.POINTER(i64), P]
    lib.nnm_restrict_static.restype = ctypes.c_int
    lib.nnm_cluster_host.argtypes = [P, i64, i32, ctypes.c_int, ctypes.c_int, ctypes.POINTER(nnm_options),
                                     ctypes.POINTER(nnm_restrictions), P, P, ctypes.POINTER(i64), P,
                                     ctypes.POINTER(i64)]
    lib.nnm_cluster_host.restype = ctypes.c_int
    lib.nnm_set_wait_limit.argtypes = [P, i64]
    lib.nnm_set_wait_limit.restype = ctypes.c_int
    _LIB = lib
    return lib


def _status_name(s: int) -> str:
    try:
        return load_library().nnm_status_string(s).decode()
    except Exception:
        return f"status {s}"


@dataclass
class Context:
    """An nnm_ctx handle plus the tensor it borrows."""
    handle: ctypes.c_void_p
    X: torch.Tensor
    N: int
    d: int
    precision: str
    stream: torch.cuda.Stream
    offsets: list | None = None   # batched contexts: first row of each instance, and N

    def _check(self, status: int):
        if status != NNM_OK:
            msg = load_library().nnm_last_error(self.handle)
            raise NNMError(status, (msg or b"").decode())


METRICS = {"euclidean": 0, "manhattan": 1, "chebyshev": 2}


def nnm_create(X: torch.Tensor, precision: str = "fp32", stream: torch.cuda.Stream | None = None,
               cache_k: int = 0, freeze_at_cap: bool = False, col_split: int = 0,
               tile_pruning: bool = True, metric: str = "euclidean", wait_limit_ns: int = 0) -> Context:
    """nnm_create: X is a contiguous float32 [N, d] CUDA tensor (kept alive by the context)."""
    lib = load_library()
    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float32 and X.dim() == 2):
        raise ValueError("X must be a float32 [N, d] CUDA tensor")
    X = X.contiguous()
    stream = stream or torch.cuda.current_stream(X.device)
    opt = nnm_options(int(cache_k), int(bool(freeze_at_cap)), int(col_split), int(not tile_pruning),
                      int(wait_limit_ns))
    h = ctypes.c_void_p()
    st = lib.nnm_create(ctypes.c_void_p(X.data_ptr()), X.shape[0], X.shape[1], METRICS[metric], PRECISIONS[precision],
                        ctypes.c_void_p(stream.cuda_stream), ctypes.byref(opt), ctypes.byref(h))
    if st != NNM_OK:
        raise NNMError(st, "nnm_create failed")
    return Context(h, X, X.shape[0], X.shape[1], precision, stream)


def nnm_create_batched(Xs, precision: str = "fp32", stream: torch.cuda.Stream | None = None,
                       cache_k: int = 0, col_split: int = 0, tile_pruning: bool = True,
                       metric: str = "euclidean") -> Context:
    """nnm_create_batched over a list of float32 CUDA tensors [N_b, d_b] (independent
    instances): they are concatenated into one [sum N_b, max d_b] tensor, narrower ones
    padded with zero columns (which change no distance).  Row r of instance b is row
    offsets[b] + r of the context; ``ctx.offsets`` holds the offsets."""
    lib = load_library()
    if not Xs or not all(isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.dim() == 2
                         for x in Xs):
        raise ValueError("Xs must be float32 [N_b, d_b] CUDA tensors")
    d = max(x.shape[1] for x in Xs)
    X = torch.cat([torch.nn.functional.pad(x, (0, d - x.shape[1])) for x in Xs]).contiguous()
    offsets = [0]
    for x in Xs:
        offsets.append(offsets[-1] + x.shape[0])
    off = (ctypes.c_int64 * len(offsets))(*offsets)
    stream = stream or torch.cuda.current_stream(X.device)
    opt = nnm_options(int(cache_k), 0, int(col_split), int(not tile_pruning))
    h = ctypes.c_void_p()
    st = lib.nnm_create_batched(ctypes.c_void_p(X.data_ptr()), ctypes.cast(off, ctypes.c_void_p), len(Xs), d,
                                METRICS[metric],
                                PRECISIONS[precision], ctypes.c_void_p(stream.cuda_stream), ctypes.byref(opt),
                                ctypes.byref(h))
    if st != NNM_OK:
        raise NNMError(st, "nnm_create_batched failed")
    return Context(h, X, X.shape[0], d, precision, stream, offsets)


def nnm_nearest(ctx: Context, k: int):
    """Exact k nearest neighbours of every row: (idx uint32 [N,k], D float64 [N,k]) on the device."""
    lib = load_library()
    idx = torch.empty((ctx.N, k), dtype=torch.int32, device=ctx.X.device).view(torch.uint32)
    D = torch.empty((ctx.N, k), dtype=torch.float64, device=ctx.X.device)
    ctx._check(lib.nnm_nearest(ctx.handle, k, ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(D.data_ptr())))
    return idx, D


@dataclass
class ClusterResult:
    merges_dev: torch.Tensor   # uint8 [(N-1) * 32]: nnm_merge records
    n_merges: int
    labels: torch.Tensor       # int32 [N] on the device
    n_clusters: int

    def merges(self) -> np.ndarray:
        raw = self.merges_dev[: self.n_merges * MERGE_DTYPE.itemsize].cpu().numpy()
        return raw.view(MERGE_DTYPE).copy()


def _restrictions(r) -> nnm_restrictions:
    r = dict(r or {})
    return nnm_restrictions(float(r.get("max_join_dist", 0.0)), int(r.get("kl1_stop_clusters", 0)),
                            int(r.get("kl2_max_pre_size", 0)), int(r.get("kl3_max_size", 0)),
                            int(r.get("kl4_min_size", 0)), int(r.get("semantics", 0)), 0)


def nnm_cluster(ctx: Context, restrictions=None, merges_out: torch.Tensor | None = None,
                labels_out: torch.Tensor | None = None) -> ClusterResult:
    """The merge tree and the restricted joins; outputs stay on the device."""
    lib = load_library()
    nm = max(ctx.N - 1, 1)
    merges = merges_out if merges_out is not None else torch.empty(nm * MERGE_DTYPE.itemsize, dtype=torch.uint8,
                                                                    device=ctx.X.device)
    labels = labels_out if labels_out is not None else torch.empty(ctx.N, dtype=torch.int32, device=ctx.X.device)
    r = _restrictions(restrictions)
    n_m, n_c = ctypes.c_int64(), ctypes.c_int64()
    ctx._check(lib.nnm_cluster(ctx.handle, ctypes.byref(r), ctypes.c_void_p(merges.data_ptr()), ctypes.byref(n_m),
                               ctypes.c_void_p(labels.data_ptr()), ctypes.byref(n_c)))
    return ClusterResult(merges, n_m.value, labels, n_c.value)


def nnm_get_tree(ctx: Context) -> np.ndarray:
    """Merge-tree edges of the last nnm_cluster call, key order, as a host array."""
    lib = load_library()
    buf = torch.empty(max(ctx.N - 1, 1) * EDGE_DTYPE.itemsize, dtype=torch.uint8, device=ctx.X.device)
    n = ctypes.c_int64()
    ctx._check(lib.nnm_get_tree(ctx.handle, ctypes.c_void_p(buf.data_ptr()), ctypes.byref(n)))
    return buf[: n.value * EDGE_DTYPE.itemsize].cpu().numpy().view(EDGE_DTYPE).copy()


def nnm_get_stats(ctx: Context) -> dict:
    lib = load_library()
    s = nnm_stats()
    ctx._check(lib.nnm_get_stats(ctx.handle, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in nnm_stats._fields_}


def nnm_destroy(ctx: Context) -> None:
    if ctx.handle:
        load_library().nnm_destroy(ctx.handle)
        ctx.handle = ctypes.c_void_p()


def nnm_restrict_static(tree_dev: torch.Tensor, n_edges: int, N: int, restrictions=None,
                        stream: torch.cuda.Stream | None = None, metric: str = "euclidean") -> ClusterResult:
    """nnm_restrict_static: restrictions + labels on a key-sorted tree (uint8 device bytes
    of nnm_edge records, D in the given metric), using the library's fixed scratch array
    (no allocation inside the library; the output tensors are allocated here by the
    caller's allocator)."""
    lib = load_library()
    stream = stream or torch.cuda.current_stream(tree_dev.device)
    merges = torch.empty(max(N - 1, 1) * MERGE_DTYPE.itemsize, dtype=torch.uint8, device=tree_dev.device)
    labels = torch.empty(N, dtype=torch.int32, device=tree_dev.device)
    r = _restrictions(restrictions)
    n_m, n_c = ctypes.c_int64(), ctypes.c_int64()
    st = lib.nnm_restrict_static(ctypes.c_void_p(tree_dev.data_ptr()), n_edges, N, METRICS[metric], ctypes.byref(r),
                                 ctypes.c_void_p(merges.data_ptr()), ctypes.byref(n_m),
                                 ctypes.c_void_p(labels.data_ptr()), ctypes.byref(n_c),
                                 ctypes.c_void_p(stream.cuda_stream))
    if st != NNM_OK:
        raise NNMError(st, "nnm_restrict_static failed")
    return ClusterResult(merges, n_m.value, labels, n_c.value)


def nnm_status_string(status: int) -> str:
    return load_library().nnm_status_string(status).decode()


def nnm_set_wait_limit(ctx: Context, wait_limit_ns: int) -> None:
    """Wait limit of the tensor-core sweep's device-side waits for the following calls
    (0: the 2 s default)."""
    ctx._check(load_library().nnm_set_wait_limit(ctx.handle, int(wait_limit_ns)))


def cluster_host(X, restrictions=None, precision: str = "fp32", metric: str = "euclidean", merges_out=None,
                 labels_out=None, stream: torch.cuda.Stream | None = None, **options):
    """nnm_cluster_host: end to end from host memory through the C ABI (the library
    copies X to the device, clusters, and copies merges and labels back).  X is a
    float32 [N, d] numpy array or CPU tensor (page-locked copies fastest); merges_out /
    labels_out may be preallocated CPU tensors (uint8 [(N-1)*32], int32 [N]).
    Returns (merges, labels, n_clusters) as numpy arrays."""
    lib = load_library()
    Xh = X if isinstance(X, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32))
    if Xh.is_cuda or Xh.dtype != torch.float32 or Xh.dim() != 2:
        raise ValueError("X must be a float32 [N, d] host array")
    Xh = Xh.contiguous()
    N, d = Xh.shape
    merges = merges_out if merges_out is not None else torch.empty(max(N - 1, 1) * MERGE_DTYPE.itemsize,
                                                                    dtype=torch.uint8)
    labels = labels_out if labels_out is not None else torch.empty(N, dtype=torch.int32)
    opt = nnm_options(int(options.get("cache_k", 0)), int(bool(options.get("freeze_at_cap", False))),
                      int(options.get("col_split", 0)), int(not options.get("tile_pruning", True)),
                      int(options.get("wait_limit_ns", 0)))
    r = _restrictions(restrictions)
    stream = stream or torch.cuda.current_stream()
    n_m, n_c = ctypes.c_int64(), ctypes.c_int64()
    st = lib.nnm_cluster_host(ctypes.c_void_p(Xh.data_ptr()), N, d, METRICS[metric], PRECISIONS[precision],
                              ctypes.byref(opt), ctypes.byref(r), ctypes.c_void_p(stream.cuda_stream),
                              ctypes.c_void_p(merges.data_ptr()), ctypes.byref(n_m),
                              ctypes.c_void_p(labels.data_ptr()), ctypes.byref(n_c))
    if st != NNM_OK:
        raise NNMError(st, "nnm_cluster_host failed")
    # views of the output buffers (the caller's, when given): no extra host copy
    return merges[: n_m.value * MERGE_DTYPE.itemsize].numpy().view(MERGE_DTYPE), labels.numpy(), n_c.value
