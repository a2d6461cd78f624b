"""Autotuned batched clustering: many independent instances of uneven N and d.

The paper keeps one GPU busy with one large problem through its managers and buffers
("Tasks of the first level manager", "Tasks of the second level manager").  With many
small problems the settings that keep the GPU busy depend on each problem's size and
width, so this module tunes them per bucket of (N, d) and runs every bucket as one
batched context of the library (``nnm_create_batched``), the buckets concurrently on
separate CUDA streams (one host thread each; the C calls release the GIL).

Tuned per bucket (every choice gives the same, exact result; they differ in speed):
  precision  the candidate pass: split BF16 or FP16 on the tensor cores (256-row x
             128-column tiles, K = 3d + 6 or d + 6 padded to 16), or FP32 direct
             differences on the CUDA cores (64-column tiles, d FMAs per pair);
  cache_k    exact nearest neighbours cached per row for the merge rounds;
  col_split  column ranges per row tile (0: automatic).

``tune()`` times every candidate on each bucket's own instances (CUDA events around
create + cluster + destroy, after one untimed run), then compares two ways of running the
whole set: one batched context with the best single setting, and the buckets with their
own winners concurrently; it writes the winners and the faster mode to a JSON table.
``cluster_batched()`` follows that table (``tuning/gb300_batched.json`` unless another is
given).  Everything runs through the library's C ABI; nothing here computes distances or
merges.
"""
from __future__ import annotations

import json
import os
import threading
import time

import numpy as np
import torch

from . import nnm

TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning", "gb300_batched.json")

# bucket edges: N in [N_EDGES[i], N_EDGES[i+1]), d in [D_EDGES[j], D_EDGES[j+1])
N_EDGES = (2, 4096, 16384, 1 << 31)
D_EDGES = (1, 9, 17, 33)
CANDIDATES = [{"precision": p, "cache_k": k, "col_split": 0} for p in ("bf16x3", "fp16", "fp32") for k in (4, 8)]
DEFAULT = {"precision": "bf16x3", "cache_k": 0, "col_split": 0}


def bucket_of(n: int, d: int) -> str:
    """Name of the (N, d) bucket of an instance with n rows and d features."""
    if n < N_EDGES[0] or not (D_EDGES[0] <= d < D_EDGES[-1]):
        raise ValueError(f"no bucket for n={n}, d={d}")
    i = int(np.searchsorted(N_EDGES, n, side="right")) - 1
    j = int(np.searchsorted(D_EDGES, d, side="right")) - 1
    return f"n{N_EDGES[i]}-{N_EDGES[i + 1] - 1}_d{D_EDGES[j]}-{D_EDGES[j + 1] - 1}"


def group(shapes) -> dict:
    """Instance indices per bucket, in the instances' order."""
    out: dict = {}
    for q, (n, d) in enumerate(shapes):
        out.setdefault(bucket_of(n, d), []).append(q)
    return out


def _shape(x):
    return int(x.shape[0]), int(x.shape[1])


def _device(xs):
    return [x if isinstance(x, torch.Tensor) and x.is_cuda else
            torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda() for x in xs]


def _run(xs, cfg, restrictions, stream):
    ctx = nnm.nnm_create_batched(xs, precision=cfg["precision"], stream=stream, cache_k=cfg.get("cache_k", 0),
                                 col_split=cfg.get("col_split", 0))
    try:
        res = nnm.nnm_cluster(ctx, restrictions)
        return ctx.offsets, res
    finally:
        nnm.nnm_destroy(ctx)


def time_config(xs, cfg, restrictions=None, repeats: int = 2) -> float:
    """Milliseconds per create + cluster + destroy of one batched context of xs."""
    stream = torch.cuda.current_stream()
    _run(xs, cfg, restrictions, stream)   # lazy module loading, allocator warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(repeats):
        _run(xs, cfg, restrictions, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / repeats


def _run_grouped(xs, table, restrictions, concurrent=True, mode="grouped", global_cfg=None):
    """Device results per bucket: [(instance indices, offsets, ClusterResult)].  In mode
    "single" one batched context with global_cfg holds every instance."""
    if mode == "single":
        offsets, res = _run(xs, global_cfg or DEFAULT, restrictions, torch.cuda.current_stream())
        return [(list(range(len(xs))), offsets, res)]
    buckets = sorted(group([_shape(x) for x in xs]).items())
    out, errors = [None] * len(buckets), []

    def one(q, name, idx, stream):
        try:
            with torch.cuda.stream(stream):
                offsets, res = _run([xs[i] for i in idx], table.get(name, DEFAULT), restrictions, stream)
                stream.synchronize()
            out[q] = (idx, offsets, res)
        except Exception as e:   # reported after every bucket has finished
            errors.append(e)

    if concurrent and len(buckets) > 1:
        threads = [threading.Thread(target=one, args=(q, name, idx, torch.cuda.Stream()))
                   for q, (name, idx) in enumerate(buckets)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
    else:
        for q, (name, idx) in enumerate(buckets):
            one(q, name, idx, torch.cuda.current_stream())
    if errors:
        raise errors[0]
    return out


def _time(fn, repeats):
    fn()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(repeats):
        fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) * 1e3 / repeats


def tune(instances, restrictions=None, repeats: int = 2, max_rows: int = 600_000, path: str | None = TABLE_PATH,
         candidates=None, log=print) -> dict:
    """Time every candidate setting on each bucket's instances (at most max_rows rows of
    them, taken in order) and return {bucket: setting}; then time the whole set as one
    context per candidate setting and as concurrent buckets, and keep the faster mode.
    Written to ``path`` as JSON (with the measured times) unless path is None."""
    candidates = candidates or CANDIDATES
    xs = _device(instances)
    buckets = group([_shape(x) for x in xs])
    table, timings = {}, {}
    for name, idx in sorted(buckets.items()):
        sel, rows = [], 0
        for q in idx:
            if sel and rows + xs[q].shape[0] > max_rows:
                break
            sel.append(xs[q])
            rows += xs[q].shape[0]
        ms = {}
        for cfg in candidates:
            key = f"{cfg['precision']}/k{cfg['cache_k']}/s{cfg['col_split']}"
            ms[key] = time_config(sel, cfg, restrictions, repeats)
        best = min(ms, key=ms.get)
        table[name] = next(c for c in candidates if f"{c['precision']}/k{c['cache_k']}/s{c['col_split']}" == best)
        timings[name] = {"instances": len(sel), "rows": rows, "ms": ms, "best": best}
        if log:
            log(f"{name}: {len(sel)} instances, {rows} rows: best {best} ({ms[best]:.2f} ms); " +
                ", ".join(f"{k} {v:.2f}" for k, v in ms.items()))
    # the whole set: one context per candidate setting, and the tuned buckets concurrently
    whole = {}
    for cfg in candidates:
        key = f"{cfg['precision']}/k{cfg['cache_k']}/s{cfg['col_split']}"
        whole[key] = _time(lambda: _run_grouped(xs, table, restrictions, mode="single", global_cfg=cfg), repeats)
    best_single = min(whole, key=whole.get)
    grouped_ms = _time(lambda: _run_grouped(xs, table, restrictions), repeats)
    mode = "grouped" if grouped_ms < whole[best_single] else "single"
    global_cfg = next(c for c in candidates if f"{c['precision']}/k{c['cache_k']}/s{c['col_split']}" == best_single)
    if log:
        log(f"whole set: one context {', '.join(f'{k} {v:.1f}' for k, v in whole.items())} ms; "
            f"tuned buckets concurrently {grouped_ms:.1f} ms -> {mode}")
    if path:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        doc = {"device": torch.cuda.get_device_name(), "written": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
               "n_edges": list(N_EDGES), "d_edges": list(D_EDGES), "table": table, "timings": timings,
               "mode": mode, "global": global_cfg, "whole_set_ms": {"single": whole, "grouped": grouped_ms}}
        with open(path, "w") as f:
            json.dump(doc, f, indent=1, sort_keys=True)
    return table


def load_table(path: str = TABLE_PATH) -> dict:
    """The tuned table ({bucket: setting}); {} when there is none or its buckets differ."""
    return dict(load_tuning(path).get("table", {}))


def load_tuning(path: str = TABLE_PATH) -> dict:
    """The whole tuning record: table, mode ("single" or "grouped") and the global
    setting; {} when there is none or its buckets differ."""
    try:
        with open(path) as f:
            doc = json.load(f)
    except (OSError, ValueError):
        return {}
    if tuple(doc.get("n_edges", ())) != N_EDGES or tuple(doc.get("d_edges", ())) != D_EDGES:
        return {}
    return doc


def run(instances, restrictions=None, tuning: dict | None = None, concurrent: bool = True):
    """The tuned run with results left on the device: [(instance indices, offsets,
    ClusterResult)], one entry per context."""
    tuning = load_tuning() if tuning is None else tuning
    mode = tuning.get("mode", "grouped")
    return _run_grouped(_device(instances), dict(tuning.get("table", {})), restrictions, concurrent, mode,
                        tuning.get("global"))


def cluster_batched(instances, restrictions=None, table: dict | None = None, concurrent: bool = True,
                    tuning: dict | None = None):
    """Cluster many independent instances with the tuned settings.

    instances: float32 [N_b, d_b] arrays or tensors (host or device).  With ``table``
    ({bucket: setting}) every bucket runs as its own context with its setting; otherwise
    the tuning record decides (one context with the global setting, or the buckets).
    Returns one (merges, labels, n_clusters) per instance, in order, with instance-local
    row indices: merges as nnm_merge records in acceptance order, labels int32 [N_b]
    numbered 0..K_b-1 by each cluster's smallest row."""
    if table is not None:
        tuning = {"mode": "grouped", "table": table}
    parts = run(instances, restrictions, tuning, concurrent)
    out = [None] * sum(len(idx) for idx, _, _ in parts)
    for idx, offsets, res in parts:
        merges = res.merges()
        lab = res.labels.cpu().numpy()
        off = np.asarray(offsets, dtype=np.int64)
        inst_of = np.searchsorted(off, merges["a"].astype(np.int64), side="right") - 1
        for b, q in enumerate(idx):
            lo, hi = int(off[b]), int(off[b + 1])
            m = merges[inst_of == b].copy()
            m["a"] -= lo
            m["b"] -= lo
            local = lab[lo:hi] - lab[lo]
            out[q] = (m, local.astype(np.int32), int(local.max()) + 1)
    return out


if __name__ == "__main__":
    from .inputs import batched_instances
    tune(batched_instances())
