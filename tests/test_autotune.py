"""Autotuned batched clustering: buckets, grouping and the tuned table (CPU), and the
grouped, concurrent run against the oracle instance by instance (GPU)."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1402_3789_gb300 import autotune  # noqa: E402


def test_buckets_cover_every_size_and_width():
    assert autotune.bucket_of(2, 1) == autotune.bucket_of(4095, 8)
    assert autotune.bucket_of(4095, 8) != autotune.bucket_of(4096, 8)
    assert autotune.bucket_of(4096, 9) != autotune.bucket_of(4096, 8)
    assert autotune.bucket_of(1 << 20, 32) == autotune.bucket_of(16384, 17)
    for bad in ((1, 4), (100, 0), (100, 33)):
        with pytest.raises(ValueError):
            autotune.bucket_of(*bad)
    names = {autotune.bucket_of(n, d) for n in (2, 5000, 20000) for d in (1, 10, 20)}
    assert len(names) == 9


def test_grouping_keeps_the_order_of_instances():
    shapes = [(3000, 4), (20000, 25), (3500, 5), (5000, 12), (20001, 25)]
    g = autotune.group(shapes)
    assert sorted(q for idx in g.values() for q in idx) == list(range(5))
    assert g[autotune.bucket_of(3000, 4)] == [0, 2]
    assert g[autotune.bucket_of(20000, 25)] == [1, 4]


def test_table_loading(tmp_path):
    p = tmp_path / "t.json"
    good = {"n_edges": list(autotune.N_EDGES), "d_edges": list(autotune.D_EDGES),
            "table": {"n2-4095_d1-8": {"precision": "fp32", "cache_k": 4, "col_split": 0}}}
    p.write_text(json.dumps(good))
    assert autotune.load_table(str(p)) == good["table"]
    p.write_text(json.dumps({**good, "n_edges": [2, 100]}))
    assert autotune.load_table(str(p)) == {}     # other buckets: not used
    assert autotune.load_table(str(tmp_path / "missing.json")) == {}
    # the committed table, when present, names valid settings for known buckets
    committed = autotune.load_table()
    names = {autotune.bucket_of(n, d) for n in (2, 5000, 20000) for d in (1, 10, 20)}
    for name, cfg in committed.items():
        assert name in names
        assert cfg["precision"] in ("bf16x3", "fp16", "fp32", "bf16") and 0 <= cfg["cache_k"] <= 16


@pytest.mark.gpu
@pytest.mark.parametrize("concurrent", [True, False])
def test_tuned_grouped_run_matches_the_oracle(concurrent):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1402_3789_gb300.inputs import batched_instances
    oracle.build()
    inst = [x for x in batched_instances(count=40, seed=19, n_lo=600, n_hi=6000, d_lo=3, d_hi=24)][:14]
    table = {autotune.bucket_of(*x.shape): cfg for x, cfg in
             zip(inst, [autotune.CANDIDATES[q % len(autotune.CANDIDATES)] for q in range(len(inst))])}
    restr = {"max_join_dist": 1.1, "kl3_max_size": 400, "kl4_min_size": 3}
    out = autotune.cluster_batched(inst, restr, table=table, concurrent=concurrent)
    assert len(out) == len(inst)
    for x, (m, lab, K) in zip(inst, out):
        _, om, olab, oK = oracle.cluster(x, restr)
        assert np.array_equal(m, om)
        assert np.array_equal(lab, olab) and K == oK
