"""Many filters in one launch per phase, against the oracle filter by filter.

Each filter of a many-filter call must end up exactly as if blowchoc_insert
and blowchoc_query had been called on it alone: words, bitmaps and counters
equal the oracle's for every filter, whatever the mix of sizes, hash range
kinds, choice counts, k and batch sizes in the work list.
"""
import numpy as np
import pytest

import workloads
from oracle import COST_MIX, COST_LA, COST_EXP
from oracle.oracle import GOLDEN_RATIO
from tests.gpu_helpers import to_dev, oracle_run

pytestmark = pytest.mark.gpu

# (M, k, c, cost, param, B, n)
MIX = [
    (32, 11, 2, COST_EXP, GOLDEN_RATIO, 16, 1000),
    (1000, 11, 2, COST_EXP, GOLDEN_RATIO, 1024, 30000),
    (999, 14, 3, COST_LA, 3.5, 2048, 25000),
    (6150, 9, 1, COST_MIX, 50.0, 4096, 40000),
    (1, 3, 2, COST_MIX, 50.0, 1024, 300),
    (4096, 20, 3, COST_MIX, 2.5, 100000, 60000),
    (777, 7, 2, COST_LA, 3.5, 1, 3000),        # sequential: single-filter kernel
    (2048, 16, 2, COST_EXP, GOLDEN_RATIO, 1 << 20, 50000),
    (512, 12, 3, COST_EXP, GOLDEN_RATIO, 1500, 0),   # empty
    (300, 5, 1, COST_EXP, GOLDEN_RATIO, 1024, 9000),
    (257, 32, 2, COST_MIX, 50.0, 1030, 12345),
]


def _setup(bc, cases, seed0):
    filters, keys, queries = [], [], []
    for j, (M, k, c, kind, par, B, n) in enumerate(cases):
        filters.append(bc.Filter(M, k, c, kind, par, hash_seed=seed0 + j, batch=B))
        kk = workloads.uniform_keys(seed0 * 100 + j, n)
        neg = workloads.disjoint_keys(seed0 * 100 + j + 50, n // 2 + 1, kk)
        keys.append(kk)
        queries.append(np.concatenate([kk[: n // 2], neg]))
    return filters, keys, queries


def _check_against_oracle(cases, filters, keys, queries, bitmaps, seed0):
    for j, (M, k, c, kind, par, B, n) in enumerate(cases):
        o, obm, _, _ = oracle_run(M, k, c, kind, par, seed0 + j, B, keys[j], queries[j])
        assert np.array_equal(filters[j].words_host(), o.words), j
        got = bitmaps[j].cpu().numpy().view(np.uint64)[: (len(queries[j]) + 63) // 64]
        assert np.array_equal(got, obm), j
        st = filters[j].stats()
        assert (st.inserted, st.skipped) == (o.inserted, o.skipped), j


@pytest.mark.parametrize("tune", [dict(cluster_max=16, lanes_cluster=4), dict(cluster_max=16, lanes_cluster=8),
                                  dict(cluster_max=2, lanes_cluster=4), dict(cluster_max=0)],
                         ids=["cluster16", "cluster16-lanes8", "cluster2", "worklist-only"])
def test_insert_and_query_many_match_the_oracle(tune):
    """The mix runs partly cluster-resident (small filters with at least four
    batches, one cluster per filter) and partly over the work list; with
    cluster_max = 0 all of it over the work list."""
    import torch
    import paper_2501_18977_gb300 as bc
    seed0 = 11
    filters, keys, queries = _setup(bc, MIX, seed0)
    dk = [to_dev(k) for k in keys]
    dq = [to_dev(q) for q in queries]
    bms = [torch.zeros(max(1, (len(q) + 63) // 64), dtype=torch.int64, device="cuda") for q in queries]
    batch = bc.Batch()
    try:
        batch.set_tuning(**tune)
        batch.insert_many([(f, d, len(k), None) for f, d, k in zip(filters, dk, keys)])
        batch.query_many([(f, d, len(q), b) for f, d, q, b in zip(filters, dq, queries, bms)])
        torch.cuda.synchronize()
        _check_against_oracle(MIX, filters, keys, queries, bms, seed0)
    finally:
        batch.close()
        for f in filters:
            f.close()


def test_many_equals_one_call_per_filter():
    """Two many-filter calls in a row compose like two calls per filter."""
    import torch
    import paper_2501_18977_gb300 as bc
    cases = MIX[:6]
    a, keys, _ = _setup(bc, cases, 5)
    b, _, _ = _setup(bc, cases, 5)
    batch = bc.Batch()
    try:
        halves = [(k[: len(k) // 2], k[len(k) // 2:]) for k in keys]
        for part in (0, 1):
            dks = [to_dev(h[part]) for h in halves]
            batch.insert_many([(f, d, len(h[part]), None) for f, d, h in zip(a, dks, halves)])
            for f, d, h in zip(b, dks, halves):
                f.insert(d)
        torch.cuda.synchronize()
        for fa, fb in zip(a, b):
            assert np.array_equal(fa.words_host(), fb.words_host())
    finally:
        batch.close()
        for f in a + b:
            f.close()


def test_recorded_graph_replays_the_same_work():
    import torch
    import paper_2501_18977_gb300 as bc
    cases = [MIX[1], MIX[2], MIX[5], MIX[7]]
    seed0 = 21
    filters, keys, queries = _setup(bc, cases, seed0)
    dk = [to_dev(k) for k in keys]
    dq = [to_dev(q) for q in queries]
    bms = [torch.zeros(max(1, (len(q) + 63) // 64), dtype=torch.int64, device="cuda") for q in queries]
    batch = bc.Batch()
    try:
        batch.record([(f, d, len(k), None) for f, d, k in zip(filters, dk, keys)],
                     [(f, d, len(q), b) for f, d, q, b in zip(filters, dq, queries, bms)])
        for rep in range(2):
            for f in filters:
                f.clear()
            batch.replay()
            torch.cuda.synchronize()
            _check_against_oracle(cases, filters, keys, queries, bms, seed0)
    finally:
        batch.close()
        for f in filters:
            f.close()


def test_autotune_leaves_filters_untouched_and_results_unchanged():
    import torch
    import paper_2501_18977_gb300 as bc
    cases = [MIX[1], MIX[3], MIX[7]]
    seed0 = 31
    filters, keys, queries = _setup(bc, cases, seed0)
    dk = [to_dev(k) for k in keys]
    dq = [to_dev(q) for q in queries]
    bms = [torch.zeros(max(1, (len(q) + 63) // 64), dtype=torch.int64, device="cuda") for q in queries]
    batch = bc.Batch()
    try:
        ins = [(f, d, len(k), None) for f, d, k in zip(filters, dk, keys)]
        qry = [(f, d, len(q), b) for f, d, q, b in zip(filters, dq, queries, bms)]
        best = batch.autotune(ins, qry)
        assert best.lanes_choose in (1, 2, 4) and best.ctas_per_sm in (4, 8)
        for f in filters:
            assert not f.words_host().any()
        batch.insert_many(ins)
        batch.query_many(qry)
        torch.cuda.synchronize()
        _check_against_oracle(cases, filters, keys, queries, bms, seed0)
    finally:
        batch.close()
        for f in filters:
            f.close()


def _classes_present(bc, batch, cases):
    return sorted({(batch.size_class(M), k, c) for (M, k, c, kind, par, B, n) in cases})


# class tunings forced on every (size class, k, c) of the mix
CLASS_CONFIGS = [
    dict(route=0, lanes_choose=8, tile=32, lanes_query=4, query_early=0),
    dict(route=0, lanes_choose=1, tile=1024, lanes_query=8, query_early=1),
    dict(route=0, lanes_choose=2, tile=256, lanes_query=1, query_early=0),
    dict(route=1, lanes_choose=4, tile=64, lanes_query=2, query_early=1),
    dict(route=2, lanes_choose=4, tile=128, lanes_query=1, query_early=1),
]


@pytest.mark.parametrize("cfg", CLASS_CONFIGS, ids=["wl-l8-t32", "wl-l1-t1024", "wl-l2-t256", "direct", "sorted"])
def test_class_tunings_keep_results(cfg):
    """Whatever launch configuration a size class gets (work-list lanes and
    tile, direct or sort-by-block single-filter route, query lanes and early
    exit), every filter's words, bitmap and counters equal the oracle's."""
    import torch
    import paper_2501_18977_gb300 as bc
    seed0 = 41
    cases = [c for c in MIX if c[5] != 1]
    filters, keys, queries = _setup(bc, cases, seed0)
    dk = [to_dev(k) for k in keys]
    dq = [to_dev(q) for q in queries]
    bms = [torch.zeros(max(1, (len(q) + 63) // 64), dtype=torch.int64, device="cuda") for q in queries]
    batch = bc.Batch()
    try:
        for cls, k, c in _classes_present(bc, batch, cases):
            batch.set_class_tuning(cls, k, c, **cfg)
            got, is_set = batch.class_tuning(cls, k, c)
            assert is_set and got == cfg
        batch.insert_many([(f, d, len(kk), None) for f, d, kk in zip(filters, dk, keys)])
        batch.query_many([(f, d, len(q), b) for f, d, q, b in zip(filters, dq, queries, bms)])
        torch.cuda.synchronize()
        _check_against_oracle(cases, filters, keys, queries, bms, seed0)
        # the filters' own launch fields are restored after a routed call
        for f in filters:
            t = f.tuning()
            assert (t.set_mode, t.persistent) == (0, 1)
    finally:
        batch.close()
        for f in filters:
            f.close()


def test_class_tuning_api_checks_and_classes():
    import paper_2501_18977_gb300 as bc
    batch = bc.Batch()
    try:
        # classes by filter bytes against L2: tiny, a quarter of L2, twice L2, 8 GiB
        assert batch.size_class(64) == bc.CLASS_CACHE
        assert batch.size_class(1 << 27 >> 6) in (bc.CLASS_L2, bc.CLASS_SPILL)
        assert batch.size_class((1 << 33) >> 6) == bc.CLASS_HBM
        t, is_set = batch.class_tuning(1, 11, 2)
        assert not is_set and t["route"] == 0 and t["tile"] == 128
        for bad in (dict(route=3), dict(lanes_choose=3), dict(tile=48), dict(tile=2048), dict(query_early=2)):
            with pytest.raises(bc.BlowChocError) as ei:
                batch.set_class_tuning(1, 11, 2, **bad)
            assert ei.value.code == bc.BLOWCHOC_EINVAL
        with pytest.raises(bc.BlowChocError):
            batch.class_tuning(4, 11, 2)
        batch.set_class_tuning(1, 11, 2, tile=512)
        assert batch.class_tuning(1, 11, 2)[1]
        batch.clear_class_tuning()
        assert not batch.class_tuning(1, 11, 2)[1]
    finally:
        batch.close()


def test_autotuned_classes_match_the_oracle():
    """After the per-class autotune, every (size class, k, c) of the mix has
    a cached tuning, and the tuned call is bit-exact against the oracle."""
    import torch
    import paper_2501_18977_gb300 as bc
    seed0 = 51
    cases = [c for c in MIX if c[5] != 1]
    filters, keys, queries = _setup(bc, cases, seed0)
    dk = [to_dev(k) for k in keys]
    dq = [to_dev(q) for q in queries]
    bms = [torch.zeros(max(1, (len(q) + 63) // 64), dtype=torch.int64, device="cuda") for q in queries]
    batch = bc.Batch()
    try:
        ins = [(f, d, len(kk), None) for f, d, kk in zip(filters, dk, keys)]
        qry = [(f, d, len(q), b) for f, d, q, b in zip(filters, dq, queries, bms)]
        batch.autotune(ins, qry)
        for cls, k, c in _classes_present(bc, batch, [cs for cs in cases if cs[6] > 0]):
            assert batch.class_tuning(cls, k, c)[1], (cls, k, c)
        for f in filters:
            assert not f.words_host().any()
        batch.insert_many(ins)
        batch.query_many(qry)
        torch.cuda.synchronize()
        _check_against_oracle(cases, filters, keys, queries, bms, seed0)
    finally:
        batch.close()
        for f in filters:
            f.close()


def test_many_rejects_a_repeated_filter():
    import paper_2501_18977_gb300 as bc
    f = bc.Filter(64, 8, 2, bc.COST_MIX, 50.0, hash_seed=1, batch=2048)
    batch = bc.Batch()
    try:
        d = to_dev(workloads.uniform_keys(1, 100))
        with pytest.raises(bc.BlowChocError) as ei:
            batch.insert_many([(f, d, 100, None), (f, d, 100, None)])
        assert ei.value.code == bc.BLOWCHOC_EINVAL
    finally:
        batch.close()
        f.close()


def test_many_filter_workload_full_size_matches_oracle_digests():
    """The 256-filter workload at full size, through insert_many and
    query_many, against the oracle's per-filter digests
    (tests/golden/many_filters_256.txt, written by make_golden.py many)."""
    import hashlib
    import os
    import torch
    import paper_2501_18977_gb300 as bc
    path = os.path.join(os.path.dirname(__file__), "golden", "many_filters_256.txt")
    rows = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or "|" not in line:
                continue
            f = [x.strip() for x in line.split("|")]
            rows[int(f[0])] = f
    cfg = workloads.many_filter_config()
    phi = GOLDEN_RATIO
    filters, ins, qry, bms, nq = [], [], [], [], []
    for it in cfg:
        keys, queries = workloads.many_filter_keys(it)
        f = bc.Filter(it["M"], 11, 2, bc.COST_EXP, phi, hash_seed=it["key_seed"], batch=it["B"])
        filters.append(f)
        dk, dq = to_dev(keys), to_dev(queries)
        b = torch.zeros(max(1, (len(queries) + 63) // 64), dtype=torch.int64, device="cuda")
        ins.append((f, dk, len(keys), None))
        qry.append((f, dq, len(queries), b))
        bms.append(b)
        nq.append(len(queries))
    batch = bc.Batch()
    try:
        batch.insert_many(ins)
        batch.query_many(qry)
        torch.cuda.synchronize()
        for it, f, b, n in zip(cfg, filters, bms, nq):
            row = rows[it["index"]]
            st = f.stats()
            assert (st.inserted, st.skipped) == (int(row[4]), int(row[5])), it["index"]
            assert hashlib.sha256(f.words_host().astype("<u8").tobytes()).hexdigest() == row[6], it["index"]
            h = b.cpu().numpy().view(np.uint64)[: (n + 63) // 64]
            assert hashlib.sha256(h.astype("<u8").tobytes()).hexdigest() == row[7], it["index"]
    finally:
        batch.close()
        for f in filters:
            f.close()
