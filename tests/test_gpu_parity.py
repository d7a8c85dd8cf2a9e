"""Parity of the CUDA path with the oracle, element by element.

Filter words, query bitmaps, insert/skip counters and load histograms must be
bit-identical to the oracle's on the same seeded keys, for every batch size,
choice count, cost and hash range kind, including ragged tails and empty
inputs. All calls go through the C ABI.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import COST_MIX, COST_LA, COST_EXP
from oracle.oracle import GOLDEN_RATIO, bits_of_bitmap
from tests.gpu_helpers import gpu_run, oracle_run, to_dev

pytestmark = pytest.mark.gpu

PHI = GOLDEN_RATIO

# (M, k, c, cost, param, B, n): covers c = 1..3, all costs, pow2 / odd / even
# ranges, M = 1, k = 1 and 32, sequential, single-CTA and multi-launch batches
CASES = [
    (256, 14, 2, COST_MIX, 50.0, 1, 20000),
    (256, 14, 2, COST_MIX, 50.0, 64, 20000),
    (256, 14, 2, COST_MIX, 50.0, 16384, 40000),
    (256, 14, 2, COST_MIX, 50.0, 16385, 40000),
    (256, 14, 2, COST_MIX, 50.0, 65536, 70001),
    (1024, 16, 3, COST_LA, 3.5, 1, 30000),
    (1024, 16, 3, COST_LA, 3.5, 1000, 30000),
    (1024, 16, 3, COST_LA, 3.5, 20000, 50000),
    (999, 11, 2, COST_EXP, PHI, 1, 20000),
    (999, 11, 2, COST_EXP, PHI, 777, 20000),
    (999, 11, 2, COST_EXP, PHI, 30000, 70000),
    (1000, 12, 3, COST_EXP, PHI, 30000, 70000),
    (1000, 12, 3, COST_MIX, 2.5, 5, 10000),
    (77, 7, 1, COST_EXP, PHI, 1, 10000),
    (4096, 7, 1, COST_MIX, 50.0, 50000, 90000),
    (1, 3, 2, COST_MIX, 50.0, 1, 500),
    (1, 3, 3, COST_LA, 3.5, 100, 500),
    (2, 1, 2, COST_EXP, PHI, 17, 3000),
    (64, 32, 3, COST_MIX, 50.0, 1, 5000),
    (64, 32, 3, COST_EXP, PHI, 40000, 60000),
    (6150, 10, 2, COST_LA, 3.5, 1 << 20, 100000),
]


@pytest.mark.parametrize("cluster", [16, 0], ids=["cluster", "global"])
@pytest.mark.parametrize("M,k,c,kind,par,B,n", CASES)
def test_parity_small(M, k, c, kind, par, B, n, cluster):
    """Every case with the cluster-resident insert allowed (taken wherever the
    filter fits and there are at least four batches) and with it off."""
    seed = 1000 + M + k
    keys = workloads.uniform_keys(M * 7 + k, n)
    neg = workloads.disjoint_keys(M * 7 + k + 1, n // 2 + 13, keys)
    queries = np.concatenate([keys[: n // 2 + 7], neg])
    words, bm, st = gpu_run(M, k, c, kind, par, seed, B, keys, queries, tune=dict(cluster_max=cluster))
    o, obm, hist, total = oracle_run(M, k, c, kind, par, seed, B, keys, queries)
    assert np.array_equal(words, o.words)
    assert np.array_equal(bm, obm)
    assert (st.inserted, st.skipped) == (o.inserted, o.skipped)
    assert list(st.hist) == [int(v) for v in hist] and st.set_bits == total
    assert bits_of_bitmap(bm, n // 2 + 7).all()


def test_multipliers_match_the_oracle_derivation():
    import paper_2501_18977_gb300 as bc
    from oracle import derive_multipliers
    for M, k, c in [(1 << 21, 16, 3), (6150, 11, 2), (999, 32, 3), (1, 1, 1)]:
        f = bc.Filter(M, k, c, bc.COST_EXP, PHI, hash_seed=31337, batch=1)
        ab, af = f.multipliers()
        f.close()
        oab, oaf = derive_multipliers(31337, M, k, c)
        assert ab[:c] == [int(v) for v in oab] and af[:k] == [int(v) for v in oaf]


def test_insert_split_into_calls_at_batch_edges():
    """Insert calls that start at batch boundaries compose: two calls equal one."""
    M, k, c, B = 512, 12, 2, 4096
    keys = workloads.uniform_keys(5, 40000)
    w1, _, s1 = gpu_run(M, k, c, COST_MIX, 50.0, 9, B, keys, keys[:0])
    w2, _, s2 = gpu_run(M, k, c, COST_MIX, 50.0, 9, B, keys, keys[:0], chunks=[4096 * 3, 4096 * 7])
    assert np.array_equal(w1, w2) and s1.inserted == s2.inserted


def test_empty_and_ragged():
    import torch
    import paper_2501_18977_gb300 as bc
    f = bc.Filter(128, 9, 2, bc.COST_LA, 3.5, hash_seed=3, batch=100)
    try:
        empty = torch.zeros(0, dtype=torch.int64, device="cuda")
        f.insert(empty)
        assert f.query(empty).numel() == 0
        assert not f.words_host().any()
        keys = workloads.uniform_keys(8, 1000)
        f.insert(to_dev(keys))
        for n in [1, 63, 64, 65, 127, 999, 1000]:
            bm = torch.full(((n + 63) // 64,), -1, dtype=torch.int64, device="cuda")
            f.query(to_dev(keys[:n]), bitmap=bm)
            h = bm.cpu().numpy().view(np.uint64)
            assert bits_of_bitmap(h, n).all()
            tail = n % 64
            if tail:
                assert int(h[-1]) >> tail == 0
    finally:
        f.close()


def test_stats_fpr_estimate_matches_measured():
    """fpr_est of a one-choice filter predicts the measured W/N (binomial)."""
    M, k = 4096, 8
    n = int(M * 512 * math.log(2) / k)
    keys = workloads.uniform_keys(17, n)
    neg = workloads.disjoint_keys(18, 1 << 21, keys)
    words, bm, st = gpu_run(M, k, 1, COST_EXP, PHI, 2, 1 << 16, keys, neg)
    W = int(bits_of_bitmap(bm, len(neg)).sum())
    q = st.fpr_est
    sd = math.sqrt(len(neg) * q * (1 - q))
    assert abs(W - len(neg) * q) < 4.5 * sd


def test_config_small_uniform_full():
    """1M uniform keys into 2^24 bits, k = 14, two choices, cost^MIX sigma = 50,
    B = 65536 and B = 1; queries: the 1M keys plus 1M disjoint keys."""
    M, k, c = 32768, 14, 2
    keys = workloads.uniform_keys(1, 1000000)
    neg = workloads.disjoint_keys(1001, 1000000, keys)
    queries = np.concatenate([keys, neg])
    for B in (65536, 1):
        words, bm, st = gpu_run(M, k, c, COST_MIX, 50.0, 1, B, keys, queries)
        o, obm, hist, total = oracle_run(M, k, c, COST_MIX, 50.0, 1, B, keys, queries)
        assert np.array_equal(words, o.words), B
        assert np.array_equal(bm, obm), B
        assert (st.inserted, st.skipped) == (o.inserted, o.skipped)
        assert bits_of_bitmap(bm, len(keys)).all()


@pytest.mark.parametrize("tune", [
    dict(lanes_choose=2, lanes_set=2, lanes_query=2, query_early=0, ctas_per_sm=1, persistent=0, cluster_max=0),
    dict(lanes_choose=8, lanes_set=4, lanes_query=8, query_early=1, ctas_per_sm=3, persistent=0, cluster_max=0),
    dict(lanes_choose=4, lanes_set=8, lanes_query=4, query_early=0, ctas_per_sm=16, persistent=0, cluster_max=0),
    dict(lanes_choose=1, lanes_set=1, lanes_query=1, query_early=1, ctas_per_sm=2, persistent=0, cluster_max=0),
    dict(lanes_choose=1, lanes_set=2, lanes_query=1, query_early=0, ctas_per_sm=8, persistent=1, cluster_max=0),
    dict(lanes_choose=2, lanes_set=2, lanes_query=2, query_early=1, ctas_per_sm=1, persistent=1, cluster_max=0),
    dict(lanes_choose=8, lanes_set=2, lanes_query=4, query_early=1, ctas_per_sm=16, persistent=1, cluster_max=0),
    dict(lanes_choose=2, lanes_set=2, lanes_query=1, query_early=1, ctas_per_sm=8, persistent=1,
         keys_per_cta=32, cluster_max=0),
    dict(lanes_choose=4, lanes_set=2, lanes_query=1, query_early=1, ctas_per_sm=4, persistent=1,
         keys_per_cta=1 << 20, cluster_max=0),
    dict(lanes_choose=2, lanes_set=2, lanes_query=1, query_early=1, ctas_per_sm=8, persistent=1,
         set_mode=1, cluster_max=0),
    dict(lanes_choose=4, lanes_set=2, lanes_query=1, query_early=1, ctas_per_sm=2, persistent=1,
         keys_per_cta=64, set_mode=1, cluster_max=0),
    dict(lanes_choose=8, lanes_set=2, lanes_query=1, query_early=1, ctas_per_sm=16, persistent=1,
         set_mode=1, cluster_max=0),
    dict(lanes_choose=1, lanes_set=2, lanes_query=1, query_early=1, ctas_per_sm=8, persistent=1,
         set_mode=2, cluster_max=0),
    dict(lanes_choose=2, lanes_set=2, lanes_query=1, query_early=1, ctas_per_sm=8, persistent=1,
         set_mode=2, cluster_max=0),
    dict(lanes_choose=4, lanes_set=2, lanes_query=1, query_early=1, ctas_per_sm=3, persistent=1,
         keys_per_cta=64, set_mode=2, cluster_max=0),
    dict(lanes_choose=8, lanes_set=2, lanes_query=1, query_early=1, ctas_per_sm=16, persistent=1,
         set_mode=2, cluster_max=0),
    dict(lanes_choose=2, lanes_set=4, lanes_query=1, query_early=2, ctas_per_sm=8, persistent=1, cluster_max=0),
    dict(lanes_choose=2, lanes_set=4, lanes_query=2, query_early=2, ctas_per_sm=8, persistent=1, cluster_max=0),
    dict(cluster_max=16, lanes_cluster=4),
    dict(cluster_max=16, lanes_cluster=8),
    dict(cluster_max=2, lanes_cluster=8),
    dict(cluster_max=3, lanes_cluster=4),
    dict(cluster_max=1, lanes_cluster=4),   # does not fit one CTA: global-memory kernels
])
def test_results_independent_of_launch_configuration(tune):
    """Every launch configuration gives the oracle's words and bitmap."""
    import paper_2501_18977_gb300 as bc
    M, k, c, B = 4096, 16, 3, 50000
    keys = workloads.uniform_keys(123, 200000)
    neg = workloads.disjoint_keys(124, 100000, keys)
    queries = np.concatenate([keys[:100000], neg])
    f = bc.Filter(M, k, c, bc.COST_LA, 3.5, hash_seed=7, batch=B)
    try:
        f.set_tuning(**tune)
        t = f.tuning()
        assert all(getattr(t, kk) == vv for kk, vv in tune.items())
        f.insert(to_dev(keys))
        bm = f.query(to_dev(queries)).cpu().numpy().view(np.uint64)
        words = f.words_host()
    finally:
        f.close()
    o, obm, _, _ = oracle_run(M, k, c, COST_LA, 3.5, 7, B, keys, queries)
    assert np.array_equal(words, o.words)
    assert np.array_equal(bm, obm)


def test_set_tuning_rejects_bad_values():
    import paper_2501_18977_gb300 as bc
    f = bc.Filter(64, 8, 2, bc.COST_MIX, 50.0, hash_seed=1, batch=1)
    try:
        before = (f.tuning().lanes_query, f.tuning().ctas_per_sm)
        for bad in [dict(lanes_query=3), dict(lanes_choose=16), dict(query_early=3),
                    dict(ctas_per_sm=0), dict(ctas_per_sm=17), dict(persistent=2),
                    dict(keys_per_cta=8), dict(set_mode=3), dict(seq_window=16),
                    dict(seq_window=9000), dict(cluster_max=17), dict(lanes_cluster=2),
                    dict(lanes_cluster=16), dict(cluster_keys=8), dict(cluster_keys=(1 << 20) + 1)]:
            with pytest.raises(bc.BlowChocError):
                f.set_tuning(**bad)
        assert (f.tuning().lanes_query, f.tuning().ctas_per_sm) == before
    finally:
        f.close()


@pytest.mark.parametrize("M,k,c,kind,par,B,n", [
    (999, 11, 2, COST_EXP, PHI, 4096, 60000),      # partial last range
    (1, 5, 3, COST_MIX, 50.0, 3000, 20000),        # one block, one range
    (70000, 14, 2, COST_MIX, 50.0, 65536, 300000), # many ranges, dense batches
    (32768, 14, 2, COST_MIX, 50.0, 65536, 1000000),  # the small uniform configuration
    (6150, 16, 3, COST_LA, 3.5, 1 << 20, 200000),  # one batch
])
def test_sort_by_block_set_matches_oracle(M, k, c, kind, par, B, n):
    import paper_2501_18977_gb300 as bc
    keys = workloads.uniform_keys(M + 17, n)
    neg = workloads.disjoint_keys(M + 18, 50000, keys)
    queries = np.concatenate([keys[:50000], neg])
    f = bc.Filter(M, k, c, kind, par, hash_seed=5, batch=B)
    try:
        f.set_tuning(set_mode=1, persistent=1, cluster_max=0)
        f.insert(to_dev(keys))
        bm = f.query(to_dev(queries)).cpu().numpy().view(np.uint64)
        words = f.words_host()
        st = f.stats()
    finally:
        f.close()
    o, obm, _, _ = oracle_run(M, k, c, kind, par, 5, B, keys, queries)
    assert np.array_equal(words, o.words)
    assert np.array_equal(bm, obm)
    assert (st.inserted, st.skipped) == (o.inserted, o.skipped)


@pytest.mark.parametrize("M,k,c,kind,par,n,window,dups", [
    (32768, 14, 2, COST_MIX, 50.0, 200000, 2048, False),
    (999, 11, 3, COST_EXP, PHI, 60000, 32, False),
    (1, 5, 2, COST_LA, 3.5, 3000, 512, False),       # one block: every key waits for the last
    (64, 9, 3, COST_MIX, 2.5, 20000, 8192, True),    # many repeated keys
    (4096, 16, 2, COST_EXP, PHI, 50000, 100, True),
    (6150, 12, 1, COST_EXP, PHI, 40000, 1000, False),
    (2048, 14, 2, COST_MIX, 50.0, 30000, 0, False),  # the one-warp kernel
])
def test_exact_sequential_insert_matches_oracle(M, k, c, kind, par, n, window, dups):
    """B = 1 through the reservation rounds equals the oracle's one key after
    another, for any window, including long chains of conflicting keys."""
    import paper_2501_18977_gb300 as bc
    keys = workloads.uniform_keys(M + 3, n)
    if dups:
        keys = keys[np.random.default_rng(M).integers(0, max(n // 20, 1), n)]
    queries = np.concatenate([keys[:n // 2], workloads.uniform_keys(M + 4, n // 2)])
    f = bc.Filter(M, k, c, kind, par, hash_seed=2, batch=1)
    try:
        f.set_tuning(seq_window=window)
        f.insert(to_dev(keys))
        bm = f.query(to_dev(queries)).cpu().numpy().view(np.uint64)
        words = f.words_host()
        st = f.stats()
    finally:
        f.close()
    o, obm, _, _ = oracle_run(M, k, c, kind, par, 2, 1, keys, queries)
    assert np.array_equal(words, o.words)
    assert np.array_equal(bm, obm)
    assert (st.inserted, st.skipped) == (o.inserted, o.skipped)


@pytest.mark.parametrize("M,k,c,kind,par,B,n,window,dups", [
    (65536, 12, 2, COST_EXP, PHI, 16, 60000, 2048, False),
    (70001, 14, 3, COST_MIX, 50.0, 7, 30001, 2048, True),     # odd B, repeated keys, ragged end
    (4096, 16, 2, COST_LA, 3.5, 16, 40000, 64, False),        # windows of four batches
    (1, 5, 2, COST_MIX, 50.0, 2, 3000, 64, False),            # one block: every batch waits for the last
    (9000, 11, 1, COST_EXP, PHI, 3, 50000, 2048, False),
    (300, 20, 3, COST_EXP, PHI, 13, 20000, 8192, True),
])
def test_exact_batched_insert_matches_oracle(M, k, c, kind, par, B, n, window, dups):
    """Small batches through reservation rounds over whole batches equal the
    oracle's batch-after-batch insertion (cluster-resident path off)."""
    import paper_2501_18977_gb300 as bc
    keys = workloads.uniform_keys(M + 11, n)
    if dups:
        keys = keys[np.random.default_rng(M).integers(0, max(n // 20, 1), n)]
    queries = np.concatenate([keys[:n // 2], workloads.uniform_keys(M + 12, n // 2)])
    f = bc.Filter(M, k, c, kind, par, hash_seed=4, batch=B)
    try:
        f.set_tuning(seq_window=window, cluster_max=0)
        f.insert(to_dev(keys))
        bm = f.query(to_dev(queries)).cpu().numpy().view(np.uint64)
        words = f.words_host()
        st = f.stats()
    finally:
        f.close()
    o, obm, _, _ = oracle_run(M, k, c, kind, par, 4, B, keys, queries)
    assert np.array_equal(words, o.words)
    assert np.array_equal(bm, obm)
    assert (st.inserted, st.skipped) == (o.inserted, o.skipped)


def test_stats_async_equals_stats_and_the_oracle():
    """blowchoc_stats_async + blowchoc_stats_decode give what blowchoc_stats
    gives (counters, histogram, set bits, fpr_est) and the oracle's counters
    and histogram, queued on a side stream behind an insert, with no host
    wait between the calls; two raw buffers alternate over four rounds."""
    import torch
    import paper_2501_18977_gb300 as bc
    from oracle import OracleFilter
    M, k, c, B = 1500, 13, 3, 4096
    keys = workloads.uniform_keys(41, 240000)
    f = bc.Filter(M, k, c, COST_LA, 3.5, hash_seed=6, batch=B)
    o = OracleFilter(M, k, c, COST_LA, 3.5, seed=6, batch=B)
    try:
        s = torch.cuda.Stream()
        raws = [torch.zeros(bc.STATS_RAW_WORDS, dtype=torch.int64).pin_memory() for _ in range(2)]
        parts = np.array_split(keys, 4)
        seen = []
        for r, part in enumerate(parts):
            d = to_dev(part)
            f.insert(d, s)
            f.stats_async(raws[r % 2], s)
            s.synchronize()
            got = f.stats_decode(raws[r % 2])
            want = f.stats()
            o.insert(part)
            hist, total = o.histogram()
            assert (got.inserted, got.skipped, got.set_bits) == (want.inserted, want.skipped, want.set_bits)
            assert got.fpr_est == want.fpr_est
            assert list(got.hist) == list(want.hist)
            assert (got.inserted, got.skipped) == (o.inserted, o.skipped)
            assert np.array_equal(np.array(list(got.hist), dtype=np.uint64), np.asarray(hist, dtype=np.uint64))
            assert got.set_bits == total
            seen.append(got.inserted)
        assert seen == sorted(seen) and seen[-1] > 0
        with pytest.raises(ValueError):
            f.stats_async(torch.zeros(10, dtype=torch.int64), s)
    finally:
        f.close()
