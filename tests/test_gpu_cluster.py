"""Cluster-resident insertion vs the oracle.

A filter that fits in the shared memory of one thread-block cluster is held
there for a whole insert call: each batch (Section 3.2, the library's batch
rule) reads candidate blocks from the owning CTA and ORs bits in over
distributed shared memory. Words, bitmaps and counters must equal the
oracle's, for one to sixteen CTAs per cluster, both lane widths, every choice
count and cost, distinct bit selection, repeated keys and ragged last
batches; blowchoc_cluster_ctas must report the path actually planned.
"""
import numpy as np
import pytest

import workloads
from oracle import COST_MIX, COST_LA, COST_EXP, OracleFilter
from oracle.oracle import GOLDEN_RATIO
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu

PHI = GOLDEN_RATIO

# (M, k, c, cost, param, B, n, bitsel, cluster_max, lanes_cluster, dups)
CASES = [
    (2075, 14, 2, COST_MIX, 50.0, 1024, 30000, 0, 16, 4, False),   # a small serving filter
    (2075, 14, 2, COST_MIX, 50.0, 512, 30001, 0, 1, 8, False),     # one CTA, four passes, ragged last batch
    (1, 5, 2, COST_LA, 3.5, 7, 500, 0, 16, 4, False),              # one block
    (777, 16, 1, COST_EXP, PHI, 100, 5000, 0, 4, 8, False),        # one choice
    (5000, 20, 3, COST_MIX, 2.5, 3, 2000, 0, 16, 4, False),        # three keys per batch
    (3000, 20, 2, COST_EXP, PHI, 512, 20000, 1, 16, 4, False),     # distinct bits
    (3000, 13, 3, COST_EXP, PHI, 640, 20000, 1, 2, 8, False),
    (12000, 12, 3, COST_EXP, PHI, 4096, 60000, 0, 16, 4, False),   # several CTAs needed
    (40000, 12, 2, COST_LA, 3.5, 8192, 70000, 0, 16, 8, False),    # close to the largest
    (4096, 11, 2, COST_EXP, PHI, 2048, 50000, 0, 16, 4, True),     # repeated keys
    (12000, 32, 3, COST_MIX, 50.0, 50, 9000, 0, 5, 4, False),      # k = 32, five CTAs
]


@pytest.mark.parametrize("M,k,c,kind,par,B,n,bitsel,cmax,lanes,dups", CASES)
def test_cluster_insert_matches_oracle(M, k, c, kind, par, B, n, bitsel, cmax, lanes, dups):
    import paper_2501_18977_gb300 as bc
    keys = workloads.uniform_keys(M * 3 + k, n)
    if dups:
        keys = keys[np.random.default_rng(M).integers(0, n // 10, n)]
    queries = np.concatenate([keys[: n // 2], workloads.uniform_keys(M * 3 + k + 1, n // 2)])
    f = bc.Filter(M, k, c, kind, par, hash_seed=M + 5, batch=B, bitsel=bitsel)
    try:
        # batches above 2048 keys run cluster-resident only with the
        # persistent insert off
        f.set_tuning(cluster_max=cmax, lanes_cluster=lanes, persistent=0 if B > 2048 else 1)
        S = f.cluster_ctas(n)
        if S == 0 and M > 20000:
            pytest.skip("the device co-schedules no cluster large enough")
        assert 1 <= S <= cmax
        assert f.cluster_ctas(min(n, 3 * B)) == 0          # fewer than four batches
        f.insert(to_dev(keys))
        bm = f.query(to_dev(queries)).cpu().numpy().view(np.uint64)
        words = f.words_host()
        st = f.stats()
    finally:
        f.close()
    o = OracleFilter(M, k, c, kind, par, seed=M + 5, batch=B, bitsel=bitsel)
    o.insert(keys)
    assert np.array_equal(words, o.words)
    assert np.array_equal(bm, o.query(queries))
    assert (st.inserted, st.skipped) == (o.inserted, o.skipped)


def test_cluster_insert_continues_a_filter():
    """Insert calls that alternate between the cluster-resident path and the
    global-memory kernels build the oracle's filter (each call starts its own
    batches at its first key)."""
    import paper_2501_18977_gb300 as bc
    M, k, c, B = 3001, 14, 2, 256
    keys = workloads.uniform_keys(77, 40000)
    f = bc.Filter(M, k, c, bc.COST_MIX, 50.0, hash_seed=9, batch=B)
    o = OracleFilter(M, k, c, COST_MIX, 50.0, seed=9, batch=B)
    try:
        edges = [0, 5000, 5100, 20000, 20300, 40000]
        for i, (a, b) in enumerate(zip(edges[:-1], edges[1:])):
            f.set_tuning(cluster_max=16 if i % 2 == 0 else 0)
            f.insert(to_dev(keys[a:b]))
            o.insert(keys[a:b])
        words = f.words_host()
        st = f.stats()
    finally:
        f.close()
    assert np.array_equal(words, o.words)
    assert (st.inserted, st.skipped) == (o.inserted, o.skipped)


def test_cluster_shape_limits():
    """Filters beyond the cluster's shared memory are not planned; the plan
    follows cluster_max and the batch size."""
    import paper_2501_18977_gb300 as bc
    big = bc.Filter(1 << 20, 14, 2, bc.COST_MIX, 50.0, hash_seed=1, batch=1024)
    small = bc.Filter(1000, 14, 2, bc.COST_MIX, 50.0, hash_seed=1, batch=512)
    try:
        assert big.cluster_ctas(1 << 20) == 0
        assert small.cluster_ctas(1 << 20) >= 1
        small.set_tuning(cluster_max=0)
        assert small.cluster_ctas(1 << 20) == 0
        small.set_tuning(cluster_max=1, lanes_cluster=8)
        assert small.cluster_ctas(1 << 20) == 1          # 512 keys on 128 lane groups: four passes
        small.set_tuning(cluster_max=1, lanes_cluster=8, cluster_keys=16)
        assert small.cluster_ctas(1 << 20) == 1
        wide = bc.Filter(1000, 14, 2, bc.COST_MIX, 50.0, hash_seed=1, batch=1024)
        wide.set_tuning(cluster_max=1, lanes_cluster=8)
        assert wide.cluster_ctas(1 << 20) == 0           # eight passes per batch: grid-wide kernels
        wide.close()
        # batches above 2048 keys take the persistent insert over the whole
        # grid unless it is off
        mid = bc.Filter(9022, 14, 2, bc.COST_MIX, 50.0, hash_seed=1, batch=4096)
        assert mid.cluster_ctas(1 << 20) == 0
        mid.set_tuning(persistent=0)
        assert mid.cluster_ctas(1 << 20) >= 1
        mid.close()
    finally:
        big.close()
        small.close()
