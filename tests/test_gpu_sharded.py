"""Sub-arrays (Section 3.4) on one GPU against the oracle's split filter.

The partition kernel must give each sub-array's keys in input order (exact
integer work: keys, input indices and offsets equal a stable sort by h_0),
and a filter split into T sub-arrays on the current GPU (partition, one
insert or query per sub-array, unpermute) must give the oracle's words and
bitmaps bit for bit.
"""
import numpy as np
import pytest

import workloads
from oracle.oracle import COST_MIX, COST_LA, COST_EXP, GOLDEN_RATIO
from oracle.sharded import ShardedOracle, shard_layout
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,T", [(0, 4), (1, 3), (31, 2), (4097, 5), (100003, 8), (250000, 1024), (70000, 1)])
def test_partition_is_a_stable_sort_by_h0(n, T):
    import torch
    import paper_2501_18977_gb300 as bc
    keys = workloads.uniform_keys(300 + T, n)
    a0, _, _ = shard_layout(1000, T, 42)
    ref = ShardedOracle(1000, T, 8, 2, COST_EXP, GOLDEN_RATIO, seed=42)
    sh = ref.shard_of(keys)
    order = np.argsort(sh, kind="stable")
    want_off = np.concatenate([[0], np.cumsum(np.bincount(sh, minlength=T))]).astype(np.int64)
    d = to_dev(keys) if n else torch.empty(0, dtype=torch.int64, device="cuda")
    out_k = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    out_i = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    off = torch.full((T + 1,), -1, dtype=torch.int64, device="cuda")
    sw = bc.blowchoc_shard_partition_scratch(n, T)
    scratch = torch.empty(max(sw, 1), dtype=torch.int64, device="cuda")
    bc.blowchoc_shard_partition(d, n, T, a0, out_k, out_i, off, scratch, sw)
    torch.cuda.synchronize()
    if n == 0:
        assert not off.cpu().numpy().any()
        return
    assert np.array_equal(off.cpu().numpy(), want_off)
    assert np.array_equal(out_i.cpu().numpy()[:n], order)
    assert np.array_equal(out_k.cpu().numpy().view(np.uint64)[:n], keys[order])


def test_partition_rejects_bad_arguments():
    import torch
    import paper_2501_18977_gb300 as bc
    d = to_dev(workloads.uniform_keys(1, 100))
    buf = torch.empty(100, dtype=torch.int64, device="cuda")
    off = torch.empty(4, dtype=torch.int64, device="cuda")
    sw = bc.blowchoc_shard_partition_scratch(100, 3)
    scratch = torch.empty(sw, dtype=torch.int64, device="cuda")
    for args in [(d, 100, 0, 3), (d, 100, 1025, 3), (d, 100, 3, 4)]:   # T = 0, T > 1024, even a0
        with pytest.raises(bc.BlowChocError):
            bc.blowchoc_shard_partition(args[0], args[1], args[2], args[3], buf, buf, off, scratch, sw)
    with pytest.raises(bc.BlowChocError):
        bc.blowchoc_shard_partition(d, 100, 3, 5, buf, buf, off, scratch, sw - 1)


@pytest.mark.parametrize("M,T,k,c,kind,par,B", [
    (4096, 1, 14, 2, COST_MIX, 50.0, 8192),
    (4096, 2, 14, 2, COST_MIX, 50.0, 8192),
    (3000, 3, 12, 3, COST_LA, 3.5, 1),
    (20000, 8, 11, 2, COST_EXP, GOLDEN_RATIO, 50000),
    (777, 5, 16, 1, COST_EXP, GOLDEN_RATIO, 100),
])
def test_split_filter_on_one_gpu_matches_the_oracle(M, T, k, c, kind, par, B):
    import torch
    import paper_2501_18977_gb300 as bc
    from paper_2501_18977_gb300.sharded import ShardedFilter
    n = 120000 if B > 1 else 20000
    keys = workloads.uniform_keys(500 + T, n)
    queries = np.concatenate([keys[::3], workloads.uniform_keys(600 + T, n // 2)])
    ref = ShardedOracle(M, T, k, c, kind, par, seed=77, batch=B)
    sf = ShardedFilter(M, T, k, c, kind, par, hash_seed=77, batch=B)
    try:
        # two insert calls, as two oracle insert calls
        half = n // 2
        sf.insert(to_dev(keys[:half]))
        sf.insert(to_dev(keys[half:]))
        ref.insert(keys[:half])
        ref.insert(keys[half:])
        bm = sf.query(to_dev(queries))
        torch.cuda.synchronize()
        assert np.array_equal(sf.words_host(), ref.words)
        want = ref.query(queries)
        assert np.array_equal(bm.cpu().numpy().view(np.uint64)[: len(want)], want)
        ins = sum(sf.subs[t].stats().inserted for t in sf.subs)
        assert ins == ref.inserted
    finally:
        sf.close()
