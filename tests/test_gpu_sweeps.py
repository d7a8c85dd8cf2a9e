"""The pieces of the paper-scale sweeps on the device: generated keys equal
the host input generator's stream, the counted query equals the bitmap and
the oracle, a whole sweep point equals the oracle's filter, and the
histogram FPR estimate of distinct bit selection predicts the measured rate."""
import math

import numpy as np
import pytest

import workloads
from oracle import COST_EXP, COST_MIX, OracleFilter
from oracle.oracle import GOLDEN_RATIO, bits_of_bitmap
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,n,start", [(1, 1000003, 0), (3001, 70001, 12345), (2**64 - 1, 999, 2**40),
                                          (7, 1, 5)])
def test_generated_keys_equal_the_host_stream(seed, n, start):
    import paper_2501_18977_gb300 as bc
    out = bc.generate_keys(n, seed, start).cpu().numpy().view(np.uint64)
    assert np.array_equal(out, workloads.splitmix64(seed, n, start))


def test_generated_keys_sampled_at_scale():
    """2^28 keys from a large offset: sampled positions against the host."""
    import torch
    import paper_2501_18977_gb300 as bc
    n, start = 1 << 28, 3 * 10**9
    out = bc.generate_keys(n, 42, start)
    pos = np.random.default_rng(0).integers(0, n, 4096)
    got = out[torch.from_numpy(pos).cuda()].cpu().numpy().view(np.uint64)
    assert np.array_equal(got, workloads.splitmix64_at(42, pos + start))
    del out


@pytest.mark.parametrize("M,k,c,bitsel,early", [(2048, 10, 2, 0, 1), (999, 14, 3, 1, 0), (512, 7, 1, 0, 1),
                                                (1500, 16, 3, 0, 2)])
def test_query_count_equals_bitmap_and_oracle(M, k, c, bitsel, early):
    import torch
    import paper_2501_18977_gb300 as bc
    n = int(M * 512 * math.log(2) / k)
    keys = workloads.uniform_keys(M + k, n)
    neg = workloads.uniform_keys(M + k + 1, 300001)
    queries = np.concatenate([keys[:1000], neg])
    f = bc.Filter(M, k, c, COST_EXP, GOLDEN_RATIO, hash_seed=11, batch=256, bitsel=bitsel)
    try:
        f.set_tuning(query_early=early)
        f.insert(to_dev(keys))
        dq = to_dev(queries)
        bm = f.query(dq).cpu().numpy().view(np.uint64)
        cnt = f.query_count(dq)
        acc = torch.full((1,), 5, dtype=torch.int64, device="cuda")
        f.query_count(dq, acc)
        f.query_count(dq[:0], acc)
        torch.cuda.synchronize()
    finally:
        f.close()
    o = OracleFilter(M, k, c, COST_EXP, GOLDEN_RATIO, seed=11, batch=256, bitsel=bitsel)
    o.insert(keys)
    W = int(bits_of_bitmap(o.query(queries), len(queries)).sum())
    assert cnt == int(bits_of_bitmap(bm, len(queries)).sum()) == W
    assert int(acc.item()) == W + 5


@pytest.mark.parametrize("k,c,cost,par,bitsel", [(10, 2, COST_EXP, GOLDEN_RATIO, 0), (14, 3, COST_MIX, 50.0, 1),
                                                 (4, 1, COST_EXP, GOLDEN_RATIO, 0)])
def test_sweep_point_matches_oracle(k, c, cost, par, bitsel):
    """fpr_point at a small n (device-generated keys in several chunks, the
    counted query over device-generated negatives) equals the oracle run on
    the host-generated streams."""
    from paper_2501_18977_gb300 import sweeps
    n, n_neg = 200003, 150001
    M = sweeps.blocks_for(n, k, 0.9)
    B = sweeps.batch_for(M)
    r = sweeps.fpr_point(n, M, k, c, cost, par, bitsel, key_seed=101, neg_seed=202, n_neg=n_neg,
                         hash_seed=77, chunk=3 * B + 5)
    o = OracleFilter(M, k, c, cost, par, seed=77, batch=B, bitsel=bitsel)
    o.insert(workloads.splitmix64(101, n))
    W = int(bits_of_bitmap(o.query(workloads.splitmix64(202, n_neg)), n_neg).sum())
    hist, _ = o.histogram()
    assert r["W"] == W and r["N"] == n_neg and r["B"] == B and r["M"] == M
    assert (r["inserted"], r["skipped"]) == (o.inserted, o.skipped)
    assert r["hist"] == [int(v) for v in hist]


def test_distinct_fpr_estimate_matches_measured():
    """With distinct bits a negative hits a block of load L with probability
    C(L, k) / C(512, k); the estimate from the histogram predicts W / N."""
    import paper_2501_18977_gb300 as bc
    M, k = 4096, 12
    n = int(M * 512 * math.log(2) / k)
    keys = workloads.uniform_keys(31, n)
    f = bc.Filter(M, k, 1, COST_EXP, GOLDEN_RATIO, hash_seed=3, batch=1 << 12, bitsel=1)
    try:
        f.insert(to_dev(keys))
        neg = bc.generate_keys(1 << 22, 32)
        W = f.query_count(neg)
        st = f.stats()
    finally:
        f.close()
    assert set(workloads.splitmix64(32, 1 << 22).tolist()).isdisjoint(keys.tolist())
    q = sum(int(h) * math.comb(L, k) for L, h in enumerate(st.hist)) / (M * math.comb(512, k))
    assert math.isclose(st.fpr_est, q, rel_tol=1e-9)
    N = 1 << 22
    assert abs(W - N * q) < 4.5 * math.sqrt(N * q * (1 - q))
