"""Host logic of the paper-scale sweeps (no GPU): sizes, batches and the
disjointness of the inserted and negative key streams."""
import math

import numpy as np

import workloads
from oracle.closed_forms import (bloom_blocks as oracle_bloom_blocks, bloom_fpr as oracle_bloom_fpr,
                                 blocked_bloom_fpr as oracle_blocked_bloom_fpr)
from paper_2501_18977_gb300 import sweeps


def test_sizes_follow_appendix_c():
    """m = n k / ln 2 rounded up to a multiple of 512 bits (Appendix C)."""
    for n in (10**6, 123457, 2 * 10**9):
        for k in sweeps.PAPER_KS:
            assert sweeps.blocks_for(n, k) == oracle_bloom_blocks(n, k)
    # a relative size scales m before rounding
    n, k = 2 * 10**9, 14
    m = n * k / math.log(2.0)
    assert sweeps.blocks_for(n, k, 1.1) == math.ceil(1.1 * m / 512)


def test_bloom_reference_curve():
    for n, m, k in ((10**6, 1.2e7, 8), (2e9, 4e10, 14)):
        assert math.isclose(sweeps.bloom_fpr(n, m, k), oracle_bloom_fpr(n, m, k), rel_tol=1e-12)
    # at the standard size the formula gives about 2^-k (Section 2.1)
    n = 2e9
    for k in sweeps.PAPER_KS:
        assert abs(math.log2(sweeps.bloom_fpr(n, sweeps.bloom_bits(n, k), k)) + k) < 0.01


def test_blocked_bloom_reference_curve():
    for n, M, k in ((1e6, 30000, 8), (357913941, 1 << 23, 12), (2e9, 54095000, 14)):
        assert math.isclose(sweeps.blocked_bloom_fpr(n, M, k), oracle_blocked_bloom_fpr(n, M, k), rel_tol=1e-9)


def test_batch_rule():
    assert sweeps.batch_for(1) == 1
    assert sweeps.batch_for(64 * 1000) == 512
    assert sweeps.batch_for(1 << 40) == 1 << 20
    for M in (37, 4096, 10**7):
        B = sweeps.batch_for(M)
        assert B & (B - 1) == 0 and (B == 1 or B <= M / 64)


def test_stream_overlap_is_detected_exactly():
    """A negative seed that is the key seed advanced by d states overlaps the
    inserted keys exactly when 0 <= d < n (or -n_neg < d < 0)."""
    seed = 12345
    G = sweeps.GAMMA
    for d, n, n_neg, overlap in ((5, 10, 10, True), (10, 10, 10, False), (0, 1, 1, True),
                                 (-3, 10, 4, True), (-4, 10, 4, False), (1 << 40, 10**9, 10**9, False)):
        neg_seed = (seed + d * G) & sweeps.MASK64
        assert sweeps.streams_disjoint(seed, n, neg_seed, n_neg) == (not overlap)
        if abs(d) < 20:  # check against the streams themselves
            a = set(workloads.splitmix64(seed, n).tolist())
            b = set(workloads.splitmix64(neg_seed, n_neg).tolist())
            assert (len(a & b) > 0) == overlap
    # the seeds the sweeps use are disjoint at the paper's scale
    for k in sweeps.PAPER_KS:
        for s in (1, 2, 3):
            assert sweeps.streams_disjoint(s * 1000 + k, 2 * 10**9, s * 1000 + 500 + k, 2 * 10**9)
            assert sweeps.streams_disjoint(s * 7919 + k, 2 * 10**9, s * 7919 + 4000 + k, 2 * 10**9)
