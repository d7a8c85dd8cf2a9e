"""The library's cost ranks against the oracle's double costs, on the host.

The choose kernels never evaluate a cost: they compare integer ranks that the
library computes once per filter from Eq. 4-6 (Section 3.2, Appendix A). The
ranks must order every reachable (load L, new bits a) exactly as the oracle's
IEEE-double costs do, ties included, or some choice would differ from the
oracle's. These tests check that over the whole table, for each cost kind at
the parameters the configurations use and at the edges of k.
"""
import numpy as np
import pytest

from oracle import COST_EXP, COST_LA, COST_MIX
from oracle.oracle import GOLDEN_RATIO, cost

UNREACHABLE = 0xFFFF

CASES = [
    (COST_MIX, 50.0, 14),        # small uniform and serving configurations
    (COST_MIX, 2.5, 7),          # the paper's sigma for k = 7
    (COST_MIX, 50.0, 12),        # overload sweep
    (COST_LA, 3.5, 16),          # DNA configuration
    (COST_LA, 3.5, 12),
    (COST_EXP, GOLDEN_RATIO, 11),  # many-filter configuration
    (COST_EXP, GOLDEN_RATIO, 32),  # largest k
    (COST_EXP, 1.2, 1),          # smallest k
    (COST_LA, 0.0, 5),           # mu = 0: cost^LA equals cost^MIX with sigma = 1
]


def _ranks(kind, par, k):
    import paper_2501_18977_gb300 as bc
    return bc.blowchoc_cost_ranks(kind, par, k)


@pytest.mark.parametrize("kind,par,k", CASES)
def test_ranks_order_the_oracle_costs_exactly(kind, par, k):
    ranks = _ranks(kind, par, k)
    k1 = k + 1
    assert ranks.shape == (513 * k1,)
    costs, got = [], []
    for L in range(513):
        for a in range(k1):
            if L + a > 512:
                assert ranks[L * k1 + a] == UNREACHABLE
                continue
            costs.append(cost(kind, par, k, L + a, a))
            got.append(int(ranks[L * k1 + a]))
    costs = np.array(costs)
    got = np.array(got)
    order = np.argsort(costs, kind="stable")
    c_sorted, r_sorted = costs[order], got[order]
    assert r_sorted[0] == 0
    same = c_sorted[1:] == c_sorted[:-1]
    step = np.diff(r_sorted)
    # equal doubles share a rank; a larger double has the next rank
    assert np.all(step[same] == 0)
    assert np.all(step[~same] == 1)
    assert r_sorted[-1] == len(np.unique(costs)) - 1


def test_la_with_mu_zero_ranks_like_mix_with_sigma_one():
    """cost^LA_mu(j, a) = cost^MIX_1(j + mu k, a) (Appendix A), so at mu = 0 the
    two tables are the same ranking."""
    k = 9
    assert np.array_equal(_ranks(COST_LA, 0.0, k), _ranks(COST_MIX, 1.0, k))


@pytest.mark.parametrize("kind,par,k,cap", [
    (COST_EXP, GOLDEN_RATIO, 0, None), (COST_EXP, GOLDEN_RATIO, 33, None), (7, 1.0, 4, None),
    (COST_EXP, 0.0, 4, None), (COST_MIX, -1.0, 4, None), (COST_MIX, float("nan"), 4, None),
    (COST_MIX, 50.0, 14, 513 * 15 - 1),
])
def test_bad_arguments_rejected(kind, par, k, cap):
    import ctypes
    import paper_2501_18977_gb300 as bc
    lib = bc.load_library()
    n = 513 * 34 if cap is None else cap
    out = np.zeros(max(n, 1), dtype=np.uint16)
    rc = lib.blowchoc_cost_ranks(int(kind), float(par), int(k), out.ctypes.data, ctypes.c_uint64(n))
    assert rc == bc.BLOWCHOC_EINVAL
