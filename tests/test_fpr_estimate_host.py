"""The library's histogram FPR estimate against closed forms, on the host.

blowchoc_stats turns the load histogram into an FPR estimate with host code
(blowchoc_fpr_estimate). With independent bit addresses a negative is
contained in a block of load L with probability (L/512)^k (Section 2.1 per
block); with k distinct addresses the probability is C(L, k) / C(512, k)
(Appendix B). These tests check the library's value against the oracle's
closed form and against exact rational arithmetic.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle.closed_forms import fpr_given_state


def _est(hist, k, c, bitsel=0):
    import paper_2501_18977_gb300 as bc
    return bc.blowchoc_fpr_estimate(hist, k, c, bitsel)


def _random_hist(seed, blocks=4096, mean=300.0, sd=20.0):
    rng = np.random.default_rng(seed)
    loads = np.clip(np.rint(rng.normal(mean, sd, blocks)), 0, 512).astype(np.int64)
    return np.bincount(loads, minlength=513).astype(np.uint64)


@pytest.mark.parametrize("k,c,seed", [(14, 2, 1), (16, 3, 2), (12, 1, 3), (1, 1, 4), (32, 3, 5)])
def test_random_bits_match_the_oracle_closed_form(k, c, seed):
    h = _random_hist(seed)
    assert _est(h, k, c) == pytest.approx(fpr_given_state(h, k, c), rel=1e-12, abs=1e-300)


@pytest.mark.parametrize("k,c", [(2, 1), (7, 2), (16, 3), (32, 1)])
def test_distinct_bits_match_exact_binomial_ratios(k, c):
    h = _random_hist(k + 10 * c, mean=420.0, sd=40.0)
    q = Fraction(0)
    for L, cnt in enumerate(h.tolist()):
        if cnt:
            q += cnt * Fraction(math.comb(L, k), math.comb(512, k))
    q /= int(h.sum())
    exact = 1.0 - (1.0 - float(q)) ** c
    assert _est(h, k, c, bitsel=1) == pytest.approx(exact, rel=1e-12, abs=1e-300)


def test_special_histograms():
    h = np.zeros(513, dtype=np.uint64)
    h[0] = 100                                  # empty filter: nothing is contained
    assert _est(h, 14, 3) == 0.0
    h[:] = 0
    h[512] = 7                                  # full filter: everything is contained
    assert _est(h, 14, 2) == 1.0
    assert _est(h, 14, 2, bitsel=1) == 1.0
    h[:] = 0
    h[256] = 3                                  # half-full blocks: 2^-k per candidate
    assert _est(h, 10, 1) == pytest.approx(2.0 ** -10, rel=1e-15)
    assert _est(h, 10, 2) == pytest.approx(1 - (1 - 2.0 ** -10) ** 2, rel=1e-15)
    h[:] = 0
    h[5] = 1                                    # fewer set bits than distinct addresses
    assert _est(h, 6, 1, bitsel=1) == 0.0


@pytest.mark.parametrize("k,c,bitsel,empty", [(0, 1, 0, False), (33, 1, 0, False), (4, 0, 0, False),
                                              (4, 4, 0, False), (4, 1, 2, False), (4, 1, 0, True)])
def test_bad_arguments_rejected(k, c, bitsel, empty):
    import ctypes
    import paper_2501_18977_gb300 as bc
    h = np.zeros(513, dtype=np.uint64)
    if not empty:
        h[100] = 1
    out = ctypes.c_double()
    rc = bc.load_library().blowchoc_fpr_estimate(h.ctypes.data, k, c, bitsel, ctypes.byref(out))
    assert rc == bc.BLOWCHOC_EINVAL
