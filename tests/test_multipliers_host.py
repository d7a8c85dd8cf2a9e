"""The library's hash multipliers against the oracle's, on the host.

Every address the kernels compute is a·x with multipliers the library draws
at filter creation (Section 3.4; Appendix B for distinct bits). They must be
the oracle's for every seed and hash range, including the ranges where the
coprimality redraw matters: M even, M a power of two, M = 1, and the shrinking
ranges 512 - i of distinct bit selection.
"""
import numpy as np
import pytest

from oracle.oracle import derive_multipliers

SIZES = [1, 2, 3, 5, 64, 100, 1000, 2075, 32768, 65535, 65536, (1 << 21), (1 << 21) + 6, 3 ** 13, 1 << 32]


@pytest.mark.parametrize("M", SIZES)
@pytest.mark.parametrize("bitsel", [0, 1])
def test_multipliers_equal_the_oracle(M, bitsel):
    import paper_2501_18977_gb300 as bc
    for seed in (0, 1, 42, 3001, (1 << 64) - 1):
        for k, c in ((1, 1), (14, 2), (16, 3), (32, 3)):
            got_block, got_bit = bc.blowchoc_derive_multipliers(M, k, c, seed, bitsel)
            want_block, want_bit = derive_multipliers(seed, M, k, c, bitsel)
            assert got_block == [int(v) for v in want_block]
            assert got_bit == [int(v) for v in want_bit]


def test_multipliers_rejected_with_the_create_rules():
    import paper_2501_18977_gb300 as bc
    for M, k, c, b in ((0, 14, 2, 0), ((1 << 32) + 1, 14, 2, 0), (10, 0, 2, 0), (10, 33, 2, 0), (10, 14, 0, 0),
                       (10, 14, 4, 0), (10, 14, 2, 2)):
        with pytest.raises(bc.BlowChocError):
            bc.blowchoc_derive_multipliers(M, k, c, 1, b)


def test_multipliers_odd_and_coprime():
    import math
    import paper_2501_18977_gb300 as bc
    a_block, a_bit = bc.blowchoc_derive_multipliers(6000, 32, 3, 7, 1)
    assert all(a & 1 for a in a_block + a_bit)
    assert all(math.gcd(a, 6000) == 1 for a in a_block)
    assert all(math.gcd(a, 512 - i) == 1 for i, a in enumerate(a_bit))
    assert len(set(np.array(a_bit, dtype=np.uint64).tolist())) == 32
