"""Closed forms the paper states or relies on. Test infrastructure only.

Each function names the passage it follows. They serve as pins for the
oracle (statistical agreement of measured false-positive rates) and as the
reference curves of the FPR report.
"""
import math

import numpy as np

BLOCK_BITS = 512


def bloom_fpr(n: float, m: float, k: int) -> float:
    """Standard Bloom filter FPR p1^k with p1 = 1 - e^(-nk/m) (Section 2.1, Eq. 1)."""
    return (1.0 - math.exp(-n * k / m)) ** k


def bloom_overload_fpr(gamma: float, k: int) -> float:
    """FPR of a Bloom filter sized for load 1/2 but overloaded by gamma (Eq. 2)."""
    return (1.0 - 2.0 ** (-gamma)) ** k


def bloom_bits(n: float, k: int) -> float:
    """Bloom filter size for FPR 2^-k: m = n k / ln 2 (Section 2.1)."""
    return n * k / math.log(2.0)


def bloom_blocks(n: int, k: int) -> int:
    """Number of 512-bit blocks of a filter sized like a standard Bloom filter:
    m = nk/ln 2 rounded up to the next multiple of 512 (Appendix C)."""
    return int(math.ceil(bloom_bits(n, k) / BLOCK_BITS))


def load_bound(c: int, k: int) -> float:
    """Largest block load j with local FPR (j/512)^k <= 2^-k / c (Fig. 3A,
    Appendix C): j = 256 c^(-1/k)."""
    return 256.0 * c ** (-1.0 / k)


def birthday_collision(k: int, s: int = BLOCK_BITS) -> float:
    """P(|F(x)| < k) for k independent uniform positions in [s] (Fig. 3B)."""
    p = 1.0
    for i in range(k):
        p *= 1.0 - i / s
    return 1.0 - p


def blocked_bloom_fpr(n: float, M: int, k: int, imax: int = None) -> float:
    """One-choice Blocked Bloom FPR under ideal hashing (Putze et al., the
    model Section 2.2 cites): keys per block ~ Poisson(n/M); a block with i keys
    has each bit set with probability 1 - (1 - 1/512)^(ik); a query with k
    independent positions hits with that probability to the k-th power."""
    lam = n / M
    if imax is None:
        imax = int(lam + 12.0 * math.sqrt(lam + 1.0) + 20)
    i = np.arange(imax + 1, dtype=np.float64)
    logpois = -lam + i * math.log(lam) - np.array([math.lgamma(v + 1.0) for v in i])
    p_bit = 1.0 - (1.0 - 1.0 / BLOCK_BITS) ** (i * k)
    return float(np.sum(np.exp(logpois) * p_bit ** k))


def fpr_given_state(hist, k: int, c: int = 1) -> float:
    """FPR of a built filter under ideal hashing, from its load histogram.

    A negative key with k independent positions is contained in a block of
    load L with probability (L/512)^k (Section 2.1 applied per block). With
    c = 1 this is exact in expectation over the hash: q = mean_b (L_b/512)^k.
    With c > 1 the candidate blocks are treated as independent, giving
    1 - (1 - q)^c (an estimate; the c blocks share one F(x))."""
    hist = np.asarray(hist, dtype=np.float64)
    L = np.arange(len(hist), dtype=np.float64)
    q = float(np.sum(hist * (L / BLOCK_BITS) ** k) / np.sum(hist))
    return 1.0 - (1.0 - q) ** c
