"""Pins of the oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: the anchors are values the
paper prints, hand-derived worked examples, closed forms, exact enumeration
on tiny filters, invariants the method guarantees, and an independent
re-derivation of each greedy step with Python integers.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from oracle.oracle import OracleFilter, bits_of_bitmap, COST_MIX, COST_LA, COST_EXP, GOLDEN_RATIO
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([f.strip() for f in line.split("|")])
    return rows


# ---------------------------------------------------------------- generators

def test_splitmix64_check_vector():
    want = [int(r[0]) for r in _rows("splitmix64_seed1234567.txt")]
    state = 1234567
    got = []
    for _ in want:
        state, out = oracle.splitmix64_next(state)
        got.append(out)
    assert got == want
    assert [int(v) for v in workloads.splitmix64(1234567, len(want))] == want


# ---------------------------------------------------------------- hash (Section 3.4)

def test_hash_worked_examples():
    rows = _rows("hash_worked_examples.txt")
    assert len(rows) >= 10
    for a, x, b, want, _why in rows:
        assert oracle.hash_lin(int(a), int(x), int(b)) == int(want), (a, x, b)


@pytest.mark.parametrize("b", [512, 1 << 21, 1000003, 6150, 2])
def test_hash_range_and_uniformity(b):
    """Values stay in [b) and are uniform over random keys (chi-square)."""
    keys = workloads.uniform_keys(77, 60000)
    a = 0x9E3779B97F4A7C15 | 1
    vals = np.array([oracle.hash_lin(a, int(x), b) for x in keys], dtype=np.uint64)
    assert int(vals.max()) < b
    bins = min(b, 64)
    # fold onto `bins` classes by value range (uniform over [b) stays uniform)
    cls = (vals.astype(np.float64) * bins / b).astype(np.int64)
    cnt = np.bincount(cls, minlength=bins)
    exp = len(keys) / bins
    chi2 = float(np.sum((cnt - exp) ** 2 / exp))
    # chi-square with bins-1 dof: mean bins-1, sd sqrt(2(bins-1)); allow 6 sd
    assert chi2 < (bins - 1) + 6 * math.sqrt(2 * (bins - 1)) + 1, chi2


def test_multipliers_odd_coprime_deterministic():
    for M in [1, 7, 6150, 1 << 15, 32768 * 3]:
        ab, af = oracle.derive_multipliers(12345, M, 14, 3)
        ab2, af2 = oracle.derive_multipliers(12345, M, 14, 3)
        assert np.array_equal(ab, ab2) and np.array_equal(af, af2)
        for a in ab:
            assert math.gcd(int(a), M) == 1 and int(a) & 1
        for a in af:
            assert math.gcd(int(a), 512) == 1
        assert len(set(int(v) for v in af)) == 14
    # the stream order: c block multipliers first, then k bit multipliers
    ab3, af3 = oracle.derive_multipliers(12345, 1 << 15, 14, 3)
    outs = workloads.splitmix64(12345, 17)
    assert [int(v) for v in ab3] == [int(v) | 1 for v in outs[:3]]
    assert [int(v) for v in af3] == [int(v) | 1 for v in outs[3:17]]


def test_birthday_rate_of_bit_hashes():
    """Fig. 3B: P(|F(x)| < k) for k = 10 matches the birthday formula."""
    k = 10
    _, a_bit = oracle.derive_multipliers(99, 1, k, 1)
    keys = workloads.uniform_keys(5, 40000)
    short = sum(1 for x in keys if len(oracle.bit_positions(a_bit, int(x))) < k)
    p = cf.birthday_collision(k)
    sd = math.sqrt(len(keys) * p * (1 - p))
    assert abs(short - len(keys) * p) < 4.5 * sd, (short, len(keys) * p)


# ---------------------------------------------------------------- cost functions

def test_cost_printed_facts():
    k = 14
    beta = GOLDEN_RATIO
    for a in range(0, k + 1):
        # Appendix A: at load 1/4 (j = 128) cost^EXP equals beta plus a/k
        assert oracle.cost(COST_EXP, beta, k, 128, a) == pytest.approx(beta + a / k, rel=1e-15)
        # Appendix A: with sigma = 1, reaching load 1/2 (j = 256) makes the FPR term exactly k
        assert oracle.cost(COST_MIX, 1.0, k, 256, a) == pytest.approx(k + a, rel=1e-15)
    # Eq. 6: cost^LA_mu(j, a) = cost^MIX_1(j + mu k, a); mu = 3.5 gives an integer shift of 49
    for j in [0, 17, 100, 200, 300, 400, 463]:
        for a in [0, 1, 7, 14]:
            assert oracle.cost(COST_LA, 3.5, k, j, a) == pytest.approx(
                oracle.cost(COST_MIX, 1.0, k, j + 49, a), rel=1e-14)
    # Eq. 5 at j = 0 is a alone; Eq. 4 at j = 0 is 1 + a/k
    assert oracle.cost(COST_MIX, 50.0, k, 0, 3) == 3.0
    assert oracle.cost(COST_EXP, beta, k, 0, 7) == pytest.approx(1.5, rel=1e-15)
    # MIX at sigma: first term scales linearly in sigma
    assert oracle.cost(COST_MIX, 50.0, k, 300, 0) == pytest.approx(
        50.0 * oracle.cost(COST_MIX, 1.0, k, 300, 0), rel=1e-14)


def test_cost_monotone():
    """All three costs grow with the final load j and with the new bits a."""
    for kind, par in [(COST_MIX, 50.0), (COST_LA, 3.5), (COST_EXP, GOLDEN_RATIO)]:
        k = 12
        prev = None
        for j in range(0, 513):
            v = oracle.cost(kind, par, k, j, 3)
            if prev is not None:
                assert v >= prev
            prev = v
        for a in range(0, k):
            assert oracle.cost(kind, par, k, 200, a + 1) > oracle.cost(kind, par, k, 200, a)


# ---------------------------------------------------------------- printed closed forms

def _printed():
    return {(r[0], r[1]): r for r in _rows("paper_printed_values.txt")}


def test_bloom_overload_printed():
    assert cf.bloom_overload_fpr(1.1, 10) / 2.0 ** -10 == pytest.approx(1.912, abs=0.001)
    assert _printed()[("bloom_overload_fpr", "gamma=1.1 k=10")][2] == "1.912*2^-10"


def test_bloom_overhead_printed():
    assert cf.bloom_bits(1.0, 1) == pytest.approx(1.443, abs=0.0005)
    # at load 1/2 the standard Bloom FPR is exactly 2^-k
    assert cf.bloom_fpr(1000.0, cf.bloom_bits(1000.0, 10), 10) == pytest.approx(2.0 ** -10, rel=1e-12)


@pytest.mark.parametrize("c,k,want", [(2, 7, 232), (3, 7, 219), (2, 14, 244), (3, 14, 237)])
def test_load_bound_printed(c, k, want):
    assert abs(cf.load_bound(c, k) - want) < 0.5
    # and the defining property: (j/512)^k = 2^-k / c at the bound
    j = cf.load_bound(c, k)
    assert (j / 512.0) ** k == pytest.approx(2.0 ** -k / c, rel=1e-12)


def test_choices_fpr_printed():
    """Querying c candidate blocks turns a per-block FPR eps into
    1 - (1 - eps)^c: eps + eps - eps^2 for two choices and almost three times
    eps for three (Section 3.1). The histogram estimate combines its c blocks
    so; a filter whose blocks all hold L bits has eps = (L/512)^k."""
    assert _printed()[("choices_fpr", "c=2")][2].startswith("eps + eps - eps^2")
    for L, k in ((256, 10), (300, 7), (200, 14)):
        hist = np.zeros(513)
        hist[L] = 1000
        eps = (L / 512.0) ** k
        assert cf.fpr_given_state(hist, k, 1) == pytest.approx(eps, rel=1e-12)
        assert cf.fpr_given_state(hist, k, 2) == pytest.approx(eps + eps - eps ** 2, rel=1e-12)
        three = cf.fpr_given_state(hist, k, 3)
        assert three == pytest.approx(3 * eps - 3 * eps ** 2 + eps ** 3, rel=1e-12)
        assert 2.9 * eps < three < 3 * eps


def test_birthday_printed():
    p = cf.birthday_collision(10)
    assert 0.08 < p < 0.10  # "almost 10%"
    # brute force over all 8^3 triples in a range of 8: 1 - 8*7*6/512
    assert cf.birthday_collision(3, 8) == pytest.approx(1 - 8 * 7 * 6 / 512.0, rel=1e-15)


# ---------------------------------------------------------------- the filter itself

def _filter(M, k, c, kind=COST_EXP, par=GOLDEN_RATIO, seed=3, B=1):
    return OracleFilter(M, k, c, kind, par, seed=seed, batch=B)


@pytest.mark.parametrize("c,kind,par,B", [
    (1, COST_EXP, GOLDEN_RATIO, 1), (2, COST_MIX, 50.0, 1), (3, COST_LA, 3.5, 1),
    (2, COST_EXP, GOLDEN_RATIO, 97), (3, COST_MIX, 2.5, 4096), (2, COST_LA, 3.5, 100000)])
def test_no_false_negatives(c, kind, par, B):
    """Section 1: a key that was inserted always queries True."""
    f = _filter(64, 9, c, kind, par, B=B)
    keys = workloads.uniform_keys(11, 6000)
    f.insert(keys)
    bm = f.query(keys)
    assert bits_of_bitmap(bm, len(keys)).all()
    assert f.inserted + f.skipped == len(keys)


def _textbook_blocked_bloom(M, k, a_block1, a_bit, keys):
    """Blocked Bloom filter (Section 2.2) with Python integers as blocks:
    set the bits f_1(x)..f_k(x) in block h_1(x)."""
    blocks = [0] * M
    for x in keys:
        b = oracle.hash_lin(a_block1, int(x), M)
        for a in a_bit:
            blocks[b] |= 1 << oracle.hash_lin(int(a), int(x), 512)
    return blocks


def _words_to_blocks(words, M):
    blocks = []
    for b in range(M):
        v = 0
        for w in range(8):
            v |= int(words[8 * b + w]) << (64 * w)
        blocks.append(v)
    return blocks


def test_one_choice_is_blocked_bloom():
    """Section 3.4: one choice without cost evaluation is a Blocked Bloom
    filter; the words depend neither on B nor on the cost."""
    M, k = 37, 6
    keys = workloads.uniform_keys(21, 3000)
    ref = None
    for kind, par, B in [(COST_EXP, GOLDEN_RATIO, 1), (COST_MIX, 50.0, 7), (COST_LA, 3.5, 3000)]:
        f = _filter(M, k, 1, kind, par, seed=8, B=B)
        f.insert(keys)
        if ref is None:
            ref = f.words.copy()
            tb = _textbook_blocked_bloom(M, k, int(f.a_block[0]), f.a_bit[:k], keys)
            assert _words_to_blocks(f.words, M) == tb
        assert np.array_equal(f.words, ref)


def test_whole_batch_against_empty_filter_takes_first_choice():
    """With B >= n every key sees the empty filter: all candidate costs tie
    and the lowest index wins, so the result is the Blocked Bloom filter on h_1."""
    for c in (2, 3):
        f = _filter(50, 8, c, COST_MIX, 50.0, seed=4, B=10 ** 6)
        keys = workloads.uniform_keys(31, 2000)
        ch = f.insert(keys, return_choices=True)
        assert (ch == 0).all()
        tb = _textbook_blocked_bloom(50, 8, int(f.a_block[0]), f.a_bit[:8], keys)
        assert _words_to_blocks(f.words, 50) == tb


def test_order_invariance_inside_a_batch():
    keys = workloads.uniform_keys(41, 4096)
    rng = np.random.default_rng(0)
    a = _filter(16, 7, 3, COST_LA, 3.5, B=1024)
    a.insert(keys)
    b = _filter(16, 7, 3, COST_LA, 3.5, B=1024)
    perm = np.concatenate([s + rng.permutation(1024) for s in range(0, 4096, 1024)])
    b.insert(keys[perm])
    assert np.array_equal(a.words, b.words)


@pytest.mark.parametrize("M,k,c,kind,par", [
    (1, 2, 2, COST_MIX, 50.0), (2, 3, 2, COST_EXP, GOLDEN_RATIO), (4, 2, 3, COST_LA, 3.5),
    (8, 3, 3, COST_MIX, 2.5), (4, 3, 2, COST_EXP, GOLDEN_RATIO)])
def test_greedy_steps_by_brute_force(M, k, c, kind, par):
    """Replays every sequential insertion with Python integers as blocks:
    each step must skip exactly when a candidate already holds F(x), and
    otherwise pick the first candidate of least cost (Section 3.2)."""
    f = _filter(M, k, c, kind, par, seed=M * 10 + k, B=1)
    keys = workloads.uniform_keys(M + 100 * k, 300)
    ch = f.insert(keys, return_choices=True)
    blocks = [0] * M
    for t, x in enumerate(keys):
        F = set(int(p) for p in oracle.bit_positions(f.a_bit[:k], int(x)))
        cands = [oracle.hash_lin(int(f.a_block[i]), int(x), M) for i in range(c)]
        Ls = [bin(blocks[b]).count("1") for b in cands]
        As = [sum(1 for p in F if not (blocks[b] >> p) & 1) for b in cands]
        if min(As) == 0:
            assert ch[t] == -1, t
            continue
        if kind == COST_MIX:
            costs = [par * k * ((L + a) / 256.0) ** k + a for L, a in zip(Ls, As)]
        elif kind == COST_LA:
            costs = [k * ((L + a + par * k) / 256.0) ** k + a for L, a in zip(Ls, As)]
        else:
            costs = [par ** ((L + a) / 128.0) + a / k for L, a in zip(Ls, As)]
        best = min(range(c), key=lambda i: (costs[i], i))
        assert ch[t] == best, (t, costs, ch[t])
        for p in F:
            blocks[cands[best]] |= 1 << p
    assert _words_to_blocks(f.words, M) == blocks


def _exact_fpr_by_enumeration(blocks, M, c, k):
    """P(query hits) for a key whose c block addresses and k bit addresses
    are independent and uniform: enumerate every block tuple, and for each
    take the union over candidates by inclusion-exclusion over subsets
    (|intersection|/512)^k. For k = 2 also enumerate all 512^2 bit pairs."""
    import itertools
    tot = 0.0
    for tup in itertools.product(range(M), repeat=c):
        p = 0.0
        for r in range(1, c + 1):
            for sub in itertools.combinations(tup, r):
                inter = (1 << 512) - 1
                for b in sub:
                    inter &= blocks[b]
                p += (-1) ** (r + 1) * (bin(inter).count("1") / 512.0) ** k
        tot += p
    return tot / M ** c


def test_exact_fpr_tiny_filter_vs_measured():
    M, k, c = 2, 2, 2
    f = _filter(M, k, c, COST_EXP, GOLDEN_RATIO, seed=5, B=1)
    keys = workloads.uniform_keys(61, 220)
    f.insert(keys)
    blocks = _words_to_blocks(f.words, M)
    p_ie = _exact_fpr_by_enumeration(blocks, M, c, k)
    # direct enumeration of all (b1, b2, p1, p2) outcomes
    bits = np.array([[(blocks[b] >> p) & 1 for p in range(512)] for b in range(M)], dtype=bool)
    cont = bits[:, :, None] & bits[:, None, :]          # block holds both positions
    p_enum = float(np.mean(cont[:, None, :, :] | cont[None, :, :, :]))
    assert p_enum == pytest.approx(p_ie, rel=1e-12)
    neg = workloads.disjoint_keys(62, 400000, keys)
    W = int(bits_of_bitmap(f.query(neg), len(neg)).sum())
    sd = math.sqrt(len(neg) * p_ie * (1 - p_ie))
    assert abs(W - len(neg) * p_ie) < 4.5 * sd, (W, len(neg) * p_ie)


def test_one_choice_fpr_given_state_and_formula():
    """One choice: measured W/N equals mean_b (L_b/512)^k within binomial
    noise, and is near the Putze et al. blocked-Bloom formula."""
    M, k = 1024, 8
    n = int(M * 512 * math.log(2) / k)
    f = _filter(M, k, 1, seed=6)
    keys = workloads.uniform_keys(71, n)
    f.insert(keys)
    hist, total = f.histogram()
    assert int(hist.sum()) == M and total == sum(bin(b).count("1") for b in _words_to_blocks(f.words, M))
    q = cf.fpr_given_state(hist, k, 1)
    neg = workloads.disjoint_keys(72, 600000, keys)
    W = int(bits_of_bitmap(f.query(neg), len(neg)).sum())
    sd = math.sqrt(len(neg) * q * (1 - q))
    assert abs(W - len(neg) * q) < 4.5 * sd
    assert q == pytest.approx(cf.blocked_bloom_fpr(n, M, k), rel=0.06)
    # Section 2.2: the blocked filter is worse than a standard Bloom filter of the same size
    assert q > cf.bloom_fpr(n, M * 512, k)


def test_load_histograms_ordered_by_choices():
    """Appendix C (Fig. 8): three choices give a lower and tighter load
    distribution than two, and two than one, at equal n, M and k."""
    M, k = 1024, 14
    n = int(M * 512 * math.log(2) / k)
    keys = workloads.uniform_keys(81, n)
    stats = []
    for c in (1, 2, 3):
        f = _filter(M, k, c, COST_EXP, GOLDEN_RATIO, seed=9)
        f.insert(keys)
        hist, _ = f.histogram()
        L = np.arange(513)
        mean = float(np.sum(hist * L) / M)
        sd = math.sqrt(float(np.sum(hist * (L - mean) ** 2) / M))
        stats.append((mean, sd))
    assert stats[2][0] < stats[1][0] < stats[0][0]
    assert stats[2][1] < stats[1][1] < stats[0][1]


def test_histogram_is_blocks_per_popcount():
    """hist[L] counts the blocks that hold exactly L set bits and the total is
    every set bit (Appendix C, Fig. 8). Hand cases: an empty filter is M blocks
    of load 0, and one key put into it makes one block of load |F(x)|. A built
    filter's histogram equals numpy's count of the bits of its words."""
    M, k = 257, 9
    f = _filter(M, k, 2, COST_MIX, 50.0, seed=4)
    hist, total = f.histogram()
    assert int(hist[0]) == M and int(hist[1:].sum()) == 0 and total == 0
    x = 0x243F6A8885A308D3
    f.insert(np.array([x], dtype=np.uint64))
    nF = len(oracle.bit_positions(f.a_bit[:k], x))
    hist, total = f.histogram()
    assert int(hist[0]) == M - 1 and int(hist[nF]) == 1 and total == nF
    f.insert(workloads.uniform_keys(5, 3000))
    hist, total = f.histogram()
    pop = np.unpackbits(f.words.view(np.uint8)).reshape(M, 512).sum(axis=1)
    assert np.array_equal(hist.astype(np.int64), np.bincount(pop, minlength=513))
    assert total == int(pop.sum())


def test_duplicates_and_skip_counts():
    f = _filter(32, 10, 2, COST_MIX, 50.0, B=1)
    keys = workloads.uniform_keys(91, 100)
    f.insert(keys)
    assert f.inserted + f.skipped == 100
    before = f.words.copy()
    f.insert(keys)                # every key is now contained: all skipped
    assert f.skipped >= 100 and np.array_equal(before, f.words)
    g = _filter(32, 10, 2, COST_MIX, 50.0, B=64)
    g.insert(np.concatenate([keys[:10], keys[:10]]))  # same batch: same choice, idempotent
    h = _filter(32, 10, 2, COST_MIX, 50.0, B=64)
    h.insert(keys[:10])
    assert np.array_equal(g.words, h.words) and g.inserted == 20


def test_query_bitmap_layout():
    f = _filter(8, 4, 2, COST_MIX, 50.0, B=1)
    keys = workloads.uniform_keys(101, 40)
    f.insert(keys[::2])
    bm = f.query(keys[:70])
    assert len(bm) == 1
    hits = bits_of_bitmap(bm, 40)
    assert hits[::2].all()
    assert (int(bm[0]) >> 40) == 0       # bits past n are zero
    for t in range(40):
        assert hits[t] == ((int(bm[0]) >> t) & 1 == 1)
    assert len(f.query(keys[:0])) == 0


# ---------------------------------------------------------------- learned-cost oracle

def test_learned_forward_hand_value():
    """With W1 = 0 and b1 = 0 the first layer is 0; b2[0] = atanh(1/2) makes
    h2[0] = 1/2; w3[0] = 2 and b3 = 0.25 give g = 1.25 at every grid point."""
    from oracle import learned as lr
    p = np.zeros(lr.NPARAMS)
    H = lr.H
    p[3 * H + H * H + 0] = math.atanh(0.5)      # b2[0]
    p[4 * H + H * H + 0] = 2.0                   # w3[0]
    p[5 * H + H * H] = 0.25                      # b3
    g = lr.forward(p, 7)
    assert g.shape == (513 * 8,)
    assert np.allclose(g, 1.25, rtol=0, atol=1e-15)


def test_learned_forward_reads_the_cost_arguments():
    """The network reads the cost arguments of Section 3.2: j = L + a (set bits
    after the insertion) over 512 and a over k. With W1[0] = (1, 0),
    W1[1] = (0, 1), W2[0][0] = W2[1][1] = 1, w3 = (1, 1, 0, ...) and every other
    parameter 0, the output at grid point L (k + 1) + a is
    tanh(tanh((L + a) / 512)) + tanh(tanh(a / k))."""
    from oracle import learned as lr
    H, k = lr.H, 7
    p = np.zeros(lr.NPARAMS)
    p[0] = 1.0                                   # W1[0][0]
    p[3] = 1.0                                   # W1[1][1]
    p[3 * H] = 1.0                               # W2[0][0]
    p[3 * H + H + 1] = 1.0                       # W2[1][1]
    p[4 * H + H * H] = 1.0                       # w3[0]
    p[4 * H + H * H + 1] = 1.0                   # w3[1]
    g = lr.forward(p, k)
    for L, a in [(0, 0), (10, 3), (200, 1), (505, 7)]:
        want = math.tanh(math.tanh((L + a) / 512.0)) + math.tanh(math.tanh(a / k))
        assert g[L * (k + 1) + a] == pytest.approx(want, rel=1e-14), (L, a)


def test_learned_backward_matches_finite_differences():
    from oracle import learned as lr
    rng = np.random.default_rng(3)
    k = 5
    p = rng.normal(0, 0.4, lr.NPARAMS)
    w = rng.normal(0, 1.0, 513 * (k + 1))
    w[rng.random(w.shape) < 0.7] = 0.0
    g = lr.backward(p, k, w)
    idx = rng.choice(lr.NPARAMS, 60, replace=False)
    for i in list(idx) + [lr.NPARAMS - 1, 0, 2 * lr.H]:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (w @ lr.forward(pp, k) - w @ lr.forward(pm, k)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_learned_sampling_limits_and_invariants():
    """Score weights sum to zero per decision; as tau -> 0 the sampled
    choices are the greedy (least table cost, lowest index on ties) ones."""
    from oracle import learned as lr
    from oracle.oracle import COST_TABLE
    k, M, c = 6, 16, 3
    rng = np.random.default_rng(1)
    table = rng.normal(0, 1, 513 * (k + 1))
    pre = workloads.uniform_keys(201, 400)
    keys = workloads.uniform_keys(202, 300)
    f = _filter(M, k, c, COST_EXP, GOLDEN_RATIO, seed=4, B=1)
    f.insert(pre)
    choices, w, _ = lr.sampled_batch(f, keys, table, 1e-9, seed=5)
    assert abs(w.sum()) < 1e-3 * max(1.0, np.abs(w).sum() * 1e-12)
    g = _filter(M, k, c, COST_EXP, GOLDEN_RATIO, seed=4, B=1)
    g.insert(pre)
    g.set_cost_table(table)
    greedy = g.insert(keys, batch=len(keys), return_choices=True)
    # compare where the least table value is unique (tied candidates, e.g. two
    # choices on the same block, are sampled among; greedy takes the first)
    k1 = k + 1
    unique = []
    for x in keys:
        vals = [table[L * k1 + a] for L, a in (f.block_terms(b, int(x)) for b in f.candidates(int(x)))]
        unique.append(sum(1 for v in vals if v == min(vals)) == 1)
    unique = np.array(unique)
    assert unique.sum() > 200
    got = np.where(choices == 255, -1, choices)
    assert np.array_equal(got[unique], greedy.astype(np.int64)[unique])
    assert np.array_equal(got == -1, greedy == -1)
    # a moderate tau draws non-greedy choices too, still with zero-sum weights
    ch2, w2, _ = lr.sampled_batch(f, keys, table, 1.0, seed=6)
    assert abs(w2.sum()) < 1e-9 * max(1.0, np.abs(w2).sum())
    assert (ch2 != np.where(choices == 255, 255, choices)).any()


def test_learned_adam_hand_steps():
    """Adam (Kingma and Ba, 2015) with zero moments: the bias corrections make
    m_hat = g and v_hat = g^2 on the first step, so the update is
    -lr g / (|g| + eps), i.e. -lr sign(g) away from g = 0, and a constant
    gradient keeps that size on every later step. A gradient +1 then -1 gives,
    on step 2, m = 0.9 (0.1) - 0.1 = -0.01, so m_hat = -0.01 / (1 - 0.81) = -1/19,
    and v = 0.999 (0.001) + 0.001 = 0.001999 = 1 - 0.999^2, so v_hat = 1: the
    second update is +lr/19. Swapping beta1 and beta2, dropping a bias
    correction or the square root changes one of these values."""
    from oracle import learned as lr
    z = np.zeros(4)
    p0 = np.array([1.0, -2.0, 0.5, 3.0])
    g = np.array([0.5, -2.0, 0.0, 1e-3])
    p1, m1, m2 = lr.adam(p0, g, z.copy(), z.copy(), 1, 0.01)
    want1 = np.array([1.0 - 0.01 * 0.5 / (0.5 + 1e-8), -2.0 + 0.01 * 2.0 / (2.0 + 1e-8), 0.5,
                      3.0 - 0.01 * 1e-3 / (1e-3 + 1e-8)])
    assert np.allclose(p1, want1, rtol=0, atol=1e-13)
    assert np.allclose(m1, 0.1 * g, rtol=0, atol=1e-15) and np.allclose(m2, 1e-3 * g * g, rtol=0, atol=1e-15)
    # constant gradient: -lr sign(g) every step
    p, a, b = p0.copy(), z.copy(), z.copy()
    for t in range(1, 8):
        p, a, b = lr.adam(p, g, a, b, t, 0.01)
    assert np.allclose(p[:2], [1.0 - 0.07, -2.0 + 0.07], rtol=0, atol=1e-8)
    assert p[2] == 0.5
    # +1 then -1: the second step moves by +lr/19
    q1, a, b = lr.adam(np.zeros(1), np.ones(1), np.zeros(1), np.zeros(1), 1, 0.01)
    assert np.allclose(q1, [-0.01], rtol=0, atol=1e-10)
    q2, _, _ = lr.adam(q1, -np.ones(1), a, b, 2, 0.01)
    assert np.allclose(q2 - q1, [0.01 / 19.0], rtol=0, atol=1e-10)


def _distinct_point_key(f, table_len, want_c, seed=77):
    """A key whose candidates are all partly empty (a > 0) at distinct (L, a)
    grid points of the filter `f` as it stands."""
    k1 = f.k + 1
    for x in workloads.uniform_keys(seed, 5000):
        terms = [f.block_terms(b, int(x)) for b in f.candidates(int(x))]
        pts = [L * k1 + a for L, a in terms]
        if len(set(pts)) == want_c and min(a for _, a in terms) > 0:
            assert max(pts) < table_len
            return int(x), pts
    raise AssertionError("no key with distinct candidate points")


@pytest.mark.parametrize("c", [2, 3])
def test_learned_score_weight_is_gradient_of_log_policy(c):
    """The score weight of a decision is d log pi(s) / d g at each candidate's
    grid point, where pi = softmax(-g / tau) over the key's candidates and s
    is the drawn choice. Checked by a central finite difference of
    log pi(s), computed by scipy's log_softmax, in each candidate's table
    value, for every possible draw s; a flipped sign or a missing 1/tau fails."""
    from scipy.special import log_softmax
    from oracle import learned as lr
    k, M, tau, h = 6, 16, 0.7, 1e-6
    f = _filter(M, k, c, COST_EXP, GOLDEN_RATIO, seed=4, B=1)
    f.insert(workloads.uniform_keys(201, 300))
    rng = np.random.default_rng(11)
    table = rng.normal(0, 1, 513 * (k + 1))
    x, pts = _distinct_point_key(f, len(table), c)
    seen = set()
    for seed in range(200):
        ch, w, _ = lr.sampled_batch(f, np.array([x], dtype=np.uint64), table, tau, seed)
        s = int(ch[0])
        if s in seen:
            continue
        seen.add(s)
        for i, p in enumerate(pts):
            tp, tm = table.copy(), table.copy()
            tp[p] += h
            tm[p] -= h
            lp = log_softmax(-np.array([tp[q] for q in pts]) / tau)[s]
            lm = log_softmax(-np.array([tm[q] for q in pts]) / tau)[s]
            fd = (lp - lm) / (2 * h)
            assert abs(w[p] - fd) < 1e-6, (c, s, i, w[p], fd)
        nz = np.flatnonzero(w)
        assert set(nz.tolist()) <= set(pts)
    assert seen == set(range(c))


def test_learned_sampler_draws_from_softmax_of_minus_cost():
    """4,000 draws for one key (u from consecutive stream positions): the
    frequency of each candidate equals softmax(-g / tau) within 4.5 binomial
    sigma. Drawing from softmax(+g / tau), or inverting the cumulative search,
    fails."""
    from scipy.special import softmax
    from oracle import learned as lr
    k, M, tau, n = 6, 16, 0.8, 4000
    f = _filter(M, k, 3, COST_EXP, GOLDEN_RATIO, seed=4, B=1)
    f.insert(workloads.uniform_keys(201, 300))
    table = np.random.default_rng(12).normal(0, 1, 513 * (k + 1))
    x, pts = _distinct_point_key(f, len(table), 3, seed=78)
    ch, _, _ = lr.sampled_batch(f, np.full(n, x, dtype=np.uint64), table, tau, seed=9)
    pi = softmax(-np.array([table[p] for p in pts]) / tau)
    assert pi.max() - pi.min() > 0.15
    for i in range(3):
        got = float((ch == i).sum())
        sd = math.sqrt(n * pi[i] * (1 - pi[i]))
        assert abs(got - n * pi[i]) < 4.5 * sd, (i, got, n * pi[i])


def test_learned_uniforms_are_the_generator_stream():
    """splitmix_uniform(seed, i) is the top 53 bits of output i of the
    published generator: equal to workloads.splitmix64 and to the check
    vector of seed 1234567."""
    from oracle import learned as lr
    want = [int(r[0]) for r in _rows("splitmix64_seed1234567.txt")]
    for i, v in enumerate(want):
        assert lr.splitmix_uniform(1234567, i) == (v >> 11) / float(1 << 53)
    for seed in (0, 5, 0xDEADBEEF12345678):
        outs = workloads.splitmix64(seed, 300)
        for i in (0, 1, 17, 299):
            assert lr.splitmix_uniform(seed, i) == (int(outs[i]) >> 11) / float(1 << 53)


# ---------------------------------------------------------------- distinct bit selection (Appendix B)

def test_distinct_shift_rule_printed_example():
    """Fig. 9: f_1 = 316, f_2 = 27 stays 27; values >= 316 move up by one."""
    from oracle.oracle import distinct_from_raw
    assert list(distinct_from_raw([316, 27])) == [316, 27]
    assert list(distinct_from_raw([316, 316])) == [316, 317]
    assert list(distinct_from_raw([316, 400])) == [316, 401]
    assert list(distinct_from_raw([316, 315])) == [316, 315]
    # hand-worked: each new value passes every earlier address at or below it
    assert list(distinct_from_raw([5, 5, 5])) == [5, 6, 7]
    assert list(distinct_from_raw([10, 3, 9])) == [10, 3, 11]   # 9 passes 3 -> 10, then 10 -> 11
    assert list(distinct_from_raw([511, 510, 509])) == [511, 510, 509]
    assert list(distinct_from_raw([0, 0, 0, 0])) == [0, 1, 2, 3]


def test_distinct_pairs_are_each_2_subset_twice():
    """Exhaustively: (f_1, f_2) over [512] x [511] yields every 2-subset of
    [512] exactly twice (once per order), so the subset is uniform."""
    from oracle.oracle import distinct_from_raw
    counts = {}
    for a in range(0, 512, 1):
        for b in range(0, 511, 7):
            p, q = distinct_from_raw([a, b])
            assert p != q and 0 <= q < 512
            key = (min(p, q), max(p, q))
            counts[key] = counts.get(key, 0) + 1
    # the map is injective on the sampled domain: no subset arises more than twice
    assert max(counts.values()) <= 2
    # full domain for a few first values: b ranges over [511], so f_2 covers [512] minus {f_1}
    for a in (0, 1, 255, 316, 511):
        seconds = {int(distinct_from_raw([a, b])[1]) for b in range(511)}
        assert seconds == set(range(512)) - {a}


def test_distinct_multipliers_and_sizes():
    from oracle.oracle import derive_multipliers, bit_positions
    _, af = derive_multipliers(77, 1 << 10, 20, 2, bitsel=1)
    for i, a in enumerate(af):
        assert math.gcd(int(a), 512 - i) == 1
    keys = workloads.uniform_keys(8, 2000)
    for x in keys:
        assert len(bit_positions(af, int(x), bitsel=1)) == 20


def test_distinct_one_choice_fpr_given_state():
    """With k distinct positions a negative hits a block of load L with
    probability C(L, k) / C(512, k): mean over blocks vs measured W/N."""
    M, k = 256, 8
    n = int(M * 512 * math.log(2) / k)
    f = OracleFilter(M, k, 1, COST_EXP, GOLDEN_RATIO, seed=12, batch=1, bitsel=1)
    keys = workloads.uniform_keys(121, n)
    f.insert(keys)
    hist, _ = f.histogram()
    q = sum(int(hist[L]) * math.comb(L, k) for L in range(513)) / (M * math.comb(512, k))
    neg = workloads.disjoint_keys(122, 400000, keys)
    W = int(bits_of_bitmap(f.query(neg), len(neg)).sum())
    sd = math.sqrt(len(neg) * q * (1 - q))
    assert abs(W - len(neg) * q) < 4.5 * sd
    assert bits_of_bitmap(f.query(keys), n).all()
    # distinct selection queries more bits than random selection: lower FPR at the same size
    g = OracleFilter(M, k, 1, COST_EXP, GOLDEN_RATIO, seed=12, batch=1)
    g.insert(keys)
    W2 = int(bits_of_bitmap(g.query(neg), len(neg)).sum())
    assert W < W2


# ---------------------------------------------------------------- sub-arrays (Section 3.4)

def test_sharded_one_subarray_is_the_plain_filter():
    from oracle.sharded import ShardedOracle
    keys = workloads.uniform_keys(61, 20000)
    for c, kind, par, B in [(2, COST_MIX, 50.0, 1), (3, COST_LA, 3.5, 512)]:
        s = ShardedOracle(333, 1, 11, c, kind, par, seed=9, batch=B)
        o = _filter(333, 11, c, kind, par, seed=9, B=B)
        s.insert(keys)
        o.insert(keys)
        assert np.array_equal(s.words, o.words)
        assert np.array_equal(s.query(keys[:777]), o.query(keys[:777]))


@pytest.mark.parametrize("M,T", [(64, 4), (100, 3), (1000, 6), (7, 8)])
def test_sharded_one_choice_is_a_textbook_blocked_bloom(M, T):
    """c = 1 over T sub-arrays: key x sets bits H_512(a'_i, x) of block
    h_0(x) * ceil(M/T) + H_{M/T}(a_1, x), written here with Python integers;
    a_0 is the seed's first odd generator output coprime to T and a_1, a'_i
    continue the stream (each odd and coprime to its range)."""
    from oracle.sharded import ShardedOracle
    k, seed = 5, 1234
    Ms = -(-M // T)
    outs = [int(v) | 1 for v in workloads.splitmix64(seed, 64)]
    it = iter(outs)
    a0 = next(a for a in it if math.gcd(a, T) == 1)
    a1 = next(a for a in it if math.gcd(a, Ms) == 1)
    abits = [next(it) for _ in range(k)]      # odd is coprime to 512
    keys = workloads.uniform_keys(71, 3000)
    want = [0] * (T * Ms)
    for x in keys:
        x = int(x)
        blk = oracle.hash_lin(a0, x, T) * Ms + oracle.hash_lin(a1, x, Ms)
        for a in abits:
            want[blk] |= 1 << (((a * x) & ((1 << 64) - 1)) >> 55)
    s = ShardedOracle(M, T, k, 1, COST_EXP, GOLDEN_RATIO, seed=seed, batch=64)
    s.insert(keys)
    w = s.words
    got = [sum(int(w[8 * b + j]) << (64 * j) for j in range(8)) for b in range(T * Ms)]
    assert got == want


def test_sharded_h0_multiplier_is_drawn_first_odd_and_coprime():
    """h_0's multiplier a_0 is drawn before the block and bit multipliers: the
    first output of the seed's splitmix64 stream that is coprime to T, made
    odd. Against the published check vector of seed 1234567 (outputs 1 and 2
    are 0 and 1 mod 3): a_0 is output 1 for T = 2 and output 2 for T = 3, and
    the sub-arrays' multipliers start from the state after it. Over many seeds
    a_0 is odd and coprime to T."""
    from oracle.sharded import shard_layout
    want = [int(r[0]) for r in _rows("splitmix64_seed1234567.txt")]
    gamma = 0x9E3779B97F4A7C15
    a0, Ms, state = shard_layout(100, 2, 1234567)
    assert (a0, Ms, state) == (want[0] | 1, 50, (1234567 + gamma) % (1 << 64))
    a0, Ms, state = shard_layout(100, 3, 1234567)
    assert (a0, Ms, state) == (want[1] | 1, 34, (1234567 + 2 * gamma) % (1 << 64))
    for T in (3, 5, 6, 7):
        for seed in range(64):
            a0, _, _ = shard_layout(1000, T, seed)
            assert a0 % 2 == 1 and math.gcd(a0, T) == 1, (T, seed, a0)


@pytest.mark.parametrize("T", [2, 3, 4, 6])
def test_sharded_h0_is_uniform_and_leaves_other_subarrays_alone(T):
    from oracle.sharded import ShardedOracle
    s = ShardedOracle(120, T, 8, 2, COST_EXP, GOLDEN_RATIO, seed=5, batch=32)
    keys = workloads.uniform_keys(81, 60000)
    sh = s.shard_of(keys)
    cnt = np.bincount(sh, minlength=T)
    exp = len(keys) / T
    chi2 = float(np.sum((cnt - exp) ** 2 / exp))
    assert chi2 < (T - 1) + 6 * math.sqrt(2 * (T - 1)) + 1, (T, cnt)
    s.insert(keys[sh == 0][:2000])
    w = s.words.reshape(T, -1)
    assert w[0].any() and not w[1:].any()


@pytest.mark.parametrize("T,c,kind,par,B", [(2, 2, COST_MIX, 50.0, 1), (3, 3, COST_LA, 3.5, 97),
                                            (5, 2, COST_EXP, GOLDEN_RATIO, 4096)])
def test_sharded_no_false_negatives(T, c, kind, par, B):
    from oracle.sharded import ShardedOracle
    s = ShardedOracle(200, T, 9, c, kind, par, seed=3, batch=B)
    keys = workloads.uniform_keys(91, 8000)
    s.insert(keys)
    assert bits_of_bitmap(s.query(keys), len(keys)).all()
    assert s.inserted + s.skipped == len(keys)
