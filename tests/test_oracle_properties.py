"""Invariants of the method on random filter shapes (CPU, hypothesis).

tests/test_oracle_pins.py checks each rule on a few fixed shapes. The rules
below hold for every shape, so here they run on shapes drawn at random: one
block or a few thousand, odd, even and power-of-two block counts, k from 1 to
32, both bit selections, every cost, any batch size and a ragged last batch.

  - An inserted key always queries True, and every key is counted once as
    inserted or skipped (Section 1, Section 3.2).
  - One choice is the textbook Blocked Bloom filter of Section 2.2 (random
    bits), and its words depend neither on the cost nor on B (Section 3.4).
  - A batch against the empty filter takes its first candidate: every cost
    ties there, and ties go to the lowest index.
  - Keys permuted inside their batches give the same words; a call split at
    a batch edge gives the same words as one call (batch semantics).
  - The histogram counts every block once and every set bit once
    (Appendix C).
  - Distinct selection gives k distinct positions in [512] (Appendix B);
    random selection at most k.

The examples are derandomised, so every run checks the same shapes.
"""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
from oracle.oracle import OracleFilter, bits_of_bitmap, COST_MIX, COST_LA, COST_EXP, GOLDEN_RATIO  # noqa: E402
import workloads  # noqa: E402

SETTINGS = settings(max_examples=300, deadline=None, derandomize=True, database=None)
COSTS = st.sampled_from([(COST_MIX, 2.5), (COST_MIX, 50.0), (COST_LA, 3.5), (COST_EXP, GOLDEN_RATIO),
                         (COST_EXP, 1.2)])
BLOCKS = st.one_of(st.integers(1, 8), st.sampled_from([63, 64, 100, 127, 128, 257, 1000, 4096]))
SEEDS = st.integers(0, (1 << 64) - 1)


def _keys(seed, n):
    return workloads.uniform_keys(seed, n)


def _blocks_of(words, M):
    return [sum(int(words[8 * b + w]) << (64 * w) for w in range(8)) for b in range(M)]


@SETTINGS
@given(M=BLOCKS, k=st.integers(1, 32), c=st.integers(1, 3), cost=COSTS, B=st.integers(1, 700),
       n=st.integers(0, 600), bitsel=st.integers(0, 1), seed=SEEDS, kseed=st.integers(0, 1 << 20))
def test_no_false_negatives_and_every_key_counted(M, k, c, cost, B, n, bitsel, seed, kseed):
    f = OracleFilter(M, k, c, cost[0], cost[1], seed=seed, batch=B, bitsel=bitsel)
    keys = _keys(kseed, n)
    f.insert(keys)
    assert f.inserted + f.skipped == n
    assert bits_of_bitmap(f.query(keys), n).all()
    hist, total = f.histogram()
    pop = np.unpackbits(f.words.view(np.uint8)).reshape(M, 512).sum(axis=1)
    assert int(hist.sum()) == M and total == int(pop.sum())
    assert np.array_equal(hist.astype(np.int64), np.bincount(pop, minlength=513))


@SETTINGS
@given(M=BLOCKS, k=st.integers(1, 32), cost=COSTS, B=st.integers(1, 700), n=st.integers(0, 400),
       seed=SEEDS, kseed=st.integers(0, 1 << 20))
def test_one_choice_is_the_textbook_blocked_bloom_filter(M, k, cost, B, n, seed, kseed):
    keys = _keys(kseed, n)
    f = OracleFilter(M, k, 1, cost[0], cost[1], seed=seed, batch=B)
    f.insert(keys)
    blocks = [0] * M
    for x in keys:
        b = oracle.hash_lin(int(f.a_block[0]), int(x), M)
        for a in f.a_bit[:k]:
            blocks[b] |= 1 << oracle.hash_lin(int(a), int(x), 512)
    assert _blocks_of(f.words, M) == blocks
    g = OracleFilter(M, k, 1, COST_EXP, GOLDEN_RATIO, seed=seed, batch=1)
    g.insert(keys)
    assert np.array_equal(g.words, f.words)


@SETTINGS
@given(M=BLOCKS, k=st.integers(1, 32), c=st.integers(2, 3), cost=COSTS, n=st.integers(1, 500),
       bitsel=st.integers(0, 1), seed=SEEDS, kseed=st.integers(0, 1 << 20))
def test_a_batch_against_the_empty_filter_takes_the_first_candidate(M, k, c, cost, n, bitsel, seed, kseed):
    f = OracleFilter(M, k, c, cost[0], cost[1], seed=seed, batch=n, bitsel=bitsel)
    ch = f.insert(_keys(kseed, n), return_choices=True)
    assert (ch == 0).all()


@SETTINGS
@given(M=BLOCKS, k=st.integers(1, 32), c=st.integers(1, 3), cost=COSTS, B=st.integers(1, 200),
       batches=st.integers(1, 5), tail=st.integers(0, 199), bitsel=st.integers(0, 1), seed=SEEDS,
       kseed=st.integers(0, 1 << 20), pseed=st.integers(0, 1 << 20))
def test_batch_semantics(M, k, c, cost, B, batches, tail, bitsel, seed, kseed, pseed):
    n = batches * B + tail % B
    keys = _keys(kseed, n)
    ref = OracleFilter(M, k, c, cost[0], cost[1], seed=seed, batch=B, bitsel=bitsel)
    ref.insert(keys)
    # permuted inside every batch
    rng = np.random.default_rng(pseed)
    perm = np.concatenate([s + rng.permutation(min(B, n - s)) for s in range(0, n, B)])
    p = OracleFilter(M, k, c, cost[0], cost[1], seed=seed, batch=B, bitsel=bitsel)
    p.insert(keys[perm])
    assert np.array_equal(p.words, ref.words)
    assert (p.inserted, p.skipped) == (ref.inserted, ref.skipped)
    # split at a batch edge into two calls
    cut = B * int(rng.integers(0, batches + 1))
    s = OracleFilter(M, k, c, cost[0], cost[1], seed=seed, batch=B, bitsel=bitsel)
    s.insert(keys[:cut])
    s.insert(keys[cut:])
    assert np.array_equal(s.words, ref.words)
    assert (s.inserted, s.skipped) == (ref.inserted, ref.skipped)


@SETTINGS
@given(k=st.integers(1, 32), seed=SEEDS, x=st.integers(0, (1 << 64) - 1))
def test_bit_positions(k, seed, x):
    _, a_bit = oracle.derive_multipliers(seed, 1, k, 1, bitsel=1)
    d = oracle.bit_positions(a_bit, x, bitsel=1)
    assert len(d) == k and len(set(d.tolist())) == k and int(d.max()) < 512
    _, a_bit = oracle.derive_multipliers(seed, 1, k, 1, bitsel=0)
    r = oracle.bit_positions(a_bit, x, bitsel=0)
    assert 1 <= len(r) <= k and int(r.max()) < 512
    assert len(r) == len({oracle.hash_lin(int(a), x, 512) for a in a_bit})
