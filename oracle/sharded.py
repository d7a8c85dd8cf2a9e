"""Oracle of a filter split into T sub-arrays (Section 3.4, parallelization).
TEST INFRASTRUCTURE ONLY: used by tests/, never by the library.

The paper subdivides the bit array into T sub-arrays of M/T blocks (M
rounded up to a multiple of T). An additional hash h_0 : U -> [T],
independent of the block hashes, picks the sub-array of a key; the block
hashes h_1..h_c then address [M/T] inside it, and each sub-array takes its
keys in the order they arrive, one writer per sub-array.

Readings (the paper leaves them open):
  - h_0 is the linear hash of Section 3.4 with range T and its own
    multiplier a_0, drawn first from the hash seed's splitmix64 stream (odd,
    coprime to T); a_1..a_c (range M/T) and a'_1..a'_k continue the same
    stream. With T = 1 no a_0 is drawn and h_0 = 0, so the filter is the
    unsplit one.
  - Batches: each sub-array inserts its own subsequence of the keys in
    batches of B of its keys (its writer's batch rule).
  - Layout: sub-array t is blocks t (M/T) .. (t+1) (M/T) - 1 of the array.
Pinned in tests/test_oracle_pins.py (T = 1, one choice against a textbook
blocked Bloom filter, h_0 uniformity, no false negatives, stream order).
"""
import math

import numpy as np

from .oracle import OracleFilter, derive_multipliers, hash_lin, splitmix64_next


def shard_layout(M: int, T: int, seed: int):
    """(a_0, blocks per sub-array, seed of the sub-arrays' multipliers):
    a_0 is the first odd splitmix64 output of `seed` coprime to T (0 for
    T = 1), and the sub-arrays' multipliers are drawn from the stream state
    that follows it."""
    M, T = int(M), int(T)
    assert M >= 1 and T >= 1
    Ms = -(-M // T)
    if T == 1:
        return 0, Ms, int(seed)
    state = int(seed) & ((1 << 64) - 1)
    while True:
        state, out = splitmix64_next(state)
        a0 = out | 1
        if math.gcd(a0, T) == 1:
            return a0, Ms, state


class ShardedOracle:
    """T sub-arrays of Ms = ceil(M / T) blocks, each an OracleFilter with the
    shared multipliers; h_0(x) = hash_lin(a_0, x, T) routes a key."""

    def __init__(self, M, T, k, c, cost_kind, cost_param, seed=0, batch=1, bitsel=0):
        self.T = int(T)
        self.a0, self.Ms, sub_seed = shard_layout(M, T, seed)
        a_block, a_bit = derive_multipliers(sub_seed, self.Ms, k, c, bitsel)
        self.subs = [OracleFilter(self.Ms, k, c, cost_kind, cost_param, batch=batch,
                                  a_block=a_block, a_bit=a_bit, bitsel=bitsel)
                     for _ in range(self.T)]

    def shard_of(self, keys):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        if self.T == 1:
            return np.zeros(len(keys), dtype=np.int64)
        return np.array([hash_lin(self.a0, int(x), self.T) for x in keys], dtype=np.int64)

    def insert(self, keys):
        """Each sub-array inserts, in order, the keys that h_0 sends to it."""
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        sh = self.shard_of(keys)
        for t in range(self.T):
            self.subs[t].insert(keys[sh == t])

    def query(self, keys):
        """LSB-first bitmap: key i is present in sub-array h_0(x_i)."""
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        sh = self.shard_of(keys)
        hit = np.zeros(len(keys), dtype=bool)
        for t in range(self.T):
            idx = np.flatnonzero(sh == t)
            if len(idx):
                bm = self.subs[t].query(keys[idx])
                b = np.unpackbits(bm.view(np.uint8), bitorder="little")[: len(idx)].astype(bool)
                hit[idx] = b
        out = np.zeros(max((len(keys) + 63) // 64, 1), dtype=np.uint64)
        packed = np.packbits(hit, bitorder="little")
        out.view(np.uint8)[: len(packed)] = packed
        return out[: (len(keys) + 63) // 64]

    @property
    def words(self):
        """The whole array: sub-array t at blocks t Ms .. (t + 1) Ms - 1."""
        return np.concatenate([s.words for s in self.subs])

    @property
    def inserted(self):
        return sum(s.inserted for s in self.subs)

    @property
    def skipped(self):
        return sum(s.skipped for s in self.subs)
