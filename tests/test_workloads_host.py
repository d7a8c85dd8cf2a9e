"""The seeded input generators against plain definitions, on the host.

Every parity case and every benchmark draws its keys from `workloads`, so the
generators are pinned here to straightforward restatements: splitmix64 with
Python integers, canonical k-mers from strings and their reverse complement,
and the stated recipes of the many-filter and serving workloads.
"""
import math

import numpy as np
import pytest

import workloads

MASK = (1 << 64) - 1


def _splitmix64_py(seed, n, start=0):
    out = []
    for i in range(start, start + n):
        z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & MASK
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    return out


@pytest.mark.parametrize("seed,start", [(0, 0), (1, 0), (2, 1000), (MASK, 7), (3001, 123456)])
def test_splitmix64_matches_python_integers(seed, start):
    assert workloads.splitmix64(seed, 50, start).tolist() == _splitmix64_py(seed, 50, start)
    pos = [5, 0, 999, 3]
    assert workloads.splitmix64_at(seed, pos).tolist() == [_splitmix64_py(seed, 1, p)[0] for p in pos]


def test_genome_bases_come_low_bits_first():
    g = workloads.random_genome(2, 100)
    words = _splitmix64_py(2, 4)
    want = [(words[i // 32] >> (2 * (i % 32))) & 3 for i in range(100)]
    assert g.tolist() == want
    assert g.dtype == np.uint8


def _canonical_from_strings(bases, q):
    s = "".join("ACGT"[b] for b in bases)
    comp = {"A": "T", "C": "G", "G": "C", "T": "A"}
    enc = {"A": 0, "C": 1, "G": 2, "T": 3}

    def code(t):
        v = 0
        for ch in t:
            v = (v << 2) | enc[ch]
        return v

    out = []
    for i in range(len(s) - q + 1):
        w = s[i:i + q]
        rc = "".join(comp[ch] for ch in reversed(w))
        out.append(min(code(w), code(rc)))
    return out


@pytest.mark.parametrize("q", [1, 2, 5, 16, 21, 31, 32])
def test_canonical_kmers_match_strings(q):
    g = workloads.random_genome(7, 300)
    assert workloads.canonical_kmers(g, q).tolist() == _canonical_from_strings(g.tolist(), q)


def test_canonical_kmers_edges():
    assert len(workloads.canonical_kmers(np.array([0, 1, 2], dtype=np.uint8), 31)) == 0
    # a sequence and its reverse complement give the same canonical set
    g = workloads.random_genome(9, 500)
    rc = (3 - g[::-1]).astype(np.uint8)
    assert workloads.canonical_kmers(g, 31).tolist() == workloads.canonical_kmers(rc, 31).tolist()[::-1]
    with pytest.raises(ValueError):
        workloads.canonical_kmers(g, 33)


def test_disjoint_keys_avoid_the_excluded_set_in_stream_order():
    keys = workloads.uniform_keys(1, 5000)
    stream = workloads.splitmix64(1001, 6000)
    exclude = np.concatenate([keys, stream[::3]])     # every third candidate is excluded
    got = workloads.disjoint_keys(1001, 3000, exclude)
    ex = set(exclude.tolist())
    want = [v for v in stream.tolist() if v not in ex][:3000]
    assert got.tolist() == want


def test_many_filter_recipe():
    cfg = workloads.many_filter_config()
    assert len(cfg) == 256
    assert sum(it["n"] for it in cfg) == 84_962_004
    counts = np.array([it["n"] for it in cfg])
    assert counts.min() >= 1000 and counts.max() <= 20_000_000
    assert 100_000 < np.median(counts) < 400_000
    for it in cfg:
        assert it["M"] == -(-16 * it["n"] // 512)
        assert it["B"] == 1 << max(0, math.floor(math.log2(max(it["M"] / 2, 1))))
        assert it["B"] <= max(1, it["M"] // 2) or it["M"] == 1


def test_many_filter_keys_recipe():
    """A filter's queries are its first ceil(n / 2) keys followed by
    floor(n / 2) keys of its query stream, which it does not hold."""
    cfg = sorted(workloads.many_filter_config(), key=lambda it: it["n"])[:8]
    for it in cfg:
        keys, queries = workloads.many_filter_keys(it)
        n, half = it["n"], (it["n"] + 1) // 2
        assert len(keys) == n and len(queries) == n
        assert np.array_equal(keys, workloads.splitmix64(it["key_seed"], n))
        assert np.array_equal(queries[:half], keys[:half])
        assert np.array_equal(queries[half:], workloads.splitmix64(it["query_seed"], n // 2))
        assert not np.isin(queries[half:], keys).any()


def test_serving_recipe():
    filters, reqs = workloads.serving_config(n_requests=4000)
    assert len(filters) == 64
    for f in filters:
        assert 2 ** 20 // 512 <= f["M"] <= 2 ** 31 // 512
        assert f["B"] == 1 << max(0, math.floor(math.log2(max(f["M"] / 2, 1))))
    arrivals = [r["arrival"] for r in reqs]
    assert arrivals[0] == 0.0 and all(b >= a for a, b in zip(arrivals, arrivals[1:]))
    frac = sum(r["kind"] == 1 for r in reqs) / len(reqs)
    assert abs(frac - 0.7) < 0.03
    assert all(1 <= r["n"] <= 1_000_000 for r in reqs)
    # inserts of a filter take consecutive stretches of its key stream
    nxt = [0] * 64
    for r in reqs:
        if r["kind"] == 0:
            assert r["key_start"] == nxt[r["filter"]]
            nxt[r["filter"]] += r["n"]
    # a query's members are keys inserted into its filter before it arrived
    for r in reqs[:400]:
        if r["kind"] == 1 and r["members_from"] and r["n"] >= 2:
            keys = workloads.serving_keys(filters, r)
            f = filters[r["filter"]]
            inserted = set(workloads.splitmix64(f["key_seed"], r["members_from"]).tolist())
            assert set(keys[: r["n"] // 2].tolist()) <= inserted
