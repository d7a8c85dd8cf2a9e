"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the filter method: it only makes keys.
Both the oracle-side tests and the GPU path draw their inputs from here, so
that the two sides see identical keys.

* uniform 64-bit keys: successive splitmix64 outputs (Steele, Lea and Flood,
  OOPSLA 2014) of a seed, standing in for the paper's random 64-bit integers
  (Section 4.1, Section 4.2);
* DNA: a uniform random genome over A/C/G/T, 2 bits per base, and its
  canonical 31-mers encoded as 64-bit integers, standing in for the genomes
  of Section 4.3 (which are not available offline).
"""
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+n-1 of splitmix64 seeded with `seed` (uint64)."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64_at(seed: int, positions) -> np.ndarray:
    """splitmix64 outputs of `seed` at the given 0-based stream positions."""
    with np.errstate(over="ignore"):
        idx = np.asarray(positions, dtype=np.uint64) + np.uint64(1)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_keys(seed: int, n: int) -> np.ndarray:
    """n uniform 64-bit keys: the first n splitmix64 outputs of `seed`."""
    return splitmix64(seed, n)


def disjoint_keys(seed: int, n: int, exclude: np.ndarray) -> np.ndarray:
    """n uniform 64-bit keys from `seed` that do not occur in `exclude`,
    in stream order (rejection against a sorted copy of `exclude`)."""
    ex = np.sort(np.asarray(exclude, dtype=np.uint64))
    out = []
    have = 0
    start = 0
    while have < n:
        want = (n - have) + (n - have) // 64 + 16
        cand = splitmix64(seed, want, start)
        start += want
        if len(ex):
            pos = np.searchsorted(ex, cand)
            pos[pos == len(ex)] = 0
            cand = cand[ex[pos] != cand]
        out.append(cand[: n - have])
        have += len(out[-1])
    return np.concatenate(out) if out else np.zeros(0, dtype=np.uint64)


def random_genome(seed: int, nbases: int) -> np.ndarray:
    """Uniform random DNA, one base per uint8 in {0,1,2,3} = A,C,G,T.
    Base 32w+i is bits 2i..2i+1 of splitmix64 output w (low bits first)."""
    nwords = (nbases + 31) // 32
    w = splitmix64(seed, nwords)
    shifts = (2 * np.arange(32, dtype=np.uint64))
    bases = ((w[:, None] >> shifts[None, :]) & np.uint64(3)).astype(np.uint8)
    return bases.reshape(-1)[:nbases]


def _windows(vals: np.ndarray, q: int, first_high: bool) -> np.ndarray:
    """Pack every length-q window of 2-bit symbols into a uint64 by doubling.
    first_high: the window's first symbol is most significant; otherwise the
    first symbol is least significant."""
    n = len(vals) - q + 1
    pieces = {1: vals.astype(np.uint64)}
    L = 1
    while 2 * L <= q:
        a = pieces[L]
        m = len(a) - L
        if first_high:
            pieces[2 * L] = (a[:m] << np.uint64(2 * L)) | a[L:L + m]
        else:
            pieces[2 * L] = a[:m] | (a[L:L + m] << np.uint64(2 * L))
        L *= 2
    acc = None
    acc_len = 0
    for L in sorted(pieces, reverse=True):
        if acc_len + L > q:
            continue
        p = pieces[L]
        if acc is None:
            acc = p[:n].copy()
        else:
            seg = p[acc_len:acc_len + n]
            if first_high:
                acc = (acc << np.uint64(2 * L)) | seg
            else:
                acc = acc | (seg << np.uint64(2 * acc_len))
        acc_len += L
        if acc_len == q:
            break
    return acc


def canonical_kmers(bases: np.ndarray, q: int = 31) -> np.ndarray:
    """Canonical q-mers of a base sequence, 2-bit encoded (A=0, C=1, G=2,
    T=3, first base most significant): min(forward, reverse complement).
    Duplicates are kept, in sequence order."""
    if q < 1 or q > 32:
        raise ValueError("q must be in 1..32")
    bases = np.asarray(bases, dtype=np.uint8)
    if len(bases) < q:
        return np.zeros(0, dtype=np.uint64)
    fwd = _windows(bases, q, first_high=True)
    rc = _windows((3 - bases).astype(np.uint8), q, first_high=False)
    return np.minimum(fwd, rc)


def lognormal_counts(seed: int, n_filters: int, median: float = 200000.0,
                     sigma: float = 1.0, lo: int = 1000, hi: int = 20000000):
    """Per-filter key counts round(median * exp(sigma Z)), clipped to [lo, hi],
    Z standard normal by Box-Muller on splitmix64 uniforms."""
    u = splitmix64(seed, 2 * n_filters)
    u1 = ((u[0::2] >> np.uint64(11)).astype(np.float64) + 0.5) / float(1 << 53)
    u2 = ((u[1::2] >> np.uint64(11)).astype(np.float64) + 0.5) / float(1 << 53)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    n = np.rint(median * np.exp(sigma * z)).astype(np.int64)
    return np.clip(n, lo, hi)


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in (0, 1) from splitmix64 (53-bit mantissa)."""
    u = splitmix64(seed, n)
    return ((u >> np.uint64(11)).astype(np.float64) + 0.5) / float(1 << 53)


def many_filter_config(seed: int = 4, n_filters: int = 256, bits_per_key: int = 16):
    """The many-filter workload: key counts lognormal (median 200,000, sigma 1,
    clipped to 1,000..20,000,000, seed `seed`), M_f = ceil(bits_per_key n_f / 512)
    blocks, batch B_f = 2^floor(log2(M_f / 2)) (at least 1); keys of filter f are
    the splitmix64 stream of seed (seed << 32) | f, its queries are its first
    ceil(n_f / 2) keys followed by floor(n_f / 2) keys of seed ((seed + 1) << 32) | f."""
    counts = lognormal_counts(seed, n_filters)
    out = []
    for f, n in enumerate(counts):
        n = int(n)
        M = -(-bits_per_key * n // 512)
        B = 1 << max(0, int(math.floor(math.log2(max(M / 2.0, 1.0)))))
        out.append(dict(index=f, n=n, M=M, B=B, key_seed=(seed << 32) | f,
                        query_seed=((seed + 1) << 32) | f))
    return out


def many_filter_keys(item):
    """(keys, queries) of one filter of many_filter_config."""
    keys = splitmix64(item["key_seed"], item["n"])
    half = (item["n"] + 1) // 2
    other = splitmix64(item["query_seed"], item["n"] // 2)
    return keys, np.concatenate([keys[:half], other])


def serving_config(seed: int = 5, n_filters: int = 64, n_requests: int = 10000,
                   query_frac: float = 0.7, max_keys: int = 1000000):
    """The serving workload: filters of 2^U bits with U uniform in [20, 31]
    (rounded up to whole 512-bit blocks), batch 2^floor(log2(M / 2)) (at
    least 1); requests with exponential inter-arrival gaps of mean 1 (scaled
    by the caller to an offered rate), kind query with probability query_frac,
    target filter uniform, size log-uniform in [1, max_keys]. Insert request j
    of filter f takes the next keys of the filter's splitmix64 stream (seed
    (seed << 40) | f); a query takes half of its keys from keys inserted
    earlier into its filter (uniform positions) and half from a fresh stream
    (seed (seed << 40) | (1 << 32) | j)."""
    u = uniform01(seed, n_filters)
    filters = []
    for f in range(n_filters):
        U = 20.0 + 11.0 * float(u[f])
        M = int(math.ceil((2.0 ** U) / 512.0))
        B = 1 << max(0, int(math.floor(math.log2(max(M / 2.0, 1.0)))))
        filters.append(dict(index=f, M=M, B=B, key_seed=(seed << 40) | f))
    r = uniform01(seed + 1, 4 * n_requests).reshape(n_requests, 4)
    gaps = -np.log(r[:, 0])
    arrivals = np.cumsum(gaps) - gaps[0]
    requests = []
    inserted = [0] * n_filters
    for j in range(n_requests):
        kind = 1 if r[j, 1] < query_frac else 0
        f = min(n_filters - 1, int(r[j, 2] * n_filters))
        n = max(1, min(max_keys, int(math.floor(math.exp(r[j, 3] * math.log(max_keys + 1.0))))))
        req = dict(index=j, arrival=float(arrivals[j]), kind=kind, filter=f, n=n)
        if kind == 0:
            req["key_start"] = inserted[f]
            inserted[f] += n
        else:
            req["members_from"] = inserted[f]
        requests.append(req)
    return filters, requests


def serving_keys(filters, req, seed: int = 5):
    """Keys of one request of serving_config."""
    f = filters[req["filter"]]
    n = req["n"]
    if req["kind"] == 0:
        return splitmix64(f["key_seed"], n, req["key_start"])
    have = req["members_from"]
    n_mem = n // 2 if have else 0
    fresh = splitmix64((seed << 40) | (1 << 32) | req["index"], n - n_mem)
    if n_mem == 0:
        return fresh
    pos = splitmix64((seed << 40) | (2 << 32) | req["index"], n_mem) % np.uint64(have)
    return np.concatenate([splitmix64_at(f["key_seed"], pos), fresh])
