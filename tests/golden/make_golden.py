"""Writes the stored expected values of the full-size configurations.

Calls only the oracle (oracle/) and the input generators (workloads/); it
never touches the CUDA path. Each output file records the configuration, the
SHA-256 of the oracle's filter words (little-endian bytes) and query bitmap,
the insert/skip counts, the number of positive answers, and the mean index of
the first candidate block holding each inserted key (pbar, used for the
algorithmic bytes of member queries).

Usage: python tests/golden/make_golden.py dna        (about 5 minutes on one core)
       python tests/golden/make_golden.py sweep I    (one filter setting I = 0..6 of the
                                                      overload sweep, about 60 minutes)
       python tests/golden/make_golden.py many       (the 256-filter workload, about 6 minutes)
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import OracleFilter, COST_LA, COST_MIX, COST_EXP  # noqa: E402
from oracle.oracle import GOLDEN_RATIO  # noqa: E402
from oracle.oracle import bits_of_bitmap  # noqa: E402


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<u8").tobytes()).hexdigest()


def dna():
    """DNA 31-mer workload: 5e7-base genome (seed 2), canonical 31-mers, M = 2^21,
    k = 16, c = 3, cost^LA mu = 3.5, B = 2^20, hash seed 2; queries: the 31-mers,
    then 31-mers of a second genome (seed 3)."""
    t0 = time.time()
    keys = workloads.canonical_kmers(workloads.random_genome(2, 50_000_000), 31)
    other = workloads.canonical_kmers(workloads.random_genome(3, 50_000_000), 31)
    o = OracleFilter(1 << 21, 16, 3, COST_LA, 3.5, seed=2, batch=1 << 20)
    o.insert(keys)
    queries = np.concatenate([keys, other])
    bm, first = o.query(queries, return_first=True)
    hist, total = o.histogram()
    hits = bits_of_bitmap(bm, len(queries))
    pbar = float(first[: len(keys)].astype(np.float64).mean())
    lines = [
        "# Oracle results of the DNA 31-mer workload (written by make_golden.py dna).",
        "# 50,000,000-base genome (splitmix64 seed 2) -> canonical 31-mers; filter M = 2^21 blocks,",
        "# k = 16, c = 3, cost^LA mu = 3.5, B = 2^20, hash_seed = 2. Queries: the 31-mers, then",
        "# the 31-mers of a second genome (seed 3).",
        "n_insert = %d" % len(keys),
        "n_query = %d" % len(queries),
        "inserted = %d" % o.inserted,
        "skipped = %d" % o.skipped,
        "set_bits = %d" % total,
        "words_sha256 = %s" % sha(o.words),
        "bitmap_sha256 = %s" % sha(bm),
        "query_hits = %d" % int(hits.sum()),
        "false_positives = %d" % int(hits[len(keys):].sum()),
        "pbar_positive = %.6f" % pbar,
        "hist_sha256 = %s" % sha(hist),
        "oracle_seconds = %.0f" % (time.time() - t0),
    ]
    with open(os.path.join(HERE, "dna_kmer_31_c3_la.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines))


# Overload sweep: M = 2^23 blocks (512 MiB), k = 12, B = 2^20; keys are the
# splitmix64 stream of seed 3001, grown through n = floor(2^32 / b) for
# b = 20, 18, ..., 6 bits per key (Sec. 4.1: the FPR under overload), one insert
# call per step; 10^8 negatives from seed 3002 queried at every point.
SWEEP_SETTINGS = [(1, COST_EXP, GOLDEN_RATIO), (2, COST_MIX, 50.0), (2, COST_LA, 3.5),
                  (2, COST_EXP, GOLDEN_RATIO), (3, COST_MIX, 50.0), (3, COST_LA, 3.5),
                  (3, COST_EXP, GOLDEN_RATIO)]
SWEEP_BITS = [20, 18, 16, 14, 12, 10, 8, 6]
SWEEP_M, SWEEP_K, SWEEP_B, SWEEP_NEG = 1 << 23, 12, 1 << 20, 100_000_000
COST_NAMES = {COST_MIX: "MIX", COST_LA: "LA", COST_EXP: "EXP"}


def sweep_name(idx):
    c, kind, _ = SWEEP_SETTINGS[idx]
    return "overload_sweep_c%d_%s.txt" % (c, COST_NAMES[kind])


def sweep(idx):
    idx = int(idx)
    c, kind, par = SWEEP_SETTINGS[idx]
    t0 = time.time()
    o = OracleFilter(SWEEP_M, SWEEP_K, c, kind, par, seed=3001, batch=SWEEP_B)
    neg = workloads.uniform_keys(3002, SWEEP_NEG)
    chunk = 32 * SWEEP_B
    lines = ["# Oracle results of the overload sweep (written by make_golden.py sweep %d)." % idx,
             "# M = 2^23, k = 12, c = %d, cost %s param %.17g, B = 2^20, hash_seed = 3001;" % (
                 c, COST_NAMES[kind], par),
             "# keys: splitmix64 seed 3001 grown to floor(2^32/b); negatives: 1e8 from seed 3002.",
             "# b | n | inserted | skipped | set_bits | false_positives | words_sha256 | neg_bitmap_sha256"]
    n_prev = 0
    for b in SWEEP_BITS:
        n = (1 << 32) // b
        # one insert call for keys [n_prev, n): batches restart at n_prev;
        # chunks of 32 batches are the same batches
        s0 = n_prev
        while s0 < n:
            cnt = min(chunk, n - s0)
            o.insert(workloads.splitmix64(3001, cnt, s0))
            s0 += cnt
        n_prev = n
        bm = o.query(neg)
        hist, total = o.histogram()
        W = int(bits_of_bitmap(bm, len(neg)).sum())
        lines.append("%d | %d | %d | %d | %d | %d | %s | %s" % (
            b, n, o.inserted, o.skipped, total, W, sha(o.words), sha(bm)))
        print(lines[-1], "(%.0f s)" % (time.time() - t0), flush=True)
    lines.append("# oracle_seconds = %.0f" % (time.time() - t0))
    with open(os.path.join(HERE, sweep_name(idx)), "w") as fh:
        fh.write("\n".join(lines) + "\n")


def many():
    """256 independent filters (workloads.many_filter_config): k = 11, c = 2,
    cost^EXP beta = golden ratio, hash_seed = the filter's key seed, B_f as
    configured; per filter: all keys inserted, then its queries."""
    t0 = time.time()
    cfg = workloads.many_filter_config()
    lines = ["# Oracle results of the 256-filter workload (written by make_golden.py many).",
             "# k = 11, c = 2, cost^EXP beta = golden ratio; per filter: n, M, B, hash_seed = key seed.",
             "# f | n | M | B | inserted | skipped | words_sha256 | bitmap_sha256"]
    for it in cfg:
        keys, queries = workloads.many_filter_keys(it)
        o = OracleFilter(it["M"], 11, 2, COST_EXP, GOLDEN_RATIO, seed=it["key_seed"], batch=it["B"])
        o.insert(keys)
        bm = o.query(queries)
        lines.append("%d | %d | %d | %d | %d | %d | %s | %s" % (
            it["index"], it["n"], it["M"], it["B"], o.inserted, o.skipped, sha(o.words), sha(bm)))
    lines.append("# oracle_seconds = %.0f" % (time.time() - t0))
    with open(os.path.join(HERE, "many_filters_256.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print(lines[-1])


if __name__ == "__main__":
    args = sys.argv[1:] or ["dna"]
    if args[0] == "sweep":
        sweep(args[1])
    else:
        for w in args:
            globals()[w]()
