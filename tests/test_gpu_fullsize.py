"""Full-size parity: the DNA 31-mer workload at its real size, in the launch
configuration the benchmark times, against the oracle's stored results.

tests/golden/dna_kmer_31_c3_la.txt was written by tests/golden/make_golden.py,
which runs only the oracle (about five minutes on one core). The GPU filter
words and query bitmap must hash to the same SHA-256, and the counters must
match.
"""
import hashlib
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                out[k.strip()] = v.strip()
    return out


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<u8").tobytes()).hexdigest()


def test_dna_kmer_workload_matches_oracle_digests():
    import torch
    import bench
    import paper_2501_18977_gb300 as bc
    g = _golden("dna_kmer_31_c3_la.txt")
    keys, queries = bench.make_workload()
    assert len(keys) == int(g["n_insert"]) and len(queries) == int(g["n_query"])
    C = bench.CONFIG
    f = bc.Filter(C["nblocks"], C["k"], C["choices"], bc.COST_LA, C["mu"],
                  hash_seed=C["hash_seed"], batch=C["batch"])
    try:
        dk = torch.from_numpy(keys.view(np.int64)).cuda()
        dq = torch.from_numpy(queries.view(np.int64)).cuda()
        f.insert(dk)
        bm = f.query(dq).cpu().numpy().view(np.uint64)
        st = f.stats()
        words = f.words_host()
    finally:
        f.close()
    assert (st.inserted, st.skipped, st.set_bits) == (
        int(g["inserted"]), int(g["skipped"]), int(g["set_bits"]))
    hits = int(np.unpackbits(bm.view(np.uint8), bitorder="little")[: len(queries)].sum())
    assert hits == int(g["query_hits"])
    assert _sha(bm) == g["bitmap_sha256"]
    assert _sha(words) == g["words_sha256"]
    assert _sha(np.array(list(st.hist), dtype=np.uint64)) == g["hist_sha256"]
