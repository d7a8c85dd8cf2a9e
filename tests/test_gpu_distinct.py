"""Distinct bit selection (Appendix B) on the GPU against the oracle.

The GPU computes the f_i-th free position by counting free bits per word;
the oracle follows the paper's increment rule with an insertion sort. Filter
words, bitmaps and counters must agree on every insert and query path.
"""
import numpy as np
import pytest

import workloads
from oracle import COST_MIX, COST_LA, COST_EXP
from oracle.oracle import GOLDEN_RATIO, OracleFilter
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu

PHI = GOLDEN_RATIO


def _oracle(M, k, c, kind, par, seed, B, keys, queries):
    o = OracleFilter(M, k, c, kind, par, seed=seed, batch=B, bitsel=1)
    o.insert(keys)
    return o, o.query(queries)


@pytest.mark.parametrize("M,k,c,kind,par,B,n,tune", [
    (1024, 14, 2, COST_EXP, PHI, 50000, 120000, {}),                      # persistent
    (999, 11, 3, COST_LA, 3.5, 1000, 30000, {}),                          # single CTA
    (512, 16, 2, COST_MIX, 50.0, 1, 20000, {}),                           # exact sequential rounds
    (300, 20, 3, COST_EXP, PHI, 1, 5000, dict(seq_window=0)),              # one warp
    (4096, 12, 2, COST_MIX, 50.0, 65536, 200000, dict(set_mode=1)),        # sort by block
    (4096, 12, 3, COST_LA, 3.5, 65536, 200000, dict(set_mode=2)),          # bulk set
    (2048, 32, 2, COST_EXP, PHI, 30000, 60000, dict(persistent=0, lanes_choose=8, lanes_set=2,
                                                    lanes_query=8, query_early=0)),
    (6150, 9, 1, COST_EXP, PHI, 20000, 60000, dict(lanes_query=4)),
])
def test_distinct_matches_oracle(M, k, c, kind, par, B, n, tune):
    import paper_2501_18977_gb300 as bc
    keys = workloads.uniform_keys(M + 31, n)
    neg = workloads.disjoint_keys(M + 32, n // 2, keys)
    queries = np.concatenate([keys[: n // 2], neg])
    f = bc.Filter(M, k, c, kind, par, hash_seed=6, batch=B, bitsel=1)
    try:
        if tune:
            f.set_tuning(**tune)
        f.insert(to_dev(keys))
        bm = f.query(to_dev(queries)).cpu().numpy().view(np.uint64)
        words = f.words_host()
        st = f.stats()
        ab, af = f.multipliers()
    finally:
        f.close()
    o, obm = _oracle(M, k, c, kind, par, 6, B, keys, queries)
    assert af[:k] == [int(v) for v in o.a_bit[:k]]
    assert np.array_equal(words, o.words)
    assert np.array_equal(bm, obm)
    assert (st.inserted, st.skipped) == (o.inserted, o.skipped)
    # every key sets exactly k bits somewhere: popcount of each inserted mask
    assert st.set_bits == int(sum(bin(int(w)).count("1") for w in o.words))


def test_distinct_in_many_filter_launch():
    import torch
    import paper_2501_18977_gb300 as bc
    specs = [(777, 12, 2, COST_EXP, PHI, 4096, 40000, 1), (500, 10, 3, COST_MIX, 50.0, 2048, 20000, 0),
             (2000, 16, 2, COST_LA, 3.5, 8192, 60000, 1)]
    filters, ins, qry, bms, data = [], [], [], [], []
    for j, (M, k, c, kind, par, B, n, bitsel) in enumerate(specs):
        keys = workloads.uniform_keys(900 + j, n)
        queries = np.concatenate([keys[: n // 2], workloads.uniform_keys(950 + j, n // 2)])
        f = bc.Filter(M, k, c, kind, par, hash_seed=40 + j, batch=B, bitsel=bitsel)
        filters.append(f)
        b = torch.zeros((len(queries) + 63) // 64, dtype=torch.int64, device="cuda")
        ins.append((f, to_dev(keys), n, None))
        qry.append((f, to_dev(queries), len(queries), b))
        bms.append(b)
        data.append((keys, queries))
    batch = bc.Batch()
    try:
        batch.insert_many(ins)
        batch.query_many(qry)
        torch.cuda.synchronize()
        for (M, k, c, kind, par, B, n, bitsel), f, b, (keys, queries), j in zip(specs, filters, bms, data,
                                                                                range(len(specs))):
            o = OracleFilter(M, k, c, kind, par, seed=40 + j, batch=B, bitsel=bitsel)
            o.insert(keys)
            assert np.array_equal(f.words_host(), o.words)
            assert np.array_equal(b.cpu().numpy().view(np.uint64), o.query(queries))
    finally:
        batch.close()
        for f in filters:
            f.close()
