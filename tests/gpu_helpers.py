"""Shared helpers of the GPU tests: run one configuration through the C ABI
and through the oracle on the same seeded keys."""
import numpy as np

from oracle import OracleFilter


def to_dev(keys):
    import torch
    return torch.from_numpy(np.ascontiguousarray(keys, dtype=np.uint64).view(np.int64)).cuda()


def gpu_run(M, k, c, kind, par, seed, B, keys, queries, chunks=None, tune=None):
    """Insert `keys` (optionally in several insert calls, split at `chunks`),
    query `queries`; returns (words, bitmap, stats) as host values. `tune`
    holds launch-configuration fields to set first."""
    import paper_2501_18977_gb300 as bc
    f = bc.Filter(M, k, c, kind, par, hash_seed=seed, batch=B)
    try:
        if tune:
            f.set_tuning(**tune)
        dk = to_dev(keys)
        if chunks:
            edges = [0] + list(chunks) + [len(keys)]
            for a, b in zip(edges[:-1], edges[1:]):
                f.insert(dk[a:b])
        else:
            f.insert(dk)
        bm = f.query(to_dev(queries)).cpu().numpy().view(np.uint64) if len(queries) else \
            np.zeros(0, dtype=np.uint64)
        words = f.words_host()
        st = f.stats()
        return words, bm, st
    finally:
        f.close()


def oracle_run(M, k, c, kind, par, seed, B, keys, queries):
    o = OracleFilter(M, k, c, kind, par, seed=seed, batch=B)
    o.insert(keys)
    bm = o.query(queries)
    hist, total = o.histogram()
    return o, bm, hist, total
