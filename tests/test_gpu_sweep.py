"""Full-size parity of the overload sweep against the oracle's stored results.

For every filter setting whose oracle results exist in tests/golden
(written by make_golden.py sweep I), the GPU filter is grown through the same
load points, 20 down to 6 bits per key (Sec. 4.1: the FPR under overload; one
insert call per point) and its words, counters and false
positives among 10^8 negatives must match the oracle's exactly.
"""
import hashlib
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SETTINGS = [(1, "EXP"), (2, "MIX"), (2, "LA"), (2, "EXP"), (3, "MIX"), (3, "LA"), (3, "EXP")]


def _rows(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        return None
    out = []
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or "|" not in line:
                continue
            f = [x.strip() for x in line.split("|")]
            out.append(dict(b=int(f[0]), n=int(f[1]), inserted=int(f[2]), skipped=int(f[3]),
                            set_bits=int(f[4]), fp=int(f[5]), words=f[6], bitmap=f[7]))
    return out


@pytest.fixture(scope="module")
def sweep_inputs():
    import torch
    import workloads
    nmax = max([r["n"] for c, cost in SETTINGS
                for r in (_rows("overload_sweep_c%d_%s.txt" % (c, cost)) or [])] + [1])
    keys = torch.empty(nmax, dtype=torch.int64, device="cuda")
    chunk = 1 << 25
    for s0 in range(0, nmax, chunk):
        c = min(chunk, nmax - s0)
        keys[s0:s0 + c].copy_(torch.from_numpy(workloads.splitmix64(3001, c, s0).view(np.int64)))
    neg = torch.from_numpy(workloads.uniform_keys(3002, 100_000_000).view(np.int64)).cuda()
    return keys, neg


@pytest.mark.parametrize("c,cost", SETTINGS)
def test_overload_sweep_matches_oracle(c, cost, sweep_inputs):
    import torch
    import paper_2501_18977_gb300 as bc
    rows = _rows("overload_sweep_c%d_%s.txt" % (c, cost))
    if rows is None:
        pytest.skip("oracle results for this setting not stored")
    keys, neg = sweep_inputs
    par = {"MIX": 50.0, "LA": 3.5, "EXP": (1.0 + 5 ** 0.5) / 2.0}[cost]
    kind = {"MIX": bc.COST_MIX, "LA": bc.COST_LA, "EXP": bc.COST_EXP}[cost]
    f = bc.Filter(1 << 23, 12, c, kind, par, hash_seed=3001, batch=1 << 20)
    bm = torch.empty((neg.numel() + 63) // 64, dtype=torch.int64, device="cuda")
    try:
        n_prev = 0
        for row in rows:
            f.insert(keys[n_prev:row["n"]])
            n_prev = row["n"]
            f.query(neg, bm)
            h = bm.cpu().numpy().view(np.uint64)
            st = f.stats()
            assert (st.inserted, st.skipped, st.set_bits) == (row["inserted"], row["skipped"], row["set_bits"])
            assert int(np.unpackbits(h.view(np.uint8), bitorder="little").sum()) == row["fp"]
            assert hashlib.sha256(h.astype("<u8").tobytes()).hexdigest() == row["bitmap"]
            assert hashlib.sha256(f.words_host().astype("<u8").tobytes()).hexdigest() == row["words"]
    finally:
        f.close()
