"""The learned cost on the GPU against its float64 oracle.

Forward values, parameter gradients, the Adam step and the sampled training
insert (choices and score weights) of the CUDA kernels must match
oracle/learned.py; a filter using a learned cost table must match the oracle
bit for bit; and training must improve the reward it optimises.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import learned as ol
from oracle.oracle import OracleFilter, COST_EXP, GOLDEN_RATIO
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


def _net(k, seed):
    import paper_2501_18977_gb300 as bc
    return bc.Mlp(k, seed)


def test_forward_matches_oracle():
    import torch
    for k in (4, 14, 32):
        m = _net(k, 7 + k)
        try:
            t = torch.empty(513 * (k + 1), dtype=torch.float32, device="cuda")
            m.forward(t)
            got = t.double().cpu().numpy()
            want = ol.forward(m.params().astype(np.float64), k)
            assert np.allclose(got, want, rtol=1e-5, atol=1e-5)
        finally:
            m.close()


def test_backward_matches_oracle():
    import torch
    k = 12
    m = _net(k, 3)
    try:
        rng = np.random.default_rng(5)
        w = rng.normal(0, 1, 513 * (k + 1)).astype(np.float32)
        w[rng.random(w.shape) < 0.5] = 0.0
        w2 = rng.normal(0, 1, 513 * (k + 1)).astype(np.float32)
        rows = torch.from_numpy(np.stack([w, w2])).cuda()
        m.backward(rows, torch.tensor([0.75, -0.5], dtype=torch.float64, device="cuda"))
        got = m.grad()
        p = m.params().astype(np.float64)
        want = 0.75 * ol.backward(p, k, w.astype(np.float64)) - 0.5 * ol.backward(p, k, w2.astype(np.float64))
        scale = np.abs(want).max()
        assert np.allclose(got, want, rtol=2e-4, atol=2e-5 * scale)
    finally:
        m.close()


def test_adam_step_matches_oracle():
    import torch
    k = 6
    m = _net(k, 9)
    try:
        rng = np.random.default_rng(2)
        w = torch.from_numpy(rng.normal(0, 1, 513 * (k + 1)).astype(np.float32)).cuda()
        p0 = m.params().astype(np.float64)
        m.backward(w, torch.ones(1, dtype=torch.float64, device="cuda"))
        g = m.grad()
        m.adam_step(1e-2)
        want, _, _ = ol.adam(p0, g.astype(np.float32).astype(np.float64), np.zeros_like(p0),
                             np.zeros_like(p0), 1, 1e-2)
        assert np.allclose(m.params(), want, rtol=1e-5, atol=1e-6)
        assert not m.grad().any()
    finally:
        m.close()


@pytest.mark.parametrize("c,tau", [(2, 0.5), (3, 0.1), (3, 2.0)])
def test_sampled_insert_matches_oracle(c, tau):
    """One batch against a pre-filled filter: every choice equals the
    oracle's draw unless the uniform sits within 1e-6 of a boundary, and the
    score weights agree."""
    import torch
    import paper_2501_18977_gb300 as bc
    M, k, seed = 64, 8, 11
    pre = workloads.uniform_keys(301, 900)
    keys = workloads.uniform_keys(302, 2000)
    rng = np.random.default_rng(c)
    table = rng.normal(0, 1, 513 * (k + 1)).astype(np.float32)
    f = bc.Filter(M, k, c, bc.COST_EXP, GOLDEN_RATIO, hash_seed=4, batch=len(keys))
    try:
        f.insert(to_dev(pre))
        o = OracleFilter(M, k, c, COST_EXP, GOLDEN_RATIO, seed=4, batch=len(keys))
        o.insert(pre)
        assert np.array_equal(f.words_host(), o.words)
        dw = torch.zeros(513 * (k + 1), dtype=torch.float32, device="cuda")
        dch = torch.zeros(len(keys), dtype=torch.uint8, device="cuda")
        bc.blowchoc_insert_sampled(f.handle, to_dev(keys), len(keys), torch.from_numpy(table).cuda(), tau,
                                   seed, dw, dch)
        got_ch = dch.cpu().numpy().astype(np.int64)
        ch, w, margins = ol.sampled_batch(o, keys, table.astype(np.float64), tau, seed)
        close = margins < 1e-6
        assert (got_ch[~close] == ch[~close]).all()
        assert close.sum() < 5
        if not close.any():
            assert np.allclose(dw.cpu().numpy(), w, rtol=1e-4, atol=1e-3)
    finally:
        f.close()


def test_learned_table_filter_matches_oracle():
    """A cost table from the network drives the exact greedy insert: GPU
    words equal the oracle's with the same table."""
    import torch
    import paper_2501_18977_gb300 as bc
    M, k, c, B = 2048, 14, 2, 8192
    m = _net(k, 21)
    try:
        t = torch.empty(513 * (k + 1), dtype=torch.float32, device="cuda")
        m.forward(t)
        table = t.double().cpu().numpy()
    finally:
        m.close()
    keys = workloads.uniform_keys(401, 60000)
    f = bc.Filter(M, k, c, bc.COST_EXP, GOLDEN_RATIO, hash_seed=8, batch=B)
    try:
        f.set_cost_table(table)
        f.insert(to_dev(keys))
        words = f.words_host()
    finally:
        f.close()
    o = OracleFilter(M, k, c, COST_EXP, GOLDEN_RATIO, seed=8, batch=B)
    o.set_cost_table(table)
    o.insert(keys)
    assert np.array_equal(words, o.words)


def test_training_improves_its_reward():
    """A short run on small filters: the mean reward of the last steps beats
    the first steps' (the policy learns what it is rewarded for)."""
    from paper_2501_18977_gb300.learned import train_cost_table
    M, k, c, B = 256, 14, 2, 256
    n = int(M * 512 * math.log(2) / k)
    table, rewards, mlp = train_cost_table(M, k, c, B, n, steps=60, filters=32, tau=0.05, lr=1e-2, seed=3)
    mlp.close()
    assert np.isfinite(table).all()
    first, last = np.mean(rewards[:10]), np.mean(rewards[-10:])
    print("reward first/last", first, last)
    assert last > first, (first, last)


def _held_out_fpr(bc, table, M, k, c, B, keys, neg, bm):
    """Measured FPR (W/N over `neg`) of a held-out filter built greedily with
    cost^EXP (beta = golden ratio), or with `table` in its place."""
    import torch
    f = bc.Filter(M, k, c, bc.COST_EXP, GOLDEN_RATIO, hash_seed=1, batch=B)
    try:
        if table is not None:
            f.set_cost_table(table)
        f.insert(keys)
        f.query(neg, bm)
        torch.cuda.synchronize()
        W = int(np.unpackbits(bm.cpu().numpy().view(np.uint8), bitorder="little")[: neg.numel()].sum())
        return W / neg.numel()
    finally:
        f.close()


def test_learned_gain_over_exp_cost(record_property):
    """What the trained network gains over the method without it: a short
    training run (32 filters of 512 blocks per step, 16 bits per key, k = 14,
    c = 2), then a held-out filter of 4096 blocks at the same load built with
    the learned table and with cost^EXP (beta = golden ratio, App. C), FPR
    measured over 10^7 negatives. The gain (FPR of cost^EXP / FPR learned)
    is recorded as measured and may be below 1; the floor of 0.8 fails a
    broken table, which the test shows by scoring the negated cost^EXP table
    (it prefers the fuller block) the same way."""
    import torch
    import paper_2501_18977_gb300 as bc
    from paper_2501_18977_gb300.learned import train_cost_table
    k, c = 14, 2
    Mt = 512
    nt = Mt * 512 // 16
    table, rewards, mlp = train_cost_table(Mt, k, c, nt // 16, nt, steps=80, filters=32, tau=0.05,
                                           lr=3e-3, seed=7)
    mlp.close()
    M = 4096
    n = M * 512 // 16
    keys = to_dev(workloads.uniform_keys(11, n))
    neg = to_dev(workloads.uniform_keys(12, 10_000_000))
    bm = torch.empty((neg.numel() + 63) // 64, dtype=torch.int64, device="cuda")
    fpr_exp = _held_out_fpr(bc, None, M, k, c, n // 16, keys, neg, bm)
    fpr_learned = _held_out_fpr(bc, table, M, k, c, n // 16, keys, neg, bm)
    # the negated cost^EXP table: the same rank order reversed
    L = np.repeat(np.arange(513, dtype=np.float64), k + 1)
    a = np.tile(np.arange(k + 1, dtype=np.float64), 513)
    broken = -(GOLDEN_RATIO ** ((L + a) / 128.0) + a / k)
    fpr_broken = _held_out_fpr(bc, broken, M, k, c, n // 16, keys, neg, bm)
    gain, gain_broken = fpr_exp / fpr_learned, fpr_exp / fpr_broken
    record_property("learned_gain_vs_exp", gain)
    record_property("broken_table_gain_vs_exp", gain_broken)
    print("FPR exp %.6g learned %.6g broken %.6g; gain %.4f, broken %.4f"
          % (fpr_exp, fpr_learned, fpr_broken, gain, gain_broken))
    assert gain_broken < 0.8
    assert gain > 0.8, (fpr_exp, fpr_learned)
