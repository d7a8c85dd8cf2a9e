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
