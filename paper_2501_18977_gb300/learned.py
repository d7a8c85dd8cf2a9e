"""Training loop of the learned block-selection cost (not in the paper).

Control flow only: every computation (network forward and backward, sampled
insertion, load statistics, Adam) runs in the library's CUDA kernels.

Policy: for each key that is not already contained, pick candidate i with
probability softmax(-g(x_i) / tau). Reward of one build: R = -log2 of the
filter's histogram FPR estimate after inserting its keys. The score-function
gradient of E[R] is E[(R - b) sum_decisions d log pi / d g]. One training
step builds F independent filters of the same shape (F reward samples), each
with its own keys, and uses the mean reward of the others as each one's
baseline b; the sampled inserts accumulate the per-point weights
d log pi / d g per filter, and one backward launch applies the chain rule to
all rows with their advantages.
"""
import math

import numpy as np

from . import binding as _b


def train_cost_table(M, k, c, B, n, steps=200, filters=32, tau=0.05, lr=3e-3, seed=1, key_seed=1000,
                     log=None):
    """Trains the network on building `filters` filters of M blocks (k, c,
    batch B) from n keys each (splitmix64 streams key_seed + f, fresh per
    step); returns (cost table as float64 numpy array of 513 (k + 1) values,
    list of per-step mean rewards, the network)."""
    import torch
    import workloads
    k1 = k + 1
    P = 513 * k1
    mlp = _b.Mlp(k, seed)
    table = torch.empty(P, dtype=torch.float32, device="cuda")
    w = torch.zeros(filters, P, dtype=torch.float32, device="cuda")
    fs = [_b.Filter(M, k, c, _b.COST_EXP, (1 + 5 ** 0.5) / 2, hash_seed=seed + i, batch=B)
          for i in range(filters)]
    rewards = []
    try:
        for step in range(steps):
            mlp.forward(table)
            w.zero_()
            R = np.zeros(filters)
            for i, f in enumerate(fs):
                keys = workloads.splitmix64(key_seed + 7919 * step + i, n)
                d = torch.from_numpy(keys.view(np.int64)).cuda()
                f.clear()
                _b.blowchoc_insert_sampled(f.handle, d, n, table, tau, seed * 1000003 + step * 131 + i, w[i])
                R[i] = -math.log2(max(f.stats().fpr_est, 1e-300))
            rewards.append(float(R.mean()))
            # leave-one-out baseline; the loss is -(R - b) log pi, so scale by -(R - b)
            adv = R - (R.sum() - R) / max(filters - 1, 1)
            scales = torch.from_numpy(-adv).cuda()
            mlp.backward(w, scales)
            mlp.adam_step(lr)
            if log:
                log(step, float(R.mean()))
        mlp.forward(table)
        out = table.double().cpu().numpy()
    finally:
        for f in fs:
            f.close()
    return out, rewards, mlp
