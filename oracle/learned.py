"""Oracle of the learned block-selection cost. TEST INFRASTRUCTURE ONLY.

Not in the paper: the learned cost is a library extension whose network takes
the paper's cost arguments (Section 3.2: j, the block's set bits after the
insertion, and a, the newly set bits) as x = (j / 512, a / k) and outputs a
cost g(x). Everything here is plain numpy in float64, written from the
definitions: a two-hidden-layer tanh network, its exact gradient, the softmax
policy over a key's candidates and the score-function weight
d log pi(chosen) / d g. Pinned in tests/test_oracle_pins.py: the forward pass
by a hand-derived value, the gradient by finite differences, the score weight
by a finite difference of log pi(s) (scipy's log_softmax) and the sampler by
draw frequencies against softmax(-g / tau), Adam by hand-computed first and
second steps, and the uniforms by the generator's check vector.
"""
import numpy as np

from .oracle import OracleFilter

H = 32
NPARAMS = H * H + 5 * H + 1


def unpack(params):
    """W1 (H x 2), b1 (H), W2 (H x H, row = output unit), b2 (H), w3 (H), b3."""
    p = np.asarray(params, dtype=np.float64)
    assert p.shape == (NPARAMS,)
    W1 = p[0:2 * H].reshape(H, 2)
    b1 = p[2 * H:3 * H]
    W2 = p[3 * H:3 * H + H * H].reshape(H, H)
    b2 = p[3 * H + H * H:4 * H + H * H]
    w3 = p[4 * H + H * H:5 * H + H * H]
    b3 = p[5 * H + H * H]
    return W1, b1, W2, b2, w3, b3


def grid_inputs(k):
    """x for every grid point p = L (k + 1) + a: ((L + a) / 512, a / k)."""
    L = np.repeat(np.arange(513, dtype=np.float64), k + 1)
    a = np.tile(np.arange(k + 1, dtype=np.float64), 513)
    return np.stack([(L + a) / 512.0, a / float(k)], axis=1)


def forward(params, k):
    """g(x_p) at every grid point."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    X = grid_inputs(k)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ w3 + b3


def backward(params, k, w):
    """sum_p w_p d g(x_p) / d params, by the chain rule, in float64."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    X = grid_inputs(k)
    w = np.asarray(w, dtype=np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    d2 = (w[:, None] * w3[None, :]) * (1.0 - h2 ** 2)          # dL/d(pre-activation 2)
    d1 = (d2 @ W2) * (1.0 - h1 ** 2)                             # dL/d(pre-activation 1)
    g = np.zeros(NPARAMS)
    g[0:2 * H] = (d1.T @ X).reshape(-1)
    g[2 * H:3 * H] = d1.sum(axis=0)
    g[3 * H:3 * H + H * H] = (d2.T @ h1).reshape(-1)
    g[3 * H + H * H:4 * H + H * H] = d2.sum(axis=0)
    g[4 * H + H * H:5 * H + H * H] = h2.T @ w
    g[5 * H + H * H] = w.sum()
    return g


def splitmix_uniform(seed, idx):
    """Uniform in [0, 1) from splitmix64 (Steele, Lea and Flood 2014) of `seed`
    at stream position idx: the top 53 bits of the idx-th output."""
    M64 = (1 << 64) - 1
    z = (seed + (idx + 1) * 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    z ^= z >> 31
    return (z >> 11) / float(1 << 53)


def sampled_batch(filt: OracleFilter, keys, table, tau, seed):
    """One batch of training-mode choices against the filter as it stands:
    per key, skip if a candidate holds F(x); otherwise pi_i proportional to
    exp(-table[p_i] / tau), the choice is the first i whose cumulative weight
    exceeds u * sum (u from splitmix_uniform(seed, key index)), and
    w[p_i] += (pi_i - 1{i chosen}) / tau. Returns (choices, w, margins) where
    margins[t] is the distance of u * sum to the nearest cumulative boundary
    divided by the sum (small margins may flip under float rounding)."""
    k1 = filt.k + 1
    table = np.asarray(table, dtype=np.float64)
    w = np.zeros(513 * k1)
    choices = np.full(len(keys), 255, dtype=np.int64)
    margins = np.full(len(keys), np.inf)
    for t, x in enumerate(keys):
        terms = [filt.block_terms(b, int(x)) for b in filt.candidates(int(x))]
        if min(a for _, a in terms) == 0:
            continue
        pts = [L * k1 + a for L, a in terms]
        g = np.array([table[p] for p in pts])
        e = np.exp(-(g - g.min()) / tau)
        z = e.sum()
        u = splitmix_uniform(seed, t) * z
        cdf = np.cumsum(e)
        s = int(np.searchsorted(cdf[:-1], u, side="right"))
        choices[t] = s
        margins[t] = np.min(np.abs(cdf[:-1] - u)) / z if len(cdf) > 1 else np.inf
        for i, p in enumerate(pts):
            w[p] += (e[i] / z - (1.0 if i == s else 0.0)) / tau
    return choices, w, margins


def adam(params, grad, m1, m2, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015) on float64 copies."""
    m1 = b1 * m1 + (1 - b1) * grad
    m2 = b2 * m2 + (1 - b2) * grad ** 2
    mh = m1 / (1 - b1 ** step)
    vh = m2 / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m1, m2
