"""False-positive-rate and load sweeps at the paper's scale, on the device.

The evaluation of Section 4.1 (Fig. 4) and Appendix C (Fig. 8, Fig. 10)
inserts n = 2 * 10^9 uniform 64-bit keys and counts the false positives W of
N = 2 * 10^9 keys that were not inserted (FPR = W / N). Here every key is
generated on the device (blowchoc_generate_keys: splitmix64 streams of two
seeds), inserted in chunks whose edges fall on batch edges, and the negatives
are counted by blowchoc_query_count, so a point needs no host transfer
beyond a few counters.

Sizes follow Appendix C: a standard Bloom filter for FPR 2^-k has
m = n k / ln 2 bits, rounded up to a multiple of 512; a relative size rho
(the x-axis of Fig. 4) scales m before rounding.

Insertion runs in batches (the library's batch rule) of
B = 2^floor(log2(M / 64)) keys (at most 2^20): a batch holds at most 1/64 of
the blocks, where the measured cost of batching against one key at a time is
far below the noise of W.
"""
import math
import time

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1
PHI = (1.0 + math.sqrt(5.0)) / 2.0
LN2 = math.log(2.0)

# the grids of the paper's figures (k values of Fig. 10; Fig. 4 shows a subset)
PAPER_KS = (4, 7, 10, 14, 17, 20)
REL_SIZES = (0.80, 0.85, 0.90, 0.95, 1.00, 1.05, 1.10, 1.15, 1.20, 1.25, 1.30)
COST_PARAMS = {  # cost kind (binding constant) -> parameter grid
    0: (1.0, 2.5, 5.0, 10.0, 20.0, 50.0, 100.0),          # mixed, sigma
    1: (0.5, 1.0, 2.0, 3.5, 5.0, 7.0, 10.0),              # lookahead, mu
    2: (1.2, 1.4, 1.5, 1.6, PHI, 1.7, 1.8, 2.0, 2.5),     # exponential, beta
}


def bloom_bits(n, k, rho=1.0):
    """Standard Bloom size for FPR 2^-k, m = n k / ln 2 bits (Section 2.1),
    scaled by rho."""
    return rho * n * k / LN2


def blocks_for(n, k, rho=1.0):
    """512-bit blocks of the filter: m rounded up to a multiple of 512."""
    return max(1, int(math.ceil(bloom_bits(n, k, rho) / 512.0)))


def batch_for(M):
    """Batch size of a sweep point: 2^floor(log2(M / 64)), in [1, 2^20]."""
    return 1 << max(0, min(20, int(math.floor(math.log2(max(M / 64.0, 1.0))))))


def bloom_fpr(n, m, k):
    """Standard Bloom filter FPR (1 - e^(-k n / m))^k (Section 2.1, Eq. 1);
    the reference curve of Fig. 4."""
    return (1.0 - math.exp(-k * n / m)) ** k


def blocked_bloom_fpr(n, M, k):
    """One-choice Blocked Bloom FPR under ideal hashing, the model of Putze,
    Sanders and Singler (2007) that Section 2.2 cites: a block receives
    i ~ Poisson(n / M) keys, each of its bits is set with probability
    1 - (1 - 1/512)^(i k), and a negative needs k independent positions set."""
    lam = n / M
    total = 0.0
    i = 0
    top = lam + 12.0 * math.sqrt(lam + 1.0) + 20.0
    while i <= top:
        logp = -lam + (i * math.log(lam) if lam > 0 else (0.0 if i == 0 else -math.inf)) - math.lgamma(i + 1.0)
        total += math.exp(logp) * (1.0 - (1.0 - 1.0 / 512.0) ** (i * k)) ** k
        i += 1
    return total


def streams_disjoint(key_seed, n, neg_seed, n_neg):
    """True if outputs 0..n-1 of splitmix64(key_seed) and 0..n_neg-1 of
    splitmix64(neg_seed) share no value. Output i is a bijection of the state
    seed + (i + 1) * GAMMA (mod 2^64), so output j of the first equals output
    i of the second exactly when (j - i) * GAMMA = neg_seed - key_seed, i.e.
    j - i = d with d = (neg_seed - key_seed) * GAMMA^-1 mod 2^64."""
    d = ((neg_seed - key_seed) * pow(GAMMA, -1, 1 << 64)) & MASK64
    return not (d < n or d > (1 << 64) - n_neg)


def fpr_point(n, M, k, c, cost, param, bitsel=0, B=None, key_seed=1, neg_seed=2, n_neg=None,
              hash_seed=None, chunk=1 << 27, stream=None):
    """Build one filter of M blocks from n generated keys and count the false
    positives of n_neg generated negatives. Returns a dict with W, N, fpr,
    the filter's counters and histogram summary, and the device times."""
    import torch

    from .binding import Filter, generate_keys

    n_neg = n if n_neg is None else n_neg
    B = batch_for(M) if B is None else B
    if not streams_disjoint(key_seed, n, neg_seed, n_neg):
        raise ValueError("the negative stream overlaps the inserted keys")
    step = max(B, (chunk // B) * B)  # chunk edges on batch edges
    hash_seed = (key_seed * 0x100000001B3 + M * 31 + k) & MASK64 if hash_seed is None else hash_seed
    s = torch.cuda.current_stream() if stream is None else stream
    buf = torch.empty(min(step, max(n, n_neg, 1)), dtype=torch.int64, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    f = Filter(M, k, c, cost, param, hash_seed=hash_seed, batch=B, bitsel=bitsel, stream=s)
    try:
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(s)
        for start in range(0, n, step):
            cnt = min(step, n - start)
            generate_keys(cnt, key_seed, start, out=buf, stream=s)
            f.insert(buf[:cnt], stream=s)
        e1.record(s)
        for start in range(0, n_neg, buf.numel()):
            cnt = min(buf.numel(), n_neg - start)
            generate_keys(cnt, neg_seed, start, out=buf, stream=s)
            f.query_count(buf[:cnt], count, stream=s)
        e2.record(s)
        e2.synchronize()
        W = int(count.item())
        st = f.stats()
    finally:
        f.close()
    hist = [int(v) for v in st.hist]
    mean = sum(L * h for L, h in enumerate(hist)) / M
    var = sum(h * (L - mean) ** 2 for L, h in enumerate(hist)) / M
    fpr = W / n_neg if n_neg else 0.0
    return dict(n=n, N=n_neg, M=M, k=k, c=c, cost=cost, param=param, bitsel=bitsel, B=B, W=W, fpr=fpr,
                log2_fpr=math.log2(fpr) if W else None, fpr_est=st.fpr_est, inserted=int(st.inserted),
                skipped=int(st.skipped), load_mean=mean, load_sd=math.sqrt(var), hist=hist,
                insert_ms=e0.elapsed_time(e1), query_ms=e1.elapsed_time(e2))


def fig4(n=2 * 10**9, ks=PAPER_KS, rel_sizes=REL_SIZES, choices=(1, 2, 3), bitsels=(0, 1), seed=1, log=None):
    """log2 FPR against relative filter size (Section 4.1, Fig. 4): cost^EXP
    with beta = golden ratio; the standard Bloom formula beside each point."""
    rows = []
    for k in ks:
        for rho in rel_sizes:
            M = blocks_for(n, k, rho)
            for bitsel in bitsels:
                for c in choices:
                    t = time.perf_counter()
                    r = fpr_point(n, M, k, c, 2, PHI, bitsel, key_seed=seed * 1000 + k,
                                  neg_seed=seed * 1000 + 500 + k)
                    r.pop("hist")
                    r.update(rel_size=rho, bloom_fpr=bloom_fpr(n, 512.0 * M, k), wall_s=time.perf_counter() - t)
                    rows.append(r)
                    if log:
                        log(r)
    return rows


def fig10(n=2 * 10**9, ks=PAPER_KS, costs=(0, 1, 2), choices=(2, 3), bitsels=(0, 1), runs=(1, 2, 3), log=None):
    """log2 FPR against the cost parameter of each cost kind at the standard
    Bloom size (Appendix C, Fig. 10); runs differ in keys and hash seeds."""
    rows = []
    for k in ks:
        M = blocks_for(n, k)
        for cost in costs:
            for param in COST_PARAMS[cost]:
                for c in choices:
                    for bitsel in bitsels:
                        for run in runs:
                            r = fpr_point(n, M, k, c, cost, param, bitsel, key_seed=run * 7919 + k,
                                          neg_seed=run * 7919 + 4000 + k)
                            r.pop("hist")
                            r.update(run=run)
                            rows.append(r)
                            if log:
                                log(r)
    return rows


def fig8(n=2 * 10**9, settings=((7, 0, 2.5), (7, 1, 3.5), (7, 2, PHI), (14, 0, 50.0), (14, 1, 3.5), (14, 2, PHI)),
         choices=(1, 2, 3), seed=8, log=None):
    """Load histograms after inserting n keys into a filter of the standard
    Bloom size (Appendix C, Fig. 8) for each (k, cost, parameter) and c."""
    rows = []
    for k, cost, param in settings:
        M = blocks_for(n, k)
        for c in choices:
            r = fpr_point(n, M, k, c, cost, param, 0, key_seed=seed * 100 + k, neg_seed=seed * 100 + 50 + k)
            if log:
                log(r)
            rows.append(r)
    return rows
