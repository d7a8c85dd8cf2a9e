"""blowchoc_insert_noalloc against blowchoc_insert, through the C ABI.

The no-allocation variant exists for callers that cannot let the library
allocate device memory at insert time (their memory is handed out by their
own allocator or budget, or they run latency-critical loops where an
allocation may synchronise the device). Its filter words and counters must
equal those of the regular entry point, exactly, over two calls in a row on
the same filter (the second call reuses the shared fixed scratch array).
"""
import numpy as np
import pytest

import workloads
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


def _two_calls(bc, noalloc, M, k, c, cost, par, B, a, b):
    f = bc.Filter(M, k, c, cost, par, hash_seed=77, batch=B)
    try:
        ins = bc.blowchoc_insert_noalloc if noalloc else bc.blowchoc_insert
        ins(f.handle, a, a.numel())
        ins(f.handle, b, b.numel())
        words = f.words_host()
        st = f.stats()
        return words, (st.inserted, st.skipped)
    finally:
        f.close()


@pytest.mark.parametrize("M,k,c,cost,par,B", [
    (2048, 16, 3, 1, 3.5, 100000),      # choices in the fixed array
    (999, 11, 2, 2, 1.6180339887498949, 1 << 22),  # batch at the limit
    (4096, 10, 1, 0, 50.0, 100000),     # one choice on the fixed array
    (3000, 12, 2, 1, 3.5, 8192),        # over the single-CTA limit: fixed array
    (5000, 13, 3, 2, 1.6180339887498949, 1 << 24),  # B over the limit, n under it
    (512, 14, 2, 0, 50.0, 1000),        # single-CTA kernel, no scratch
    (256, 12, 2, 0, 50.0, 1),           # sequential, no scratch
])
def test_noalloc_matches_insert(M, k, c, cost, par, B):
    import torch
    import paper_2501_18977_gb300 as bc
    n1, n2 = (250000, 170001) if B > 1 else (20000, 7001)
    if B == 1 << 22:
        n1 = B                          # one full batch at the limit
    if B == 1 << 24:
        n1, n2 = 1000000, 300001        # min(B, n) fits: accepted
    a = to_dev(workloads.uniform_keys(M + 1, n1))
    b = to_dev(workloads.uniform_keys(M + 2, n2))
    torch.cuda.synchronize()
    want_words, want_counts = _two_calls(bc, False, M, k, c, cost, par, B, a, b)
    got_words, got_counts = _two_calls(bc, True, M, k, c, cost, par, B, a, b)
    assert np.array_equal(got_words, want_words)
    assert got_counts == want_counts


def test_noalloc_rejects_batches_over_the_limit():
    import paper_2501_18977_gb300 as bc
    n = (1 << 22) + 1
    keys = to_dev(workloads.uniform_keys(3, n))
    f = bc.Filter(1024, 8, 2, bc.COST_MIX, 50.0, hash_seed=1, batch=n)
    try:
        with pytest.raises(bc.BlowChocError) as ei:
            bc.blowchoc_insert_noalloc(f.handle, keys, n)
        assert ei.value.code == bc.BLOWCHOC_EINVAL
        assert "4194304" in bc.blowchoc_last_error()
        assert not f.words_host().any()          # nothing was launched
    finally:
        f.close()


def test_noalloc_leaves_device_memory_unchanged():
    """A large batch that the regular path would back with a freshly
    allocated 3 MB choice buffer runs without changing free device memory."""
    import torch
    import paper_2501_18977_gb300 as bc
    n = 3 * (1 << 20)
    keys = to_dev(workloads.uniform_keys(5, n))
    f = bc.Filter(1 << 16, 12, 2, bc.COST_EXP, 1.6180339887498949, hash_seed=5, batch=n)
    try:
        bc.blowchoc_insert_noalloc(f.handle, keys, n)   # first call: per-device set-up
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        bc.blowchoc_insert_noalloc(f.handle, keys, n)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] >= free0
    finally:
        f.close()
