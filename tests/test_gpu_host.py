"""Insert and query from host buffers (blowchoc_insert_host /
blowchoc_query_host) give exactly what the device-buffer calls give: the
chunked copies through the staging ring keep every batch edge, and the bitmap
layout is the same, for pinned and pageable memory, ragged lengths, batch
sizes that do not divide the chunk and a batch larger than the chunk. The
results are also the oracle's."""
import numpy as np
import pytest

import workloads
from oracle import COST_MIX, COST_EXP, OracleFilter
from oracle.oracle import GOLDEN_RATIO
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


def _host(a, pinned):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a).view(np.int64))
    return t.pin_memory() if pinned else a


@pytest.mark.parametrize("M,k,c,B,n,pinned", [
    (4096, 14, 2, 65536, 1000003, True),      # several chunks of whole batches
    (3000, 12, 3, 1000, 5000001, True),       # B not dividing the chunk sizes: 1,048,000 keys first
    (777, 9, 2, 1, 200001, False),            # one key at a time, pageable memory
    (8192, 16, 3, 5 << 20, 12 << 20, True),   # one batch larger than the first chunks
    (100, 7, 1, 64, 63, False),               # fewer keys than a bitmap word
])
def test_host_buffers_equal_device_buffers(M, k, c, B, n, pinned):
    import torch
    import paper_2501_18977_gb300 as bc
    keys = workloads.uniform_keys(M + n, n)
    queries = np.concatenate([keys[: n // 2], workloads.uniform_keys(M + n + 1, n // 2 + 7)])
    a = bc.Filter(M, k, c, COST_EXP, GOLDEN_RATIO, hash_seed=5, batch=B)
    b = bc.Filter(M, k, c, COST_EXP, GOLDEN_RATIO, hash_seed=5, batch=B)
    try:
        s = torch.cuda.current_stream()
        hk, hq = _host(keys, pinned), _host(queries, pinned)
        a.insert_host(hk, s)
        bm_host = a.query_host(hq, stream=s)
        s.synchronize()
        b.insert(to_dev(keys))
        bm_dev = b.query(to_dev(queries)).cpu().numpy().view(np.uint64)
        assert np.array_equal(a.words_host(), b.words_host())
        assert np.array_equal(bm_host[: len(bm_dev)], bm_dev)
        sa, sb = a.stats(), b.stats()
        assert (sa.inserted, sa.skipped) == (sb.inserted, sb.skipped)
    finally:
        a.close()
        b.close()
    if n <= 300000:
        o = OracleFilter(M, k, c, COST_EXP, GOLDEN_RATIO, seed=5, batch=B)
        o.insert(keys)
        assert np.array_equal(bm_host[: (len(queries) + 63) // 64], o.query(queries))


def test_host_calls_reuse_staging_across_calls_and_streams():
    """Back-to-back host calls on two streams of one filter, with the caller
    ordering the streams, build the same filter as one device call."""
    import torch
    import paper_2501_18977_gb300 as bc
    M, k, c, B = 2048, 14, 2, 4096
    keys = workloads.uniform_keys(99, 3000000)
    f = bc.Filter(M, k, c, COST_MIX, 50.0, hash_seed=1, batch=B)
    g = bc.Filter(M, k, c, COST_MIX, 50.0, hash_seed=1, batch=B)
    try:
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        h = _host(keys, True)
        f.insert_host(h[:1000000], s1)
        s2.wait_stream(s1)
        f.insert_host(h[1000000:], s2)
        s2.synchronize()
        g.insert(to_dev(keys[:1000000]))
        g.insert(to_dev(keys[1000000:]))
        assert np.array_equal(f.words_host(), g.words_host())
    finally:
        f.close()
        g.close()


def test_staging_ring_wraps_within_and_across_calls():
    """A ring of 2^18 keys (chunks of at most 2^16): one call of 5 M keys
    wraps it 19 times, then alternating small insert and query calls wrap it
    again across calls. Words and every bitmap equal the device calls'."""
    import torch
    import paper_2501_18977_gb300 as bc
    M, k, c, B = 1 << 16, 12, 2, 1 << 16
    big = workloads.uniform_keys(123, 5_000_000)
    a = bc.Filter(M, k, c, COST_EXP, GOLDEN_RATIO, hash_seed=9, batch=B)
    b = bc.Filter(M, k, c, COST_EXP, GOLDEN_RATIO, hash_seed=9, batch=B)
    try:
        a.set_tuning(host_ring_keys=1 << 18)
        s = torch.cuda.current_stream()
        hb = _host(big, True)
        a.insert_host(hb, s)
        b.insert(to_dev(big))
        small_bms, alive = [], []   # pinned buffers stay alive until the stream completes
        for j in range(40):
            ks = workloads.uniform_keys(1000 + j, 30000 + 17 * j)
            qs = workloads.uniform_keys(2000 + j, 20000 + 29 * j)
            hk, hq = _host(ks, True), _host(qs, True)
            alive += [hk, hq]
            a.insert_host(hk, s)
            small_bms.append((a.query_host(hq, stream=s), qs))
            b.insert(to_dev(ks))
        s.synchronize()
        assert np.array_equal(a.words_host(), b.words_host())
        # the queries saw the filter after their own call's inserts: replay on b's prefix
        c2 = bc.Filter(M, k, c, COST_EXP, GOLDEN_RATIO, hash_seed=9, batch=B)
        try:
            c2.insert(to_dev(big))
            for j, (bm, qs) in enumerate(small_bms):
                ks = workloads.uniform_keys(1000 + j, 30000 + 17 * j)
                c2.insert(to_dev(ks))
                want = c2.query(to_dev(qs)).cpu().numpy().view(np.uint64)
                assert np.array_equal(bm[: len(want)], want), j
        finally:
            c2.close()
    finally:
        a.close()
        b.close()


def test_more_pending_chunks_than_event_sets():
    """A ring of 2^16 keys grown by a first call of 60,000 keys, then 300
    calls of 100 keys (B = 64): about 500 chunks fit in the ring, more than
    the staging's 64 event sets, so the oldest pending chunks are retired
    before their space comes round again. Results equal the device calls',
    on two alternating caller streams."""
    import torch
    import paper_2501_18977_gb300 as bc
    M, k, c, B = 1024, 10, 3, 64
    a = bc.Filter(M, k, c, COST_EXP, GOLDEN_RATIO, hash_seed=4, batch=B)
    b = bc.Filter(M, k, c, COST_EXP, GOLDEN_RATIO, hash_seed=4, batch=B)
    try:
        a.set_tuning(host_ring_keys=1 << 16)
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        first = workloads.uniform_keys(77, 60000)
        h0 = _host(first, True)
        a.insert_host(h0, s1)
        b.insert(to_dev(first))
        alive, got, want = [h0], [], []
        for j in range(300):
            st, other = (s1, s2) if j % 2 == 0 else (s2, s1)
            st.wait_stream(other)   # the caller orders its streams; the staging orders the ring
            ks = workloads.uniform_keys(5000 + j, 100)
            hk = _host(ks, True)
            alive.append(hk)
            a.insert_host(hk, st)
            b.insert(to_dev(ks))
            if j % 10 == 9:
                qs = workloads.uniform_keys(9000 + j, 100)
                hq = _host(qs, True)
                alive.append(hq)
                got.append(a.query_host(hq, stream=st))
                want.append(b.query(to_dev(qs)).cpu().numpy().view(np.uint64))
        torch.cuda.synchronize()
        assert np.array_equal(a.words_host(), b.words_host())
        for g, w in zip(got, want):
            assert np.array_equal(g[: len(w)], w)
        sa, sb = a.stats(), b.stats()
        assert (sa.inserted, sa.skipped) == (sb.inserted, sb.skipped)
    finally:
        a.close()
        b.close()


def test_host_ring_keys_is_checked():
    import paper_2501_18977_gb300 as bc
    f = bc.Filter(256, 8, 2, COST_EXP, GOLDEN_RATIO, hash_seed=1, batch=64)
    try:
        for bad in (1, 1000, (1 << 16) - 1, 1 << 31):
            with pytest.raises(Exception):
                f.set_tuning(host_ring_keys=bad)
        f.set_tuning(host_ring_keys=(1 << 16) + 5)
        assert f.tuning().host_ring_keys == (1 << 16) + 5
        f.set_tuning(host_ring_keys=0)
    finally:
        f.close()
