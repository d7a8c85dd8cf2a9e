"""The serving loop: every request's result equals the result of running the
requests of its filter alone, one after another, in arrival order (tolerance
0), while waves of requests of different filters share launches and overlap
on several streams; filters beyond the HBM budget wait for admission.

Every served query bitmap and every filter's final words are also compared
with the oracle replaying each filter's requests in arrival order (Sec. 3.1
and 3.2: an insert request is its own sequence of B-key batches; a query sees
exactly the inserts that arrived before it)."""
import numpy as np
import pytest

import workloads
from oracle import OracleFilter, COST_MIX
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


def _small_trace(n_filters=12, n_requests=300, max_keys=20000, seed=7):
    filters, reqs = workloads.serving_config(seed=seed, n_filters=n_filters, n_requests=n_requests,
                                             max_keys=max_keys)
    for f in filters:          # smaller filters for a quick test: 2^16..2^22 bits
        f["M"] = max(1, f["M"] // 512)
        f["B"] = 1 << max(0, (max(f["M"] // 2, 1)).bit_length() - 1)
    return filters, reqs


def _alone(bc, filters, reqs, keys):
    """Each filter's requests through the plain API, in arrival order."""
    import torch
    fs = [bc.Filter(f["M"], 14, 2, bc.COST_MIX, 50.0, hash_seed=f["key_seed"], batch=f["B"])
          for f in filters]
    out = {}
    for r in sorted(reqs, key=lambda r: (r["arrival"], r["index"])):
        f = fs[r["filter"]]
        d = to_dev(keys[r["index"]])
        if r["kind"] == 0:
            f.insert(d)
        else:
            out[r["index"]] = f.query(d).cpu().numpy().view(np.uint64).copy()
    torch.cuda.synchronize()
    words = [f.words_host() for f in fs]
    for f in fs:
        f.close()
    return out, words


def _oracle(filters, reqs, keys):
    """Each filter's requests replayed by the oracle in arrival order."""
    fs = [OracleFilter(f["M"], 14, 2, COST_MIX, 50.0, seed=f["key_seed"], batch=f["B"])
          for f in filters]
    out = {}
    for r in sorted(reqs, key=lambda r: (r["arrival"], r["index"])):
        f = fs[r["filter"]]
        if r["kind"] == 0:
            f.insert(keys[r["index"]])
        else:
            out[r["index"]] = np.asarray(f.query(keys[r["index"]]), dtype=np.uint64)
    return out, [np.asarray(f.words, dtype=np.uint64) for f in fs]


def _check_oracle(filters, reqs, keys, served, served_words):
    want, want_words = _oracle(filters, reqs, keys)
    assert set(want) == set(served)
    for j, bm in want.items():
        assert np.array_equal(served[j], bm), j
    for f, a, b in zip(filters, want_words, served_words):
        assert np.array_equal(a, b), f["index"]


def _serve(bc, filters, reqs, keys, budget=1 << 30, streams=3, wave=8, time_scale=1e-4,
           remove=(), tune=None):
    srv = bc.Server(budget, staging_bytes=64 << 20, streams=streams, max_wave_requests=wave)
    if tune:
        srv.set_tuning(**tune)
    ids = [srv.add_filter(f["M"], 14, 2, bc.COST_MIX, 50.0, f["key_seed"], f["B"]) for f in filters]
    bms = {}
    for r in reqs:
        h = keys[r["index"]]
        bm = np.zeros((r["n"] + 63) // 64, dtype=np.uint64) if r["kind"] == 1 else None
        if bm is not None:
            bms[r["index"]] = bm
        srv.submit(ids[r["filter"]], r["kind"], h, bm, r["arrival"] * time_scale)
    pending_before = srv.stats().filters_pending
    srv.start()
    for fid in remove:
        srv.remove_filter(fid)
    srv.wait(60.0)
    st = srv.stats()
    words = [srv.words_host(i) for i in ids]
    srv.close()
    return bms, words, st, pending_before


def test_served_results_equal_alone_results():
    import paper_2501_18977_gb300 as bc
    filters, reqs = _small_trace()
    keys = {r["index"]: workloads.serving_keys(filters, r, seed=7) for r in reqs}
    alone, alone_words = _alone(bc, filters, reqs, keys)
    served, served_words, st, _ = _serve(bc, filters, reqs, keys)
    assert st.completed == len(reqs)
    assert st.waves >= 1 and st.mean_wave_requests >= 1.0
    assert st.p50_latency_s <= st.p99_latency_s <= st.max_latency_s
    for j, bm in alone.items():
        assert np.array_equal(served[j], bm), j
    for a, b in zip(alone_words, served_words):
        assert np.array_equal(a, b)
    _check_oracle(filters, reqs, keys, served, served_words)


@pytest.mark.parametrize("tune", [dict(cluster_max=0, lanes_choose=4, lanes_query=1),
                                  dict(cluster_max=16, lanes_cluster=4, cluster_keys=16, lanes_query=4),
                                  dict(cluster_max=2, lanes_cluster=8, query_early=0, ctas_per_sm=3)])
def test_server_launch_configuration_keeps_results(tune):
    """A server-wide launch configuration (filters and many-filter calls)
    changes no result; it is refused once the server runs."""
    import paper_2501_18977_gb300 as bc
    filters, reqs = _small_trace(n_filters=8, n_requests=150, seed=10)
    keys = {r["index"]: workloads.serving_keys(filters, r, seed=10) for r in reqs}
    alone, alone_words = _alone(bc, filters, reqs, keys)
    served, served_words, st, _ = _serve(bc, filters, reqs, keys, time_scale=0.0, tune=tune)
    assert st.completed == len(reqs)
    for j, bm in alone.items():
        assert np.array_equal(served[j], bm), j
    for a, b in zip(alone_words, served_words):
        assert np.array_equal(a, b)
    _check_oracle(filters, reqs, keys, served, served_words)
    srv = bc.Server(1 << 24, staging_bytes=1 << 20, streams=1, max_wave_requests=1)
    try:
        with pytest.raises(bc.BlowChocError):
            srv.set_tuning(lanes_cluster=2)
        srv.start()
        with pytest.raises(bc.BlowChocError):
            srv.set_tuning(**tune)
    finally:
        srv.close()


def test_concurrent_waves_share_launches():
    """With all requests arriving at once, waves carry many filters' requests."""
    import paper_2501_18977_gb300 as bc
    filters, reqs = _small_trace(n_filters=16, n_requests=200, seed=8)
    keys = {r["index"]: workloads.serving_keys(filters, r, seed=8) for r in reqs}
    alone, _ = _alone(bc, filters, reqs, keys)
    served, served_words, st, _ = _serve(bc, filters, reqs, keys, time_scale=0.0, wave=16, streams=4)
    assert st.mean_wave_requests > 2.0
    for j, bm in alone.items():
        assert np.array_equal(served[j], bm), j
    _check_oracle(filters, reqs, keys, served, served_words)


def test_admission_waits_for_budget():
    import paper_2501_18977_gb300 as bc
    filters, reqs = _small_trace(n_filters=4, n_requests=80, seed=9)
    for f in filters:
        f["M"], f["B"] = 4096, 2048
    one = 4096 * 64 + 513 * 15 * 2 + 520 * 8
    keys = {r["index"]: workloads.serving_keys(filters, r, seed=9) for r in reqs}
    alone, _ = _alone(bc, filters, reqs, keys)
    served, _, st, pending = _serve(bc, filters, reqs, keys, budget=int(2.5 * one), remove=(0, 1))
    assert pending == 2
    assert st.completed == len(reqs)
    assert st.max_filter_bytes_used <= int(2.5 * one)
    for j, bm in alone.items():
        assert np.array_equal(served[j], bm), j
    want, _ = _oracle(filters, reqs, keys)
    for j, bm in want.items():
        assert np.array_equal(served[j], bm), j


def test_server_rejects_what_cannot_fit():
    import paper_2501_18977_gb300 as bc
    srv = bc.Server(1 << 20, staging_bytes=1 << 16, streams=1, max_wave_requests=1)
    try:
        with pytest.raises(bc.BlowChocError) as ei:
            srv.add_filter(1 << 20, 14, 2, bc.COST_MIX, 50.0, 1, 1024)
        assert ei.value.code == bc.BLOWCHOC_EBUDGET
        fid = srv.add_filter(64, 14, 2, bc.COST_MIX, 50.0, 1, 1024)
        big = workloads.uniform_keys(1, 1 << 14)
        with pytest.raises(bc.BlowChocError) as ei:
            srv.submit(fid, bc.REQ_INSERT, big)
        assert ei.value.code == bc.BLOWCHOC_EBUDGET
        with pytest.raises(bc.BlowChocError):
            srv.submit(fid, 7, big[:10])
    finally:
        srv.close()


def test_runs_of_queries_share_a_launch_and_keep_exact_bitmaps():
    """All requests arrive at once; a filter's consecutive queries (odd
    sizes, so each is padded inside the shared launch item) share a launch,
    every bitmap equals the oracle's, and the bits past each request's last
    key are zero."""
    import paper_2501_18977_gb300 as bc
    M, B = 4096, 2048
    seed = 3
    keys_ins = workloads.uniform_keys(31, 50000)
    reqs, keys = [], {}
    # filter 0: one insert, then a run of 40 queries of odd sizes; filter 1 the same shape
    for f in range(2):
        j = len(reqs)
        reqs.append(dict(index=j, arrival=0.0, kind=0, filter=f, n=len(keys_ins)))
        keys[j] = keys_ins
        for q in range(40):
            j = len(reqs)
            n = 1 + 37 * q
            qk = np.concatenate([keys_ins[q * 100: q * 100 + n // 2], workloads.uniform_keys(700 + j, n - n // 2)])
            reqs.append(dict(index=j, arrival=0.0, kind=1, filter=f, n=n))
            keys[j] = qk
    filters = [dict(index=f, M=M, B=B, key_seed=seed + f) for f in range(2)]
    served, served_words, st, _ = _serve(bc, filters, reqs, keys, time_scale=0.0, wave=64, streams=2)
    assert st.completed == len(reqs)
    assert st.mean_wave_requests > 2.0
    _check_oracle(filters, reqs, keys, served, served_words)
    for r in reqs:
        if r["kind"] == 1 and r["n"] % 64:
            assert int(served[r["index"]][-1]) >> (r["n"] % 64) == 0, r["index"]
