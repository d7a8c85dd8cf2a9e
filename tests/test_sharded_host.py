"""Sub-array sharding (Section 3.4) across ranks, on the CPU.

One rank per sub-array: each rank partitions its own keys by h_0, the
library's exchange (paper_2501_18977_gb300.sharded: insert_routed,
query_routed) sends every sub-array's keys to its owner and the answers
back. Ranks here are gloo processes on the CPU, and each owner's insert and
query are the oracle's sub-array; the result must equal the oracle's split
filter fed with all ranks' keys, rank 0's first. The sub-array layout the
library derives (a_0, sub-array size, sub-array seed) must equal the
oracle's. The GPU kernels of the same path (partition, unpermute) are
checked in tests/test_gpu_sharded.py.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads
from oracle.oracle import COST_LA, COST_EXP, GOLDEN_RATIO, OracleFilter, derive_multipliers
from oracle.sharded import ShardedOracle, shard_layout

CASES = [  # (M, k, c, cost, param, B, keys per rank)
    (300, 9, 2, COST_EXP, GOLDEN_RATIO, 64, 4000),
    (1000, 12, 3, COST_LA, 3.5, 1, 1500),
]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_keys(rank, n):
    return workloads.uniform_keys(700 + rank, n)


def _rank_main(rank, world, port, case, out):
    import torch
    import torch.distributed as dist
    from paper_2501_18977_gb300 import sharded
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        M, k, c, kind, par, B, n = case
        ref = ShardedOracle(M, world, k, c, kind, par, seed=17, batch=B)
        a0, Ms, sub_seed = shard_layout(M, world, 17)
        a_block, a_bit = derive_multipliers(sub_seed, Ms, k, c)
        mine = OracleFilter(Ms, k, c, kind, par, batch=B, a_block=a_block, a_bit=a_bit)
        keys = _rank_keys(rank, n)
        # this rank's keys by sub-array, each in input order (what the
        # partition kernel computes on a GPU)
        sh = ref.shard_of(keys)
        order = np.argsort(sh, kind="stable")
        counts = np.bincount(sh, minlength=world).tolist()
        part = torch.from_numpy(keys[order].view(np.int64).copy())

        def local_insert(d):
            mine.insert(d.numpy().view(np.uint64))

        def local_query(d, out_words):
            bm = mine.query(d.numpy().view(np.uint64))
            out_words.copy_(torch.from_numpy(bm.view(np.int64)[: out_words.numel()]))

        sharded.insert_routed(part, counts, local_insert, None)
        dist.barrier()
        queries = np.concatenate([keys[: n // 2], workloads.uniform_keys(900 + rank, n // 2)])
        qsh = ref.shard_of(queries)
        qorder = np.argsort(qsh, kind="stable")
        qcounts = np.bincount(qsh, minlength=world).tolist()
        seg = sharded.query_routed(torch.from_numpy(queries[qorder].view(np.int64).copy()), qcounts,
                                   local_query, None)
        # answers back in input order
        hit = np.zeros(len(queries), dtype=bool)
        wpos = kpos = 0
        segw = seg.numpy().view(np.uint64)
        for t in range(world):
            bits = np.unpackbits(segw[wpos:wpos + (qcounts[t] + 63) // 64].view(np.uint8),
                                 bitorder="little")[: qcounts[t]].astype(bool)
            hit[qorder[kpos:kpos + qcounts[t]]] = bits
            wpos += (qcounts[t] + 63) // 64
            kpos += qcounts[t]
        out.put((rank, mine.words.copy(), hit, mine.inserted, mine.skipped))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", CASES, ids=["c2-exp-B64", "c3-la-B1"])
def test_ranks_build_the_split_filter_of_all_keys(world, case):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, case, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted([out.get(timeout=180) for _ in procs], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    M, k, c, kind, par, B, n = case
    ref = ShardedOracle(M, world, k, c, kind, par, seed=17, batch=B)
    ref.insert(np.concatenate([_rank_keys(r, n) for r in range(world)]))
    for rank, words, hit, ins, skp in results:
        assert np.array_equal(words, ref.subs[rank].words), rank
        assert (ins, skp) == (ref.subs[rank].inserted, ref.subs[rank].skipped)
        keys = _rank_keys(rank, n)
        queries = np.concatenate([keys[: n // 2], workloads.uniform_keys(900 + rank, n // 2)])
        want = np.unpackbits(ref.query(queries).view(np.uint8), bitorder="little")[: len(queries)].astype(bool)
        assert np.array_equal(hit, want), rank
        assert hit[: n // 2].all()


@pytest.mark.parametrize("M,T,seed", [(1, 1, 5), (1000, 1, 7), (1 << 21, 2, 3), (999, 3, 11), (64, 6, 12345),
                                      (1 << 30, 1024, 2**64 - 1)])
def test_layout_equals_the_oracle(M, T, seed):
    import paper_2501_18977_gb300 as bc
    assert bc.blowchoc_shard_layout(M, T, seed) == shard_layout(M, T, seed)


def test_layout_rejects_bad_arguments():
    import paper_2501_18977_gb300 as bc
    for args in [(0, 2, 1), (10, 0, 1), (10, 1025, 1)]:
        with pytest.raises(bc.BlowChocError):
            bc.blowchoc_shard_layout(*args)
