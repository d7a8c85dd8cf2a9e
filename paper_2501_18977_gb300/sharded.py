"""Filters split into sub-arrays (Section 3.4, parallelization), all on one
GPU or one sub-array per GPU rank.

A filter of M blocks becomes T sub-arrays of ceil(M / T) blocks, and h_0
routes each key to one (blowchoc_shard_layout). With `group=None` the T
sub-arrays live on the current GPU. With a torch.distributed process group of
T ranks, rank t owns sub-array t: an insert partitions the rank's keys by h_0
and sends each sub-array's keys to its owner with one all-to-all; a query
does the same and returns the owners' answers with a second all-to-all of
bitmap words. A sub-array receives its keys in the order of the ranks'
arrays, so the result equals inserting the concatenation of all ranks' keys
(rank 0 first) into the split filter. Every step on the data runs in the
library's kernels (partition by h_0, insert, query, unpermute); this module
only moves tensors between them.
"""
from . import binding as _b


def words_for(counts):
    """Bitmap words of segments of `counts` keys each."""
    return [(int(c) + 63) // 64 for c in counts]


def exchange_keys(part_keys, counts, group):
    """All-to-all of keys partitioned by sub-array: counts[t] keys of
    part_keys (in order of t) go to rank t. Returns (received keys, one
    segment per source rank in rank order; received count per source)."""
    import torch
    import torch.distributed as dist
    if len(counts) != dist.get_world_size(group) or sum(int(c) for c in counts) != part_keys.numel():
        raise ValueError("one count per rank, summing to the number of partitioned keys")
    send = torch.tensor([int(c) for c in counts], dtype=torch.int64, device=part_keys.device)
    recv = torch.empty_like(send)
    dist.all_to_all_single(recv, send, group=group)
    rc = [int(v) for v in recv.cpu()]
    out = torch.empty(sum(rc), dtype=part_keys.dtype, device=part_keys.device)
    dist.all_to_all_single(out, part_keys, output_split_sizes=rc, input_split_sizes=[int(c) for c in counts],
                           group=group)
    return out, rc


def insert_routed(part_keys, counts, local_insert, group):
    """Sends each sub-array's keys to its owner and inserts what arrives at
    this rank with local_insert(keys)."""
    recv, _ = exchange_keys(part_keys, counts, group)
    if recv.numel():
        local_insert(recv)


def query_routed(part_keys, counts, local_query, group):
    """Sends each sub-array's keys to its owner; the owner answers every
    source's segment with local_query(keys, out_words) into a bitmap of
    ceil(count / 64) words, and the answers come back. Returns this rank's
    answers: per sub-array t, ceil(counts[t] / 64) words, in order of t."""
    import torch
    import torch.distributed as dist
    recv, rc = exchange_keys(part_keys, counts, group)
    rw = words_for(rc)
    answers = torch.zeros(sum(rw), dtype=torch.int64, device=part_keys.device)
    kpos = wpos = 0
    for c, w in zip(rc, rw):
        if c:
            local_query(recv[kpos:kpos + c], answers[wpos:wpos + w])
        kpos += c
        wpos += w
    mine = words_for(counts)
    out = torch.zeros(sum(mine), dtype=torch.int64, device=part_keys.device)
    dist.all_to_all_single(out, answers, output_split_sizes=mine, input_split_sizes=rw, group=group)
    return out


class ShardedFilter:
    """A filter of M blocks split into T sub-arrays (Section 3.4). Keys and
    bitmaps are int64 CUDA tensors; with a process group, each rank passes
    its own keys and receives the answers for them."""

    def __init__(self, M, T, k, c, cost=_b.COST_EXP, cost_param=(1 + 5 ** 0.5) / 2, hash_seed=0, batch=1,
                 bitsel=0, group=None):
        self.T = int(T)
        self.a0, self.Ms, self.sub_seed = _b.blowchoc_shard_layout(M, T, hash_seed)
        self.group = group
        if group is None:
            owned = range(self.T)
        else:
            import torch.distributed as dist
            if dist.get_world_size(group) != self.T:
                raise ValueError("one rank per sub-array: the group must have T ranks")
            owned = [dist.get_rank(group)]
        self.subs = {t: _b.Filter(self.Ms, k, c, cost, cost_param, hash_seed=self.sub_seed, batch=batch,
                                  bitsel=bitsel) for t in owned}

    def partition(self, keys, stream=None):
        """(keys by sub-array, their input indices, device offsets, host offsets)."""
        import torch
        n = keys.numel()
        out_keys = torch.empty_like(keys)
        out_index = torch.empty(n, dtype=torch.int64, device=keys.device)
        offsets = torch.empty(self.T + 1, dtype=torch.int64, device=keys.device)
        sw = _b.blowchoc_shard_partition_scratch(n, self.T)
        scratch = torch.empty(max(sw, 1), dtype=torch.int64, device=keys.device)
        _b.blowchoc_shard_partition(keys, n, self.T, self.a0, out_keys, out_index, offsets, scratch, sw, stream)
        return out_keys, out_index, offsets, [int(v) for v in offsets.cpu()]

    def insert(self, keys, stream=None):
        part, _, _, off = self.partition(keys, stream)
        counts = [off[t + 1] - off[t] for t in range(self.T)]
        if self.group is None:
            for t in range(self.T):
                if counts[t]:
                    self.subs[t].insert(part[off[t]:off[t + 1]], stream)
            return
        (t,) = self.subs
        insert_routed(part, counts, lambda d: self.subs[t].insert(d, stream), self.group)

    def query(self, keys, bitmap=None, stream=None):
        """LSB-first bitmap of ceil(n / 64) words for `keys`, in their order."""
        import torch
        n = keys.numel()
        if bitmap is None:
            bitmap = torch.empty(max((n + 63) // 64, 1), dtype=torch.int64, device=keys.device)
        if n == 0:
            return bitmap
        part, index, offsets, off = self.partition(keys, stream)
        counts = [off[t + 1] - off[t] for t in range(self.T)]
        if self.group is None:
            wc = words_for(counts)
            seg = torch.zeros(max(sum(wc), 1), dtype=torch.int64, device=keys.device)
            wpos = 0
            for t in range(self.T):
                if counts[t]:
                    self.subs[t].query(part[off[t]:off[t + 1]], seg[wpos:wpos + wc[t]], stream)
                wpos += wc[t]
        else:
            (t,) = self.subs
            seg = query_routed(part, counts, lambda d, out: self.subs[t].query(d, out, stream), self.group)
        _b.blowchoc_shard_unpermute(seg, offsets, index, n, self.T, bitmap, stream)
        return bitmap

    def words_host(self):
        """Words of the sub-arrays this process holds, in order of t."""
        import numpy as np
        return np.concatenate([self.subs[t].words_host() for t in sorted(self.subs)])

    def close(self):
        for f in self.subs.values():
            f.close()
        self.subs = {}
