#!/usr/bin/env python3
"""Benchmark of the BlowChoc filter hot path on one GB300 (or N replicas).

Workload (the DNA k-mer configuration): a 50,000,000-base uniform random
genome (splitmix64 seed 2, 2 bits per base) gives 49,999,970 canonical
31-mers, inserted with B = 2^20 into a filter of 2^30 bits (M = 2^21 blocks,
128 MiB), k = 16, three choices, cost^LA with mu = 3.5; the query set is the
same 31-mers followed by 49,999,970 31-mers of an independent genome (seed 3).

One step = clear the filter, insert all keys, query all query keys, read the
load statistics: every row of the hot path over one batch of input. The
metric is keys processed (inserted + queried) per second, in Mkeys/s.

--impl reference runs the CPU oracle (plain single-threaded C) on a bounded
sample of the same workload, as the reference arm.

Other measurements (--workload): `gather` sweeps the random 64-byte gather
ceiling of the device over footprints from 2 MiB to 4 GiB; `many` runs 256
independent filters of lognormal sizes (k = 11, c = 2, cost^EXP) as plain
per-filter calls, as one launch per phase over a work list, and as a replayed
CUDA graph, and checks that all three give the same words and bitmaps;
`serve` runs the request-serving loop on 64 filters under a Poisson stream of
10,000 insert/query requests at 50/80/95% of its measured capacity; `sweep`
grows 512 MiB filters (k = 12; one choice, and two and three choices under
each cost) from 20 to 6 bits per key against 10^8 negatives per point;
`batching` reports the FPR and load-balance cost of batch size B against
one-key-at-a-time insertion; `small` times the small uniform configuration
(10^6 keys into 2^24 bits, k = 14, two choices, cost^MIX, B = 65536 and 1);
`learn` trains the learned cost on the small configuration's shape and
compares its greedy filter with cost^EXP and cost^MIX on held-out keys;
`fig4`, `fig8` and `fig10` run the paper's FPR-against-size, load-histogram
and cost-parameter sweeps at 2*10^9 keys per point (`--keys` scales them),
with keys generated on the device; `cluster` compares cluster-resident with
global-memory inserts on serving-sized filters; `lanes` times the persistent
insert with 1, 2, 4 and 8 lanes per key for filters of 2 MiB to 512 MiB (the
measurements behind the default lanes per filter size); `variants` times the
sort-by-block set against the direct set, and distinct against random bit
selection.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

CONFIG = dict(workload="dna_kmer_31_c3_la", genome_bases=50_000_000, q=31, genome_seed=2,
              other_genome_seed=3, nblocks=1 << 21, filter_bits=1 << 30, k=16, choices=3,
              cost="LA", mu=3.5, batch=1 << 20, hash_seed=2)
N_KEYS = CONFIG["genome_bases"] - CONFIG["q"] + 1
COST_LA = 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=["dna", "gather", "many", "serve", "sweep", "batching", "small",
                                           "learn", "fig4", "fig8", "fig10", "cluster", "lanes", "variants",
                                           "hbm", "shard"],
                    default="dna")
    ap.add_argument("--keys", type=float, default=2e9, help="fig4/fig8/fig10: keys inserted and negatives")
    ap.add_argument("--ks", type=str, default="4,7,10,14,17,20", help="fig4/fig10: k values")
    ap.add_argument("--runs", type=int, default=1, help="fig10: repetitions with other seeds")
    ap.add_argument("--train-steps", type=int, default=400)
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--reps", type=int, default=3, help="hbm: timed passes after one untimed pass")
    ap.add_argument("--no-extra-records", action="store_true",
                    help="leave the gather ceilings and the hbm_resident record out of the DNA line")
    return ap.parse_args()


def make_workload():
    g1 = workloads.random_genome(CONFIG["genome_seed"], CONFIG["genome_bases"])
    keys = workloads.canonical_kmers(g1, CONFIG["q"])
    del g1
    g2 = workloads.random_genome(CONFIG["other_genome_seed"], CONFIG["genome_bases"])
    other = workloads.canonical_kmers(g2, CONFIG["q"])
    del g2
    queries = np.concatenate([keys, other])
    return keys, queries


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value, world, device):
    """The largest `value` over the job's ranks (the slowest replica's step
    time); `value` itself with one rank."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mkeys_per_s(keys_per_rank, world, ms_per_step):
    """Whole-job throughput: every rank's keys over the slowest rank's step."""
    return world * keys_per_rank / (ms_per_step / 1e3) / 1e6


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    count = 0

    def __init__(self, index):
        self.index = index
        self.proc = None
        ClockSampler.count += 1  # unique file per sampler: several may run at once
        self.path = os.path.join("/tmp", "bc_clocks_%d_%d_%d.csv" % (os.getpid(), index, ClockSampler.count))

    def start(self, settle_s=0.0):
        """Starts sampling; with settle_s > 0, waits (up to settle_s) until the
        first sample is written, so that nvidia-smi's start-up, which takes
        the driver's locks, is over before the caller's timed work begins."""
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t0 = time.perf_counter()
        while settle_s > 0 and time.perf_counter() - t0 < settle_s and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                time.sleep(0.1)  # a second sample's worth, for the process to settle
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, busy, smax, reasons = [], [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                try:  # samples with the GPU busy (utilization over the last interval)
                    if len(parts) > 9 and float(parts[9]) >= 50.0:
                        busy.append(sm[-1])
                except ValueError:
                    pass
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        # the median under load: over the samples with the GPU busy; a workload
        # too short for any sample to see it busy reports the highest clock seen
        return {"sm_mhz": statistics.median(busy) if busy else max(sm), "sm_max_mhz": smax,
                "sm_mhz_basis": "median of busy samples" if busy else "highest sample (no busy sample)",
                "reasons": sorted(reasons), "samples": len(sm), "samples_busy": len(busy),
                "sm_mhz_all_samples": statistics.median(sm)}


# Clock record of a --workload run: every JSON line a workload prints carries
# the SM clocks and throttle reasons sampled since the previous line.
_WORKLOAD_CLOCKS = None


def finite(obj):
    """obj with every non-finite float replaced by None (strict JSON has no NaN)."""
    if isinstance(obj, float):
        return obj if math.isfinite(obj) else None
    if isinstance(obj, dict):
        return {k: finite(v) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [finite(v) for v in obj]
    return obj


def emit(record):
    """Print one workload JSON line with the clocks sampled since the last one."""
    global _WORKLOAD_CLOCKS
    if _WORKLOAD_CLOCKS is not None and "clocks" not in record:
        record = dict(record, clocks=_WORKLOAD_CLOCKS.stop())
        _WORKLOAD_CLOCKS = ClockSampler(_WORKLOAD_CLOCKS.index)
        _WORKLOAD_CLOCKS.start()
    print(json.dumps(finite(record), allow_nan=False), flush=True)


def ratio(a, b, nd=4):
    """round(a / b, nd), or None where b was not measured."""
    return None if b is None or not b else round(a / b, nd)


def rounded(v, nd):
    return None if v is None else round(v, nd)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# sources that define each profiled kernel, and the launch-configuration
# fields that select its instance and grid
KERNEL_SOURCES = {
    "persistent_insert_kernel": ["bc_insert.cu", "bc_phases.cuh", "bc_device.cuh", "bc_launch.h"],
    "query_kernel": ["bc_query.cu", "bc_phases.cuh", "bc_device.cuh", "bc_launch.h"],
}
KERNEL_LAUNCH_FIELDS = {
    "persistent_insert_kernel": ["lanes_choose", "ctas_per_sm", "keys_per_cta", "persistent", "set_mode"],
    "query_kernel": ["lanes_query", "query_early", "ctas_per_sm"],
}


def launch_config(tuning, kernel):
    return {k: int(getattr(tuning, k)) for k in KERNEL_LAUNCH_FIELDS[kernel]}


def sources_sha256(names):
    import hashlib
    h = hashlib.sha256()
    for name in names:
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_2501_18977_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(kernel, tuning):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, or
    None if the kernel's sources or its launch configuration (`tuning`'s
    fields that choose the instance and grid) differ from the capture's."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh).get("kernels", {})
    if kernel not in d or kernel not in KERNEL_SOURCES:
        return None
    if d[kernel].get("sources_sha256") != sources_sha256(KERNEL_SOURCES[kernel]):
        return None
    if d[kernel].get("launch") != launch_config(tuning, kernel):
        return None
    return d[kernel]["dram_bytes_per_launch"]


def gather_ceiling(bc, torch, nblocks, words=None, nreads=50_000_000, grid=None):
    """Random whole-block read rate (GB/s of 64-byte blocks) over `nblocks`
    blocks with the library's gather probe: the best over lanes per block,
    CTAs per SM and independent loads in flight per lane group (each the best
    of 3 timed runs after one untimed). Returns (GB/s, (lanes, ctas/SM, in flight))."""
    own = words is None
    if own:
        words = torch.ones(nblocks * 8, dtype=torch.int64, device="cuda")
    sink = torch.empty(4096 * 16, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream()
    if grid is None:
        grid = [(lanes, cps, inf) for lanes in (1, 2, 4) for cps in (4, 8, 16) for inf in (1, 2, 4, 8)]
    best = (0.0, None)
    for lanes, cps, inf in grid:
        t_best = None
        for r in range(4):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s)
            bc.blowchoc_gather_probe(words, nblocks, nreads, r, lanes, cps, sink, s, inflight=inf)
            b.record(s)
            torch.cuda.synchronize()
            if r:
                t = a.elapsed_time(b)
                t_best = t if t_best is None else min(t_best, t)
        g = nreads * 64 / (t_best / 1e3) / 1e9
        if g > best[0]:
            best = (g, (lanes, cps, inf))
    if own:
        del words
    return best


def run_gather(args):
    import torch
    import paper_2501_18977_gb300 as bc
    out = []
    for mib in [2, 64, 128, 512, 4096]:
        nb = mib * (1 << 20) // 64
        g, (lanes, cps, inf) = gather_ceiling(bc, torch, nb, nreads=100_000_000)
        out.append({"footprint_mib": mib, "gbs": round(g, 1), "lanes": lanes, "ctas_per_sm": cps,
                    "inflight": inf})
    emit({"workload": "gather_ceiling", "unit": "GB/s of whole 64-byte blocks",
                      "reads": 100_000_000, "results": out})


def run_shard(args):
    """Sub-arrays (Sec. 3.4) on one GPU: the DNA 31-mer filter split into T
    sub-arrays of M / T blocks. Per T: the partition of the 49,999,970 insert
    keys by h_0 and the unpermute of the 99,999,940 query answers, each as
    GB/s of algorithmic bytes against the copy peak (partition: one read of
    each key, one write of the key and of its index, 24 B; unpermute: the
    index, 8 B, plus a bit read and a bit written); and the whole split insert
    and query (partition, T sub-array calls, unpermute) against the unsplit
    filter. At T = 1 the split filter's words must equal the unsplit one's."""
    import torch
    import paper_2501_18977_gb300 as bc
    from paper_2501_18977_gb300.sharded import ShardedFilter
    keys, queries = make_workload()
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dq = torch.from_numpy(queries.view(np.int64)).cuda()
    n, nq = dk.numel(), dq.numel()
    s = torch.cuda.current_stream()
    peak, peak_src = peaks()
    reps = max(5, args.steps)

    def timed(fn):
        ts = []
        for r in range(reps + 1):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            torch.cuda.synchronize()
            if r:
                ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    plain = bc.Filter(CONFIG["nblocks"], CONFIG["k"], CONFIG["choices"], bc.COST_LA, CONFIG["mu"],
                      hash_seed=CONFIG["hash_seed"], batch=CONFIG["batch"])
    bm = torch.empty((nq + 63) // 64, dtype=torch.int64, device="cuda")

    def plain_insert():
        plain.clear(s)
        plain.insert(dk, s)

    t_plain_ins = timed(plain_insert)
    t_plain_q = timed(lambda: plain.query(dq, bm, s))
    plain_words = plain.words_host()
    plain_bits = bm.cpu().numpy().copy()
    plain.close()
    rows = []
    for T in (1, 2, 4, 8):
        sf = ShardedFilter(CONFIG["nblocks"], T, CONFIG["k"], CONFIG["choices"], bc.COST_LA, CONFIG["mu"],
                           hash_seed=CONFIG["hash_seed"], batch=CONFIG["batch"])
        out_k = torch.empty_like(dk)
        out_i = torch.empty(n, dtype=torch.int64, device="cuda")
        offs = torch.empty(T + 1, dtype=torch.int64, device="cuda")
        sw = bc.blowchoc_shard_partition_scratch(n, T)
        scratch = torch.empty(max(sw, 1), dtype=torch.int64, device="cuda")
        t_part = timed(lambda: bc.blowchoc_shard_partition(dk, n, T, sf.a0, out_k, out_i, offs, scratch, sw, s))

        def split_insert():
            for f in sf.subs.values():
                f.clear(s)
            sf.insert(dk, s)

        t_ins = timed(split_insert)
        t_q = timed(lambda: sf.query(dq, bm, s))
        # the unpermute alone, on the last query's partition of the queries
        part, index, offsets, off = sf.partition(dq, s)
        wc = [(off[t + 1] - off[t] + 63) // 64 for t in range(T)]
        seg = torch.zeros(max(sum(wc), 1), dtype=torch.int64, device="cuda")
        t_unp = timed(lambda: bc.blowchoc_shard_unpermute(seg, offsets, index, nq, T, bm, s))
        sf.query(dq, bm, s)
        torch.cuda.synchronize()
        bits = bm.cpu().numpy()
        st = [f.stats() for f in sf.subs.values()]
        row = {"T": T, "sub_blocks": sf.Ms,
               "partition_ms": round(t_part, 4), "partition_gbs": round(24 * n / (t_part / 1e3) / 1e9, 1),
               "partition_frac_of_peak": ratio(24 * n / (t_part / 1e3) / 1e9, peak),
               "unpermute_ms": round(t_unp, 4), "unpermute_gbs": round((8 + 0.25) * nq / (t_unp / 1e3) / 1e9, 1),
               "unpermute_frac_of_peak": ratio((8 + 0.25) * nq / (t_unp / 1e3) / 1e9, peak),
               "insert_ms": round(t_ins, 4), "query_ms": round(t_q, 4),
               "insert_vs_unsplit": round(t_plain_ins / t_ins, 3), "query_vs_unsplit": round(t_plain_q / t_q, 3),
               "inserted": int(sum(x.inserted for x in st)), "skipped": int(sum(x.skipped for x in st)),
               "hits": int(np.unpackbits(bits.view(np.uint8), bitorder="little")[:nq].sum())}
        if T == 1:
            row["equal_to_unsplit"] = bool(np.array_equal(sf.words_host(), plain_words) and
                                           np.array_equal(bits, plain_bits))
        rows.append(row)
        sf.close()
        del out_k, out_i, scratch, seg
        torch.cuda.empty_cache()
    emit({"workload": "sub_arrays_one_gpu", "filter": "DNA 31-mer (M = 2^21, k = 16, c = 3, cost^LA, B = 2^20)",
          "n_insert": n, "n_query": nq, "unsplit_insert_ms": round(t_plain_ins, 4),
          "unsplit_query_ms": round(t_plain_q, 4), "peak_gbs": peak, "peak_source": peak_src,
          "timing": "CUDA events, median of %d after one warm-up; split calls include the host reading "
                    "the partition's offsets" % reps, "rows": rows})


def run_many(args):
    """256 filters (lognormal key counts, median 200,000; 16 bits per key; k = 11,
    c = 2, cost^EXP beta = golden ratio; B_f = 2^floor(log2(M_f / 2))): all
    inserts, then all queries (half members), three ways."""
    import torch
    import paper_2501_18977_gb300 as bc
    cfg = workloads.many_filter_config()
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    filters, dks, dqs, bms = [], [], [], []
    for it in cfg:
        keys, queries = workloads.many_filter_keys(it)
        filters.append(bc.Filter(it["M"], 11, 2, bc.COST_EXP, phi, hash_seed=it["key_seed"],
                                 batch=it["B"]))
        dks.append(torch.from_numpy(keys.view(np.int64)).cuda())
        dqs.append(torch.from_numpy(queries.view(np.int64)).cuda())
        bms.append(torch.zeros(max(1, (len(queries) + 63) // 64), dtype=torch.int64, device="cuda"))
    n_ins = sum(it["n"] for it in cfg)
    n_q = sum(d.numel() for d in dqs)
    s = torch.cuda.current_stream()
    ins = [(f, d, d.numel(), None) for f, d in zip(filters, dks)]
    qry = [(f, d, d.numel(), b) for f, d, b in zip(filters, dqs, bms)]
    default_batch = bc.Batch()          # the fixed default configuration
    batch = bc.Batch()
    best = batch.autotune(ins, qry)     # batch tuning, then per (size class, k, c)

    def clear_all():
        for f in filters:
            f.clear(s)

    def plain():
        for f, d in zip(filters, dks):
            f.insert(d, s)
        for f, d, b in zip(filters, dqs, bms):
            f.query(d, b, s)

    def batched():
        batch.insert_many(ins, s)
        batch.query_many(qry, s)

    def batched_default():
        default_batch.insert_many(ins, s)
        default_batch.query_many(qry, s)

    batch.record(ins, qry)

    def graph():
        batch.replay(s)

    def timed(fn, reps):
        for _ in range(2):
            clear_all()
            fn()
        torch.cuda.synchronize()
        out = []
        for _ in range(reps):
            clear_all()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return out

    reps = max(5, args.steps)
    forms = (("plain", plain), ("batched_default", batched_default), ("batched", batched), ("graph", graph))
    results, digests = {}, {}
    clocks = ClockSampler(0)
    clocks.start()
    for name, fn in forms:
        launches0 = bc.blowchoc_launch_count()
        times = timed(fn, reps)
        launches = (bc.blowchoc_launch_count() - launches0) // (reps + 2)
        words = [f.words_host() for f in filters]
        bits = [b.cpu().numpy().copy() for b in bms]
        digests[name] = (words, bits)
        ms = statistics.median(times)
        results[name] = {"ms": round(ms, 4), "ms_min": round(min(times), 4), "ms_max": round(max(times), 4),
                         "mkeys_s": round((n_ins + n_q) / (ms / 1e3) / 1e6, 2), "launches": int(launches)}
    # phase split of the tuned work-list form: the insert alone into cleared
    # filters, the query alone on the filled filters
    ins_only = statistics.median(timed(lambda: batch.insert_many(ins, s), reps))
    clear_all()
    batch.insert_many(ins, s)
    torch.cuda.synchronize()
    q_only = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        batch.query_many(qry, s)
        b.record(s)
        torch.cuda.synchronize()
        q_only.append(a.elapsed_time(b))
    results["batched"]["insert_ms"] = round(ins_only, 4)
    results["batched"]["query_ms"] = round(statistics.median(q_only), 4)
    clk = clocks.stop()
    same = all(all(np.array_equal(a, b) for a, b in zip(digests[n][0], digests["plain"][0])) and
               all(np.array_equal(a, b) for a, b in zip(digests[n][1], digests["plain"][1]))
               for n, _ in forms[1:])
    classes = {}
    for key in sorted({(batch.size_class(it["M"]), 11, 2) for it in cfg}):
        t, is_set = batch.class_tuning(*key)
        members = [it for it in cfg if batch.size_class(it["M"]) == key[0]]
        classes[["cache", "l2", "spill", "hbm"][key[0]]] = dict(
            t, tuned=bool(is_set), filters=len(members), keys=int(sum(it["n"] for it in members)))
    st = [f.stats() for f in filters]
    # algorithmic bytes of the job (c = 2): insert 8 + 128 + 64 (1 - skip
    # rate) per key; queries half members (at least one block, 8 + 64 + 1/8)
    # and half random (8 + 128 + 1/8); against random whole blocks over the
    # filters' combined footprint (the gather probe)
    ins_done = sum(x.inserted for x in st)
    skip_rate = sum(x.skipped for x in st) / max(1, ins_done + sum(x.skipped for x in st))
    alg_bytes = n_ins * (8 + 128 + 64 * (1 - skip_rate)) + (n_q / 2) * (8 + 64 + 0.125) + (n_q / 2) * (8 + 128 + 0.125)
    total_blocks = int(sum(it["M"] for it in cfg))
    ceil, ceil_cfg = gather_ceiling(bc, torch, total_blocks)
    for r in results.values():
        r["gbs_lower_bound"] = round(alg_bytes / (r["ms"] / 1e3) / 1e9, 1)
        r["frac_of_gather_ceiling"] = ratio(alg_bytes / (r["ms"] / 1e3) / 1e9, ceil)
    out = {"workload": "many_filters_256", "metric": "insert+query throughput, 256 filters",
           "unit": "Mkeys/s", "n_insert": n_ins, "n_query": n_q,
           "filters": len(cfg), "filter_mib": round(sum(it["M"] for it in cfg) * 64 / 2**20, 1),
           "batch_rounds": int(max((it["n"] + it["B"] - 1) // it["B"] for it in cfg)),
           "results": results,
           "batched_vs_plain": round(results["plain"]["ms"] / results["batched"]["ms"], 3),
           "graph_vs_plain": round(results["plain"]["ms"] / results["graph"]["ms"], 3),
           "tuned_vs_default": round(results["batched_default"]["ms"] / results["batched"]["ms"], 3),
           "identical_words_and_bitmaps": bool(same),
           "inserted": int(sum(x.inserted for x in st)), "skipped": int(sum(x.skipped for x in st)),
           "autotuned": {"lanes_choose": best.lanes_choose, "lanes_query": best.lanes_query,
                         "query_early": best.query_early, "ctas_per_sm": best.ctas_per_sm,
                         "classes": classes},
           "repeats": reps, "clocks": clk,
           "gather_ceiling_gbs": round(ceil, 1),
           "gather_ceiling_config": {"lanes": ceil_cfg[0], "ctas_per_sm": ceil_cfg[1], "inflight": ceil_cfg[2]},
           "bytes_note": "algorithmic bytes with members' queries at one block each (a lower bound)",
           "timing": "CUDA events per repetition (median, min, max), filters cleared before each"}
    default_batch.close()
    batch.close()
    for f in filters:
        f.close()
    emit(out)


def run_serve(args):
    """64 device-resident filters (2^20..2^31 bits log-uniform, k = 14, c = 2,
    cost^MIX sigma = 50), 10,000 requests (70% query, sizes log-uniform in
    1..10^6 keys, uniform target filter), 80 GB HBM budget. Capacity is the
    closed-loop rate (all requests arrive at once); the Poisson stream is then
    offered at 50/80/95% of it. The same requests run through plain per-request
    calls on one stream give the comparison rate and the reference results."""
    import torch
    import paper_2501_18977_gb300 as bc
    filters, reqs = workloads.serving_config(n_requests=args.requests)
    sizes = [r["n"] for r in reqs]
    total_keys = int(sum(sizes))
    offs = np.zeros(len(reqs) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    pinned = torch.empty(total_keys, dtype=torch.int64).pin_memory()
    host = pinned.numpy().view(np.uint64)
    for r in reqs:
        host[offs[r["index"]]:offs[r["index"] + 1]] = workloads.serving_keys(filters, r)
    keys = {r["index"]: host[offs[r["index"]]:offs[r["index"] + 1]] for r in reqs}

    def serve(time_scale):
        srv = bc.Server(80 * 10**9, staging_bytes=4 << 30, streams=4, max_wave_requests=64)
        ids = [srv.add_filter(f["M"], 14, 2, bc.COST_MIX, 50.0, f["key_seed"], f["B"]) for f in filters]
        bms = {}
        for r in reqs:
            bm = np.zeros((r["n"] + 63) // 64, dtype=np.uint64) if r["kind"] == 1 else None
            if bm is not None:
                bms[r["index"]] = bm
            srv.submit(ids[r["filter"]], r["kind"], keys[r["index"]], bm, r["arrival"] * time_scale)
        launches0 = bc.blowchoc_launch_count()
        srv.start()
        srv.wait(600.0)
        st = srv.stats()
        launches = bc.blowchoc_launch_count() - launches0
        srv.close()
        span = st.last_done_s - st.first_arrival_s
        return bms, st, span, launches

    reps = max(5, min(args.steps, 10))

    def plain():
        # one request at a time, in arrival order, one stream
        fs = [bc.Filter(f["M"], 14, 2, bc.COST_MIX, 50.0, hash_seed=f["key_seed"], batch=f["B"])
              for f in filters]
        dev = torch.empty(max(sizes), dtype=torch.int64, device="cuda")
        dbm = torch.empty((max(sizes) + 63) // 64, dtype=torch.int64, device="cuda")
        bms = {}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r in sorted(reqs, key=lambda r: (r["arrival"], r["index"])):
            n = r["n"]
            dev[:n].copy_(pinned[offs[r["index"]]:offs[r["index"] + 1]], non_blocking=True)
            if r["kind"] == 0:
                fs[r["filter"]].insert(dev[:n])
            else:
                fs[r["filter"]].query(dev[:n], dbm)
                out = np.zeros((n + 63) // 64, dtype=np.uint64)
                out[:] = dbm[: (n + 63) // 64].cpu().numpy().view(np.uint64)
                bms[r["index"]] = out
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        for f in fs:
            f.close()
        return bms, secs

    plain_runs = [plain() for _ in range(reps)]
    plain_bms = plain_runs[0][0]
    plain_times = sorted(t for _, t in plain_runs)
    plain_s = statistics.median(plain_times)
    closed_runs = [serve(0.0) for _ in range(reps)]
    closed_runs.sort(key=lambda r: r[2])
    closed_bms, closed_st, closed_span, _ = closed_runs[len(closed_runs) // 2]
    capacity = total_keys / closed_span
    mean_req = total_keys / len(reqs)
    same = all(all(np.array_equal(run[0][j], b) for j, b in plain_bms.items())
               for run in plain_runs[1:] + [(c[0], None) for c in closed_runs])
    loads = []
    for load in (0.5, 0.8, 0.95):
        rate = load * capacity / mean_req          # requests per second
        bms, st, span, launches = serve(1.0 / rate)
        same = same and all(np.array_equal(bms[j], b) for j, b in plain_bms.items())
        loads.append({"offered_load": load, "offered_mkeys_s": round(load * capacity / 1e6, 1),
                      "achieved_mkeys_s": round(total_keys / span / 1e6, 1),
                      "p50_ms": round(st.p50_latency_s * 1e3, 3), "p99_ms": round(st.p99_latency_s * 1e3, 3),
                      "max_ms": round(st.max_latency_s * 1e3, 3), "waves": int(st.waves),
                      "mean_wave_requests": round(st.mean_wave_requests, 2), "gpu_launches": int(launches)})
    out = {"workload": "serving_64_filters", "metric": "served keys/s with p50/p99 latency",
           "requests": len(reqs), "keys": total_keys,
           "filter_gb": round(sum(f["M"] for f in filters) * 64 / 1e9, 3),
           "repeats": reps,
           "plain_per_request_mkeys_s": round(total_keys / plain_s / 1e6, 1),
           "plain_per_request_mkeys_s_range": [round(total_keys / plain_times[-1] / 1e6, 1),
                                               round(total_keys / plain_times[0] / 1e6, 1)],
           "served_capacity_mkeys_s": round(capacity / 1e6, 1),
           "served_capacity_mkeys_s_range": [round(total_keys / closed_runs[-1][2] / 1e6, 1),
                                             round(total_keys / closed_runs[0][2] / 1e6, 1)],
           "served_vs_plain": round(capacity / (total_keys / plain_s), 2),
           "closed_loop": {"p50_ms": round(closed_st.p50_latency_s * 1e3, 3),
                           "p99_ms": round(closed_st.p99_latency_s * 1e3, 3),
                           "waves": int(closed_st.waves),
                           "mean_wave_requests": round(closed_st.mean_wave_requests, 2),
                           "mean_wave_gpu_ms": round(closed_st.mean_wave_gpu_ms, 3),
                           "launch_host_s": round(closed_st.launch_host_s, 3),
                           "span_s": round(closed_span, 3)},
           "poisson": loads, "identical_to_plain_results": bool(same),
           "timing": "host steady clock (server) and wall clock (plain), medians of the repeats; "
                     "keys from pinned host memory"}
    emit(out)


SWEEP_SETTINGS = [(1, "EXP", 0), (2, "MIX", 50.0), (2, "LA", 3.5), (2, "EXP", 0), (3, "MIX", 50.0),
                  (3, "LA", 3.5), (3, "EXP", 0)]
SWEEP_BITS = [20, 18, 16, 14, 12, 10, 8, 6]


def run_sweep(args):
    """Overload / FPR sweep: M = 2^23 blocks (512 MiB), k = 12, B = 2^20, hash
    seed 3001; keys: splitmix64 seed 3001, grown by one insert call per point to
    floor(2^32 / b) keys for b = 20, 18, ..., 6 bits per key; 10^8 negatives
    (seed 3002) per point. Reports measured FPR W/N beside the one-choice
    blocked-Bloom formula, the standard Bloom formula and the histogram
    estimate, and insert / query rates."""
    import torch
    import paper_2501_18977_gb300 as bc
    from paper_2501_18977_gb300 import sweeps
    M, k, B = 1 << 23, 12, 1 << 20
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    kinds = {"MIX": bc.COST_MIX, "LA": bc.COST_LA, "EXP": bc.COST_EXP}
    nmax = (1 << 32) // SWEEP_BITS[-1]
    keys = torch.empty(nmax, dtype=torch.int64, device="cuda")
    chunk = 1 << 25
    for s0 in range(0, nmax, chunk):
        c = min(chunk, nmax - s0)
        keys[s0:s0 + c].copy_(torch.from_numpy(workloads.splitmix64(3001, c, s0).view(np.int64)))
    neg = torch.from_numpy(workloads.uniform_keys(3002, 100_000_000).view(np.int64)).cuda()
    bm = torch.empty((neg.numel() + 63) // 64, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream()
    rows = []
    reps = max(5, min(args.steps, 10))
    for c, cname, par in SWEEP_SETTINGS:
        par = phi if cname == "EXP" else par
        f = bc.Filter(M, k, c, kinds[cname], par, hash_seed=3001, batch=B)
        times = {b: ([], []) for b in SWEEP_BITS}
        first = {}
        for rep in range(reps):  # the filter regrown from empty each time; results are deterministic
            f.clear(s)
            n_prev = 0
            for b in SWEEP_BITS:
                n = (1 << 32) // b
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                e[0].record(s)
                f.insert(keys[n_prev:n], s)
                e[1].record(s)
                f.query(neg, bm, s)
                e[2].record(s)
                torch.cuda.synchronize()
                times[b][0].append(e[0].elapsed_time(e[1]))
                times[b][1].append(e[1].elapsed_time(e[2]))
                if rep == 0:
                    st = f.stats()
                    W = int(np.unpackbits(bm.cpu().numpy().view(np.uint8), bitorder="little")[: neg.numel()].sum())
                    first[b] = (n, n_prev, W, st)
                n_prev = n
        for b in SWEEP_BITS:
            n, n_prev, W, st = first[b]
            ti, tq = statistics.median(times[b][0]), statistics.median(times[b][1])
            rows.append({"c": c, "cost": cname, "bits_per_key": b, "n": n, "fpr": W / neg.numel(),
                         "false_positives": W, "fpr_est_hist": st.fpr_est,
                         "blocked_bloom_formula": sweeps.blocked_bloom_fpr(n, M, k),
                         "bloom_formula": sweeps.bloom_fpr(n, M * 512, k),
                         "inserted": st.inserted, "skipped": st.skipped, "set_bits": st.set_bits,
                         "insert_mkeys_s": round((n - n_prev) / (ti / 1e3) / 1e6, 1),
                         "query_mkeys_s": round(neg.numel() / (tq / 1e3) / 1e6, 1)})
        f.close()
    emit({"workload": "overload_sweep", "M": M, "k": k, "B": B, "negatives": neg.numel(),
          "repeats": reps, "timing": "CUDA events, median of the repeats", "rows": rows})


def run_batching(args):
    """FPR and load balance against the batch size B: M = 2^16 blocks (4 MiB),
    k = 12, c in {2, 3}, cost^EXP beta = golden ratio, 12 bits per key
    (2^32/12 / 128 = 2,796,202 keys, seed 3001), B from 1 (the paper's
    sequential insertion) to 2^20; 10^8 negatives (seed 3002)."""
    import torch
    import paper_2501_18977_gb300 as bc
    M, k = 1 << 16, 12
    n = ((1 << 32) // 12) >> 7
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    keys = torch.from_numpy(workloads.uniform_keys(3001, n).view(np.int64)).cuda()
    neg = torch.from_numpy(workloads.uniform_keys(3002, 100_000_000).view(np.int64)).cuda()
    bm = torch.empty((neg.numel() + 63) // 64, dtype=torch.int64, device="cuda")
    rows = []
    for c in (2, 3):
        for B in (1, 16, 256, 4096, 1 << 14, 1 << 16, 1 << 18, 1 << 20):
            f = bc.Filter(M, k, c, bc.COST_EXP, phi, hash_seed=3001, batch=B)
            s = torch.cuda.current_stream()
            ins_ms = []
            for rep in range(max(5, min(args.steps, 10))):
                f.clear(s)
                a = torch.cuda.Event(enable_timing=True)
                b2 = torch.cuda.Event(enable_timing=True)
                a.record(s)
                f.insert(keys, s)
                b2.record(s)
                torch.cuda.synchronize()
                ins_ms.append(a.elapsed_time(b2))
            f.query(neg, bm, s)
            torch.cuda.synchronize()
            st = f.stats()
            W = int(np.unpackbits(bm.cpu().numpy().view(np.uint8), bitorder="little")[: neg.numel()].sum())
            L = np.arange(513)
            h = np.array(list(st.hist), dtype=np.float64)
            mean = float((h * L).sum() / M)
            sd = float(math.sqrt((h * (L - mean) ** 2).sum() / M))
            rows.append({"c": c, "B": B, "fpr": W / neg.numel(), "fpr_est_hist": st.fpr_est,
                         "mean_load": round(mean, 3), "sd_load": round(sd, 3),
                         "insert_ms": round(statistics.median(ins_ms), 3),
                         "insert_ms_range": [round(min(ins_ms), 3), round(max(ins_ms), 3)]})
            f.close()
    emit({"workload": "batching_cost", "M": M, "k": k, "n": n, "cost": "EXP golden ratio",
                      "rows": rows})


def run_small(args):
    """10^6 uniform keys (seed 1) into M = 32768 blocks (2^24 bits, L2-resident),
    k = 14, c = 2, cost^MIX sigma = 50; B = 65536 and B = 1; queries: the keys
    plus 10^6 disjoint keys (seed 1001). Insert and query rates, FPR."""
    import torch
    import paper_2501_18977_gb300 as bc
    keys = workloads.uniform_keys(1, 1_000_000)
    neg = workloads.disjoint_keys(1001, 1_000_000, keys)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dq = torch.from_numpy(np.concatenate([keys, neg]).view(np.int64)).cuda()
    bm = torch.empty((dq.numel() + 63) // 64, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream()
    # the ceiling beside the peak for this L2-resident filter: random whole
    # 64-byte blocks over the same 2 MiB footprint (the gather probe)
    ceil, ceil_cfg = gather_ceiling(bc, torch, 32768)
    peak, peak_src = peaks()
    rows = []
    for B in (65536, 1):
        f = bc.Filter(32768, 14, 2, bc.COST_MIX, 50.0, hash_seed=1, batch=B)
        reps = max(5, args.steps) if B > 1 else 5
        ti, tq = [], []
        for _ in range(reps + 1):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            f.clear(s)
            e[0].record(s)
            f.insert(dk, s)
            e[1].record(s)
            f.query(dq, bm, s)
            e[2].record(s)
            torch.cuda.synchronize()
            ti.append(e[0].elapsed_time(e[1]))
            tq.append(e[1].elapsed_time(e[2]))
        ti, tq = ti[1:], tq[1:]  # after one warm-up
        h = bm.cpu().numpy().view(np.uint8)
        bits = np.unpackbits(h, bitorder="little")[: dq.numel()]
        st = f.stats()
        skip = st.skipped / max(1, st.inserted + st.skipped)
        # algorithmic bytes: insert 8 + 64 c + 64 (1 - skip rate) per key; query
        # negatives 8 + 64 c + 1/8, members at least 8 + 64 + 1/8 (first block)
        i_gbs = 1e6 * (8 + 128 + 64 * (1 - skip)) / (statistics.median(ti) / 1e3) / 1e9
        q_gbs = (1e6 * (8 + 128 + 0.125) + 1e6 * (8 + 64 + 0.125)) / (statistics.median(tq) / 1e3) / 1e9
        rows.append({"B": B, "insert_ms": round(statistics.median(ti), 4),
                     "insert_gbs": round(i_gbs, 1), "insert_frac_of_l2_gather_ceiling": ratio(i_gbs, ceil),
                     "query_gbs_lower_bound": round(q_gbs, 1), "query_frac_of_l2_gather_ceiling": ratio(q_gbs, ceil),
                     "insert_mkeys_s": round(1e6 / (statistics.median(ti) / 1e3) / 1e6, 1),
                     "query_ms": round(statistics.median(tq), 4),
                     "query_mkeys_s": round(2e6 / (statistics.median(tq) / 1e3) / 1e6, 1),
                     "false_negatives": int(1_000_000 - bits[:1_000_000].sum()),
                     "fpr": float(bits[1_000_000:].mean()), "fpr_est_hist": st.fpr_est,
                     "inserted": st.inserted, "skipped": st.skipped})
        f.close()
    emit({"workload": "small_uniform", "M": 32768, "k": 14, "c": 2, "cost": "MIX 50",
          "timing": "CUDA events, median of at least 5 repeats after one warm-up",
          "l2_gather_ceiling_gbs": round(ceil, 1),
          "l2_gather_ceiling_config": {"lanes": ceil_cfg[0], "ctas_per_sm": ceil_cfg[1], "inflight": ceil_cfg[2]},
          "hbm_copy_peak_gbs": peak, "peak_source": peak_src,
          "bytes_note": "members' query bytes counted at one block each (a lower bound: the first "
                        "candidate that holds a member is not counted here)",
          "rows": rows})


def run_learn(args):
    """Learned cost: train on 32 small filters per step (512 blocks, the small
    configuration's 16 bits per key, k = 14, c = 2), then insert
    10^6 held-out keys (seed 11) greedily with the learned table, cost^EXP
    (golden ratio) and cost^MIX (sigma = 50); FPR from 10^8 negatives
    (seed 12) and from the load histogram."""
    import torch
    import paper_2501_18977_gb300 as bc
    from paper_2501_18977_gb300.learned import train_cost_table
    M, k, c, B, n = 32768, 14, 2, 65536, 1_000_000
    held = torch.from_numpy(workloads.uniform_keys(11, n).view(np.int64)).cuda()
    neg = torch.from_numpy(workloads.uniform_keys(12, 100_000_000).view(np.int64)).cuda()
    bm = torch.empty((neg.numel() + 63) // 64, dtype=torch.int64, device="cuda")
    t0 = time.perf_counter()
    # training filters: 32 filters of 512 blocks at the same 16 bits per key, k, c and 16 batches
    Mt = 512
    nt = Mt * 512 // 16
    table, rewards, mlp = train_cost_table(Mt, k, c, nt // 16, nt, steps=args.train_steps, filters=32,
                                           tau=0.05, lr=3e-3, seed=7)
    train_s = time.perf_counter() - t0
    mlp.close()

    def evaluate(kind, par, tab=None):
        f = bc.Filter(M, k, c, kind, par, hash_seed=1, batch=B)
        if tab is not None:
            f.set_cost_table(tab)
        f.insert(held)
        f.query(neg, bm)
        torch.cuda.synchronize()
        W = int(np.unpackbits(bm.cpu().numpy().view(np.uint8), bitorder="little")[: neg.numel()].sum())
        st = f.stats()
        f.close()
        return {"fpr": W / neg.numel(), "fpr_est_hist": st.fpr_est, "set_bits": st.set_bits}

    phi = (1.0 + math.sqrt(5.0)) / 2.0
    learned = evaluate(bc.COST_EXP, phi, table)
    exp_cost = evaluate(bc.COST_EXP, phi)
    mix_cost = evaluate(bc.COST_MIX, 50.0)
    emit({"workload": "learned_cost", "M": M, "k": k, "c": c, "B": B, "n": n,
                      "train_steps": args.train_steps, "train_seconds": round(train_s, 2),
                      "reward_first10": float(np.mean(rewards[:10])), "reward_last10": float(np.mean(rewards[-10:])),
                      "learned": learned, "exp_golden_ratio": exp_cost, "mix_sigma50": mix_cost,
                      "fpr_gain_vs_exp": exp_cost["fpr"] / learned["fpr"] if learned["fpr"] else None,
                      "note": "gain > 1 means the learned table gives a lower FPR than cost^EXP"})


def golden_pbar():
    """Mean 1-based index of the first candidate block holding an inserted
    31-mer of this workload, as counted by the oracle (tests/golden)."""
    path = os.path.join(ROOT, "tests", "golden", "dna_kmer_31_c3_la.txt")
    if os.path.exists(path):
        with open(path) as fh:
            for line in fh:
                if line.startswith("pbar_positive"):
                    return float(line.split("=")[1].split()[0]), "oracle"
    return 1.0, "lower bound 1.0 (oracle count not stored)"


# The overload sweep's 12 bits/key point (Sec. 4.1), the HBM-resident
# filter of the benchmark: M = 2^23 blocks (512 MiB, four times L2), k = 12,
# B = 2^20, hash seed 3001; keys: the splitmix64 stream of seed 3001 grown
# through 20, 18, 16, 14 and 12 bits per key in one insert call per point;
# 10^8 negatives from seed 3002.
HBM_POINT = dict(nblocks=1 << 23, k=12, batch=1 << 20, hash_seed=3001, neg_seed=3002,
                 n_neg=100_000_000, bits=[20, 18, 16, 14, 12])
HBM_SETTINGS = [(2, "EXP"), (3, "LA")]


def sweep_golden_row(c, cost, bits):
    """The oracle's stored row of the overload sweep at `bits` per key."""
    path = os.path.join(ROOT, "tests", "golden", "overload_sweep_c%d_%s.txt" % (c, cost))
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or "|" not in line:
                continue
            f = [x.strip() for x in line.split("|")]
            if int(f[0]) == bits:
                return dict(n=int(f[1]), inserted=int(f[2]), skipped=int(f[3]), set_bits=int(f[4]),
                            fp=int(f[5]), words=f[6], bitmap=f[7])
    return None


def hbm_resident(bc, torch, peak, local, reps=3):
    """Insert and negative-query throughput of the 512 MiB filter at 12 bits
    per key, for c = 2 cost^EXP and c = 3 cost^LA: insert time is the five
    insert calls that grow the cleared filter to 357,913,941 keys, query time
    one query of 10^8 negatives; best of `reps` after one untimed pass, with
    clocks sampled. The final words and negative bitmap are compared with the
    oracle's stored digests."""
    import hashlib
    P = HBM_POINT
    stream = torch.cuda.current_stream()
    nmax = (1 << 32) // P["bits"][-1]
    keys = bc.generate_keys(nmax, P["hash_seed"], stream=stream)
    neg = bc.generate_keys(P["n_neg"], P["neg_seed"], stream=stream)
    bm = torch.empty((P["n_neg"] + 63) // 64, dtype=torch.int64, device="cuda")
    ceil, ceil_cfg = gather_ceiling(bc, torch, P["nblocks"])
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    kinds = {"MIX": (bc.COST_MIX, 50.0), "LA": (bc.COST_LA, 3.5), "EXP": (bc.COST_EXP, phi)}
    out = {"workload": "overload sweep point, 12 bits/key", "nblocks": P["nblocks"],
           "filter_mib": P["nblocks"] * 64 >> 20, "k": P["k"], "batch": P["batch"],
           "n_insert": nmax, "n_query": P["n_neg"],
           "gather_ceiling_gbs": round(ceil, 1),
           "gather_ceiling_config": {"lanes": ceil_cfg[0], "ctas_per_sm": ceil_cfg[1],
                                     "inflight": ceil_cfg[2]},
           "peak_gbs": peak, "settings": []}
    clocks = ClockSampler(local)
    clocks.start()
    for c, cost in HBM_SETTINGS:
        kind, par = kinds[cost]
        f = bc.Filter(P["nblocks"], P["k"], c, kind, par, hash_seed=P["hash_seed"], batch=P["batch"],
                      stream=stream)
        ins_ms, q_ms = [], []
        for r in range(reps + 1):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            f.clear(stream)
            e[0].record(stream)
            n_prev = 0
            for b in P["bits"]:
                n = (1 << 32) // b
                f.insert(keys[n_prev:n], stream)
                n_prev = n
            e[1].record(stream)
            f.query(neg, bm, stream)
            e[2].record(stream)
            torch.cuda.synchronize()
            if r or reps == 0:
                ins_ms.append(e[0].elapsed_time(e[1]))
                q_ms.append(e[1].elapsed_time(e[2]))
        st = f.stats()
        h = bm.cpu().numpy().view(np.uint64)
        fp = int(np.unpackbits(h.view(np.uint8), bitorder="little")[:P["n_neg"]].sum())
        words_sha = hashlib.sha256(f.words_host().astype("<u8").tobytes()).hexdigest()
        bm_sha = hashlib.sha256(h.astype("<u8").tobytes()).hexdigest()
        f.close()
        g = sweep_golden_row(c, cost, P["bits"][-1])
        if g is None:
            parity = "oracle digest not stored"
        else:
            same = (g["n"] == nmax and g["inserted"] == st.inserted and g["skipped"] == st.skipped
                    and g["set_bits"] == st.set_bits and g["fp"] == fp and g["words"] == words_sha
                    and g["bitmap"] == bm_sha)
            parity = "equal to the oracle's stored digests" if same else "DIFFERS from the oracle's stored digests"
        skip = st.skipped / max(1, st.inserted + st.skipped)
        ib = nmax * (8 + 64 * c + 64 * (1 - skip))
        qb = P["n_neg"] * (8 + 64 * c + 1 / 8)
        it, qt = min(ins_ms), min(q_ms)
        igbs, qgbs = ib / (it / 1e3) / 1e9, qb / (qt / 1e3) / 1e9
        out["settings"].append({
            "choices": c, "cost": cost, "insert_ms": round(it, 3), "query_ms": round(qt, 3),
            "insert_mkeys_s": round(nmax / (it / 1e3) / 1e6, 1),
            "query_mkeys_s": round(P["n_neg"] / (qt / 1e3) / 1e6, 1),
            "insert_gbs": round(igbs, 1), "query_gbs": round(qgbs, 1),
            "insert_frac_of_peak": round(igbs / peak, 4), "query_frac_of_peak": round(qgbs / peak, 4),
            "insert_frac_of_gather_ceiling": round(igbs / ceil, 4),
            "query_frac_of_gather_ceiling": round(qgbs / ceil, 4),
            "insert_bytes_per_key": round(8 + 64 * c + 64 * (1 - skip), 3),
            "query_bytes_per_key": round(8 + 64 * c + 1 / 8, 3),
            "inserted": st.inserted, "skipped": st.skipped, "false_positives": fp,
            "fpr": fp / P["n_neg"], "parity": parity})
    out["clocks"] = clocks.stop()
    del keys, neg, bm
    torch.cuda.empty_cache()
    return out


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(keys, queries, n_ins, n_q):
    """The oracle (single-threaded C) on a bounded sample of the workload,
    pinned to one host core, best of three runs."""
    from oracle import OracleFilter
    qs = np.concatenate([queries[: n_q // 2], queries[N_KEYS: N_KEYS + n_q // 2]])
    old_aff = os.sched_getaffinity(0) if hasattr(os, "sched_getaffinity") else None
    if old_aff:
        os.sched_setaffinity(0, {min(old_aff)})
    times = []
    try:
        for _ in range(3):
            o = OracleFilter(CONFIG["nblocks"], CONFIG["k"], CONFIG["choices"], COST_LA, CONFIG["mu"],
                             seed=CONFIG["hash_seed"], batch=CONFIG["batch"])
            t0 = time.perf_counter()
            o.insert(keys[:n_ins])
            o.query(qs)
            times.append(time.perf_counter() - t0)
            del o
    finally:
        if old_aff:
            os.sched_setaffinity(0, old_aff)
    dt = min(times)
    return {"value": round((n_ins + len(qs)) / dt / 1e6, 4), "unit": "Mkeys/s", "cores": 1,
            "kind": "oracle", "cpu": cpu_model(), "nproc": os.cpu_count(),
            "sample": "first %d inserts (one partial batch, B = 2^20) and %d queries (half "
                      "members, half other-genome 31-mers) of the same workload, best of 3 runs "
                      "of %.1f-%.1f s pinned to one core" % (n_ins, len(qs), min(times), max(times))}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    keys, queries = make_workload()
    from oracle import OracleFilter
    n_ins, n_q = 200_000, 400_000
    times = []
    for step in range(args.warmup + args.steps):
        o = OracleFilter(CONFIG["nblocks"], CONFIG["k"], CONFIG["choices"], COST_LA, CONFIG["mu"],
                         seed=CONFIG["hash_seed"], batch=CONFIG["batch"])
        qs = np.concatenate([queries[: n_q // 2], queries[N_KEYS: N_KEYS + n_q // 2]])
        t0 = time.perf_counter()
        o.insert(keys[:n_ins])
        o.query(qs)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = (n_ins + n_q) / (ms / 1e3) / 1e6
    sample = ("per step: %d inserts (B = 2^20, one partial batch) and %d queries (half members, "
              "half other-genome 31-mers) of the DNA 31-mer workload" % (n_ins, n_q))
    out = {"impl": "reference", "metric": "insert+query throughput (DNA 31-mers, c=3, k=16, cost^LA)",
           "value": round(value, 4), "unit": "Mkeys/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": dict(CONFIG, sample=sample),
           "cpu_baseline": {"value": round(value, 4), "unit": "Mkeys/s", "cores": 1,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 4), "unit": "Mkeys/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(finite(out), allow_nan=False))


def run_cluster(args):
    """Cluster-resident against global-memory insertion on serving-sized
    filters (k = 14, c = 2, cost^MIX sigma = 50, B = 2^floor(log2(M/2)),
    ~10^6 uniform keys each): per shape the insert time of the global-memory
    kernels (cluster_max = 0) and of the cluster-resident kernel (persistent
    insert off, so that every shape qualifies), the CTAs per cluster, and the
    path the defaults take. Results are checked equal."""
    import torch
    import paper_2501_18977_gb300 as bc
    shapes = [(2075, 1024, 939473), (5808, 2048, 950901), (9022, 4096, 978426), (6250, 2048, 200000)]
    s = torch.cuda.current_stream()
    rows = []
    for M, B, n in shapes:
        keys = torch.from_numpy(workloads.uniform_keys(M, n).view(np.int64)).cuda()
        f = bc.Filter(M, 14, 2, bc.COST_MIX, 50.0, hash_seed=3, batch=B, stream=s)
        row = {"M": M, "B": B, "n": n, "batches": (n + B - 1) // B}
        words = {}
        # the cluster arm turns the persistent insert off so that batches
        # above 2048 keys run cluster-resident too (by default they take the
        # persistent insert, which is faster there)
        for name, cmax, pers in (("global", 0, 1), ("cluster", 16, 0)):
            f.set_tuning(cluster_max=cmax, persistent=pers)
            times = []
            for rep in range(args.warmup + args.steps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                f.clear(s)
                a.record(s)
                f.insert(keys, s)
                b.record(s)
                torch.cuda.synchronize()
                if rep >= args.warmup:
                    times.append(a.elapsed_time(b))
            ms = statistics.median(times)
            words[name] = f.words_host()
            row[name + "_ms"] = round(ms, 4)
            row[name + "_us_per_batch"] = round(ms * 1e3 / row["batches"], 2)
        row["ctas_per_cluster"] = f.cluster_ctas(n)
        f.set_tuning(cluster_max=16, persistent=1)
        row["default_path"] = "cluster" if f.cluster_ctas(n) else "global"
        row["identical"] = bool(np.array_equal(words["global"], words["cluster"]))
        f.close()
        rows.append(row)
    emit({"workload": "cluster_resident_insert", "rows": rows,
                      "timing": "CUDA events, median of --steps after --warmup"})


def run_lanes(args):
    """Persistent insert time per lanes_choose across filter sizes: uniform
    device-generated keys at 12 bits per key, B = 2^20, cluster path off, two
    shapes (three choices, k = 16, cost^LA; two choices, k = 12, cost^EXP).
    Per row the median of --steps timed inserts after one warm-up, the
    fastest lane width and the default; the words must not depend on it."""
    import torch
    import paper_2501_18977_gb300 as bc
    s = torch.cuda.current_stream()
    phi = (1 + 5 ** 0.5) / 2
    rows = []
    for mib in (2, 8, 32, 64, 96, 128, 192, 256, 512):
        M = mib * (1 << 20) // 64
        n = M * 512 // 12
        keys = bc.generate_keys(n, 7)
        for c, k, cost, par, cname in ((3, 16, bc.COST_LA, 3.5, "LA"), (2, 12, bc.COST_EXP, phi, "EXP")):
            f = bc.Filter(M, k, c, cost, par, hash_seed=5, batch=1 << 20, stream=s)
            default = f.tuning().lanes_choose
            f.set_tuning(cluster_max=0)
            row = {"filter_mib": mib, "M": M, "n": n, "c": c, "k": k, "cost": cname, "default": default}
            digests = set()
            for lanes in (1, 2, 4, 8):
                f.set_tuning(lanes_choose=lanes)
                times = []
                for rep in range(1 + max(1, args.steps)):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    f.clear(s)
                    a.record(s)
                    f.insert(keys, s)
                    b.record(s)
                    torch.cuda.synchronize()
                    if rep:
                        times.append(a.elapsed_time(b))
                row["lanes%d_ms" % lanes] = round(statistics.median(times), 4)
                digests.add(int(f.words_view().sum().item()))
            row["best"] = min((1, 2, 4, 8), key=lambda ln: row["lanes%d_ms" % ln])
            row["identical"] = len(digests) == 1
            f.close()
            rows.append(row)
        del keys
        torch.cuda.empty_cache()
    # around the L2 size the best width also depends on the load: two and
    # four lanes at 32, 21.5 and 16 bits per key
    load_rows = []
    for mib in (96, 128, 192):
        M = mib * (1 << 20) // 64
        for bpk in (32, 21.5, 16):
            n = int(M * 512 / bpk)
            keys = bc.generate_keys(n, 7)
            for c, k, cost, par, cname in ((3, 16, bc.COST_LA, 3.5, "LA"), (2, 12, bc.COST_EXP, phi, "EXP")):
                f = bc.Filter(M, k, c, cost, par, hash_seed=5, batch=1 << 20, stream=s)
                f.set_tuning(cluster_max=0)
                row = {"filter_mib": mib, "bits_per_key": bpk, "c": c, "k": k, "cost": cname}
                for lanes in (2, 4):
                    f.set_tuning(lanes_choose=lanes)
                    times = []
                    for rep in range(1 + max(1, args.steps)):
                        a = torch.cuda.Event(enable_timing=True)
                        b = torch.cuda.Event(enable_timing=True)
                        f.clear(s)
                        a.record(s)
                        f.insert(keys, s)
                        b.record(s)
                        torch.cuda.synchronize()
                        if rep:
                            times.append(a.elapsed_time(b))
                    row["lanes%d_ms" % lanes] = round(statistics.median(times), 4)
                f.close()
                load_rows.append(row)
            del keys
            torch.cuda.empty_cache()
    emit({"workload": "insert_lanes_by_filter_size", "B": 1 << 20, "bits_per_key": 12,
          "rows": rows, "load_rows": load_rows, "timing": "CUDA events, median of --steps after one warm-up"})


def run_variants(args):
    """The set-phase and bit-selection variants beside the defaults, per
    shape (uniform device-generated keys, cluster path off): the persistent
    insert with the direct set (64-bit OR reductions at L2, set_mode 0) and
    with the sort-by-block set (set_mode 1), whose words must be identical;
    then insert and query times with random (bitsel 0) and distinct
    (bitsel 1, Appendix B) bit selection, which build different filters by
    design. Medians of --steps timed calls after one warm-up."""
    import torch
    import paper_2501_18977_gb300 as bc
    s = torch.cuda.current_stream()
    phi = (1 + 5 ** 0.5) / 2
    # filters of 2^12 .. 2^23 blocks at 16 bits per key (n = 32 M keys), with
    # batches of M / 16, M / 2, 4 M and 32 M keys (1/16 .. 32 keys per block
    # and batch; B >= n is one batch), c = 2 cost^EXP; plus the DNA shape
    shapes = [("DNA shape, 128 MiB, three choices", 1 << 21, 16, 3, bc.COST_LA, 3.5, 1 << 20, 1 << 25)]
    for lg in (12, 15, 18, 21, 23):
        M = 1 << lg
        for bm in (1 / 16, 1 / 2, 4, 32):
            B = max(1, int(M * bm))
            if B <= 2048:
                continue  # batches of one CTA: the set mode does not apply
            shapes.append(("%d MiB, B/M = %g" % (max(1, M * 64 >> 20), bm), M, 12, 2, bc.COST_EXP, phi, B,
                           32 * M))

    def timed(fn):
        times = []
        for rep in range(1 + max(1, args.steps)):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            torch.cuda.synchronize()
            if rep:
                times.append(a.elapsed_time(b))
        return round(statistics.median(times), 4)

    rows = []
    for name, M, k, c, cost, par, B, n in shapes:
        keys = bc.generate_keys(n, 31)
        negatives = bc.generate_keys(n, 32)
        bitmap = torch.empty((n + 63) // 64, dtype=torch.int64, device="cuda")
        row = {"shape": name, "M": M, "k": k, "c": c, "B": B, "n": n}
        f = bc.Filter(M, k, c, cost, par, hash_seed=9, batch=B, stream=s)
        f.set_tuning(cluster_max=0)
        words = {}
        for mode in (0, 1, 2):
            f.set_tuning(set_mode=mode)

            def ins():
                f.clear(s)
                f.insert(keys, s)
            row["set_mode%d_insert_ms" % mode] = timed(ins)
            words[mode] = f.words_host()
        row["set_modes_identical"] = bool(np.array_equal(words[0], words[1]) and np.array_equal(words[0], words[2]))
        row["fastest_set_mode"] = min((0, 1, 2), key=lambda m: row["set_mode%d_insert_ms" % m])
        f.close()
        if not (name == shapes[0][0] or B == M // 2):  # bit selection: the DNA shape and B = M / 2
            rows.append(row)
            del keys, negatives, bitmap
            torch.cuda.empty_cache()
            continue
        for bitsel in (0, 1):
            g = bc.Filter(M, k, c, cost, par, hash_seed=9, batch=B, stream=s, bitsel=bitsel)
            g.set_tuning(cluster_max=0)

            def ins_g():
                g.clear(s)
                g.insert(keys, s)
            row["bitsel%d_insert_ms" % bitsel] = timed(ins_g)
            row["bitsel%d_query_ms" % bitsel] = timed(lambda: g.query(negatives, bitmap, s))
            g.close()
        rows.append(row)
        del keys, negatives, bitmap
        torch.cuda.empty_cache()
    emit({"workload": "set_and_bit_selection_variants", "rows": rows,
                      "timing": "CUDA events, median of --steps after one warm-up"})


def run_figures(args):
    """Paper-scale FPR and load sweeps on the device (keys generated there):
    fig4 = log2 FPR vs relative size for c = 1, 2, 3 and random/distinct bits
    (Section 4.1, Fig. 4); fig10 = log2 FPR vs the parameter of each cost at
    the standard Bloom size (Appendix C, Fig. 10); fig8 = load histograms
    (Appendix C, Fig. 8). One JSON line per point, then a summary line."""
    import torch
    from paper_2501_18977_gb300 import sweeps
    n = int(args.keys)
    ks = tuple(int(v) for v in args.ks.split(","))
    t0 = time.perf_counter()
    keys_done = [0]

    def log(r):
        r = dict(r)
        hist = r.pop("hist", None)
        if hist is not None:
            r["hist_nonzero"] = {str(L): h for L, h in enumerate(hist) if h}
        keys_done[0] += r["n"] + r["N"]
        emit(r)

    if args.workload == "fig4":
        rows = sweeps.fig4(n=n, ks=ks, log=log)
    elif args.workload == "fig10":
        rows = sweeps.fig10(n=n, ks=ks, runs=tuple(range(1, args.runs + 1)), log=log)
    else:
        rows = sweeps.fig8(n=n, log=log)
    wall = time.perf_counter() - t0
    dev_s = sum(r["insert_ms"] + r["query_ms"] for r in rows) / 1e3

    def l2(r):
        return round(r["log2_fpr"], 3) if r["log2_fpr"] is not None else None

    if args.workload == "fig4":
        cols = ["k", "rel_size", "bitsel", "c", "log2_fpr", "log2_bloom_formula"]
        table = [[r["k"], r["rel_size"], r["bitsel"], r["c"], l2(r), round(math.log2(r["bloom_fpr"]), 3)]
                 for r in rows]
    elif args.workload == "fig10":
        cols = ["k", "cost", "param", "c", "bitsel", "run", "log2_fpr"]
        table = [[r["k"], r["cost"], round(r["param"], 4), r["c"], r["bitsel"], r["run"], l2(r)] for r in rows]
    else:
        cols = ["k", "cost", "param", "c", "load_mean", "load_sd", "log2_fpr"]
        table = [[r["k"], r["cost"], round(r["param"], 4), r["c"], round(r["load_mean"], 2),
                  round(r["load_sd"], 2), l2(r)] for r in rows]
    emit({"workload": args.workload, "points": len(rows), "keys_per_point": n,
                      "device_s": round(dev_s, 3), "wall_s": round(wall, 3),
                      "gkeys_per_s_device": round(keys_done[0] / dev_s / 1e9, 3),
                      "gpu": torch.cuda.get_device_name(), "columns": cols, "table": table})


def main():
    global _WORKLOAD_CLOCKS
    args = parse()
    if args.workload != "dna" and args.impl != "reference":
        _WORKLOAD_CLOCKS = ClockSampler(0)
        _WORKLOAD_CLOCKS.start()
    try:
        run_main(args)
    finally:
        if _WORKLOAD_CLOCKS is not None:
            _WORKLOAD_CLOCKS.stop()


def run_main(args):
    if args.workload in ("fig4", "fig8", "fig10"):
        run_figures(args)
        return
    if args.workload == "cluster":
        run_cluster(args)
        return
    if args.workload == "lanes":
        run_lanes(args)
        return
    if args.workload == "variants":
        run_variants(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "gather":
        run_gather(args)
        return
    if args.workload == "hbm":
        import torch
        import paper_2501_18977_gb300 as bc
        peak, _ = peaks()
        emit(hbm_resident(bc, torch, peak, 0, reps=args.reps))
        return
    if args.workload == "many":
        run_many(args)
        return
    if args.workload == "shard":
        run_shard(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    if args.workload == "sweep":
        run_sweep(args)
        return
    if args.workload == "batching":
        run_batching(args)
        return
    if args.workload == "small":
        run_small(args)
        return
    if args.workload == "learn":
        run_learn(args)
        return
    import torch
    import torch.distributed as dist
    import paper_2501_18977_gb300 as bc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    keys, queries = make_workload()
    n_ins, n_q = len(keys), len(queries)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dq = torch.from_numpy(queries.view(np.int64)).cuda()
    nwords = (n_q + 63) // 64
    bitmap = torch.empty(nwords, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    f = bc.Filter(CONFIG["nblocks"], CONFIG["k"], CONFIG["choices"], bc.COST_LA, CONFIG["mu"],
                  hash_seed=CONFIG["hash_seed"], batch=CONFIG["batch"], stream=stream)

    ev = []
    # Each step's statistics are queued into a pinned buffer (two, alternating)
    # with no host wait, so the host queues the timed steps ahead of the GPU:
    # the machine's host side pauses now and then for tens of milliseconds (seen
    # about every 0.5 s), which a per-step host wait turned into idle GPU time.
    raws = [torch.zeros(bc.STATS_RAW_WORDS, dtype=torch.int64).pin_memory() for _ in range(2)]
    nstep = [0]

    def step(record):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if record else None
        if record:
            e[0].record(stream)
        f.clear(stream)
        f.insert(dk, stream)
        if record:
            e[1].record(stream)
        f.query(dq, bitmap, stream)
        if record:
            e[2].record(stream)
        raw = f.stats_async(raws[nstep[0] % 2], stream)
        nstep[0] += 1
        if record:
            e[3].record(stream)
            ev.append(e)
        return raw

    # the sampler starts before the warm-up and stops after the last timed
    # region: its start-up and shutdown take the driver's locks and once
    # stalled a timed step by about 200 ms
    clocks = ClockSampler(local)
    clocks.start(settle_s=5.0)
    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    launches0 = bc.blowchoc_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        raw = step(True)
    t_end.record(stream)
    torch.cuda.synchronize()
    st = f.stats_decode(raw)
    barrier()
    launches = bc.blowchoc_launch_count() - launches0
    ms = max_over_ranks(t_start.elapsed_time(t_end) / args.steps, world, "cuda")
    value = job_mkeys_per_s(n_ins + n_q, world, ms)

    ins_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    qry_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    sta_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in ev)
    skip_rate = st.skipped / max(1, st.inserted + st.skipped)

    # roofline of the query kernel (one launch per step) against HBM
    c = CONFIG["choices"]
    pbar, pbar_src = golden_pbar()
    q_bytes = n_ins * (8 + 64 * pbar + 1 / 8) + (n_q - n_ins) * (8 + 64 * c + 1 / 8)
    i_bytes = n_ins * (8 + 64 * c + 64 * (1 - skip_rate))
    peak, peak_src = peaks()
    q_gbs = q_bytes / (qry_ms / 1e3) / 1e9
    i_gbs = i_bytes / (ins_ms / 1e3) / 1e9
    hits = None

    e2e = None
    if not args.no_e2e:
        h_keys = torch.from_numpy(keys.view(np.int64)).pin_memory()
        h_q = torch.from_numpy(queries.view(np.int64)).pin_memory()
        h_bm = torch.empty(nwords, dtype=torch.int64).pin_memory()

        h_bm_np = h_bm.numpy().view(np.uint64)

        def e2e_step():
            # the library's host-buffer calls: keys copied in chunks that
            # overlap the previous chunk's kernels, bitmap and statistics
            # copied back; the host waits once, after the last timed step
            f.clear(stream)
            f.insert_host(h_keys, stream)
            f.query_host(h_q, h_bm_np, stream)
            raw = f.stats_async(raws[nstep[0] % 2], stream)
            nstep[0] += 1
            return raw

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        a.record(stream)
        marks[0].record(stream)
        for i in range(args.steps):
            raw_e = e2e_step()
            marks[i + 1].record(stream)
        b.record(stream)
        torch.cuda.synchronize()
        st_e = f.stats_decode(raw_e)
        barrier()
        ems = max_over_ranks(a.elapsed_time(b) / args.steps, world, "cuda")
        per_step = sorted(marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps))
        hits = int(np.unpackbits(h_bm.numpy().view(np.uint8), bitorder="little")[:n_q].sum())
        # the copy ceiling of the same step: the pinned host-to-device rate of
        # one plain copy of the step's keys, best of 3, on this machine
        h2d_ms = None
        for _ in range(4):
            a.record(stream)
            dk.copy_(h_keys, non_blocking=True)
            dq.copy_(h_q, non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b)
            h2d_ms = t if h2d_ms is None else min(h2d_ms, t)
        e2e = {"value": round(job_mkeys_per_s(n_ins + n_q, world, ems), 3), "unit": "Mkeys/s",
               "h2d_bytes_per_step": int(8 * (n_ins + n_q)), "d2h_bytes_per_step": int(8 * nwords + 8 * bc.STATS_RAW_WORDS),
               "ms_per_step": round(ems, 3),
               "ms_per_step_min_median_max": [round(per_step[0], 3), round(statistics.median(per_step), 3),
                                              round(per_step[-1], 3)],
               "api": "blowchoc_insert_host + blowchoc_query_host (pinned) + blowchoc_stats_async",
               "query_hits": hits, "inserted": st_e.inserted, "skipped": st_e.skipped,
               "h2d_gbs": round(8 * (n_ins + n_q) / (h2d_ms / 1e3) / 1e9, 1),
               "copy_floor_ms": round(h2d_ms, 3),
               "frac_of_copy_floor": round(h2d_ms / ems, 4),
               "copy_floor_note": "pinned host-to-device copy of the step's 1.2 GB of keys alone (best of 3); "
                                  "the step cannot end before it"}
    clk = clocks.stop()

    if rank != 0:
        f.close()
        if world > 1:
            dist.destroy_process_group()
        return

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(keys, queries, 800_000, 1_600_000)

    dominant = "query_kernel" if qry_ms >= ins_ms else "persistent_insert_kernel"
    dom_ms = qry_ms if dominant == "query_kernel" else ins_ms
    dom_gbs = q_gbs if dominant == "query_kernel" else i_gbs
    traffic = ncu_traffic(dominant, f.tuning())
    if args.no_extra_records:
        ceil_filter, ceil_filter_cfg, ceil_hbm, hbm = None, (None, None, None), None, None
    else:
        ceil_filter, ceil_filter_cfg = gather_ceiling(bc, torch, CONFIG["nblocks"])
        ceil_hbm, _ = gather_ceiling(bc, torch, 1 << 26)
        hbm = hbm_resident(bc, torch, peak, local)
    out = {
        "metric": "insert+query throughput (DNA 31-mers, c=3, k=16, cost^LA)",
        "value": round(value, 3), "unit": "Mkeys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": dict(CONFIG, n_insert=n_ins, n_query=n_q, parallelism="replicas",
                       l2="inputs larger than L2 (1.2 GB of keys per step); filter cleared at step start"),
        "insert_mkeys_s": round(n_ins / (ins_ms / 1e3) / 1e6, 2),
        "query_mkeys_s": round(n_q / (qry_ms / 1e3) / 1e6, 2),
        "phase_ms": {"clear+insert": round(ins_ms, 4), "query": round(qry_ms, 4),
                     "stats": round(sta_ms, 4)},
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": round(dom_gbs, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(dom_gbs / peak, 4),
                     "traffic": (round(traffic / 1e9, 4) if traffic else None),
                     "traffic_unit": "GB per launch (ncu dram read+write)",
                     "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs, copy)",
                     "launch_ms": round(dom_ms, 4), "pbar": pbar, "pbar_source": pbar_src,
                     "residency": ("L2-assisted: the 128 MiB filter is about L2's size, so part of "
                                   "its block reads hit L2; see hbm_resident for a filter four "
                                   "times L2"),
                     "frac_of_gather_ceiling": ratio(dom_gbs, ceil_filter),
                     "gather_ceiling_gbs": {"filter_footprint_128MiB": rounded(ceil_filter, 1),
                                            "filter_footprint_config": {
                                                "lanes": ceil_filter_cfg[0],
                                                "ctas_per_sm": ceil_filter_cfg[1],
                                                "inflight": ceil_filter_cfg[2]},
                                            "hbm_4GiB": rounded(ceil_hbm, 1)}},
        "hbm_resident": hbm,
        "roofline_other": {"insert_gbs": round(i_gbs, 1), "insert_frac": round(i_gbs / peak, 4),
                           "query_gbs": round(q_gbs, 1), "query_frac": round(q_gbs / peak, 4),
                           "insert_frac_of_gather_ceiling": ratio(i_gbs, ceil_filter),
                           "query_frac_of_gather_ceiling": ratio(q_gbs, ceil_filter)},
        "skip_rate": round(skip_rate, 6), "inserted": st.inserted, "skipped": st.skipped,
        "query_hits": hits, "fpr_est": st.fpr_est,
        "gpu_launches": int(launches),
        "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
    }
    f.close()
    print(json.dumps(finite(out), allow_nan=False))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
