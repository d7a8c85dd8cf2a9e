"""Python binding of the C ABI in include/blowchoc.h (argument marshalling only).

Functions keep the C names. Device buffers are passed as torch CUDA tensors
(any 8-byte dtype, contiguous) or as raw integer device addresses; streams as
torch.cuda.Stream, raw cudaStream_t integers, or None for torch's current
stream. Every computation runs in the CUDA library; if it is missing, loading
fails loudly (there is no CPU fallback).
"""
import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libblowchoc.so")

BLOWCHOC_OK = 0
BLOWCHOC_EINVAL = -1
BLOWCHOC_ENOMEM = -2
BLOWCHOC_ECUDA = -3
BLOWCHOC_ETIMEOUT = -4
BLOWCHOC_EBUDGET = -5

COST_MIX, COST_LA, COST_EXP = 0, 1, 2

_ERRNAMES = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "EBUDGET"}


class BlowChocError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("blowchoc error %s (%d): %s" % (_ERRNAMES.get(code, "?"), code, msg))
        self.code = code


class blowchoc_params(ctypes.Structure):
    _fields_ = [("nblocks", ctypes.c_uint64), ("k", ctypes.c_uint32),
                ("choices", ctypes.c_uint32), ("cost", ctypes.c_int32),
                ("bitsel", ctypes.c_uint32), ("cost_param", ctypes.c_double),
                ("hash_seed", ctypes.c_uint64), ("batch", ctypes.c_uint64)]


class blowchoc_filter_stats(ctypes.Structure):
    _fields_ = [("inserted", ctypes.c_uint64), ("skipped", ctypes.c_uint64),
                ("set_bits", ctypes.c_uint64), ("hist", ctypes.c_uint64 * 513),
                ("fpr_est", ctypes.c_double)]


class blowchoc_tuning(ctypes.Structure):
    _fields_ = [("lanes_choose", ctypes.c_uint32), ("lanes_set", ctypes.c_uint32),
                ("lanes_query", ctypes.c_uint32), ("query_early", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("persistent", ctypes.c_uint32),
                ("keys_per_cta", ctypes.c_uint32), ("set_mode", ctypes.c_uint32),
                ("seq_window", ctypes.c_uint32), ("cluster_max", ctypes.c_uint32),
                ("lanes_cluster", ctypes.c_uint32), ("cluster_keys", ctypes.c_uint32),
                ("host_ring_keys", ctypes.c_uint32)]


class blowchoc_class_tuning(ctypes.Structure):
    _fields_ = [("route", ctypes.c_uint32), ("lanes_choose", ctypes.c_uint32), ("tile", ctypes.c_uint32),
                ("lanes_query", ctypes.c_uint32), ("query_early", ctypes.c_uint32)]


class blowchoc_work(ctypes.Structure):
    _fields_ = [("filter", ctypes.c_void_p), ("d_keys", ctypes.c_void_p),
                ("n", ctypes.c_uint64), ("d_bitmap", ctypes.c_void_p)]


class blowchoc_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("staging_bytes", ctypes.c_uint64),
                ("streams", ctypes.c_uint32), ("max_wave_requests", ctypes.c_uint32)]


class blowchoc_server_summary(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("keys", ctypes.c_uint64), ("waves", ctypes.c_uint64),
                ("first_arrival_s", ctypes.c_double), ("last_done_s", ctypes.c_double),
                ("p50_latency_s", ctypes.c_double), ("p99_latency_s", ctypes.c_double),
                ("max_latency_s", ctypes.c_double), ("mean_wave_requests", ctypes.c_double),
                ("max_filter_bytes_used", ctypes.c_uint64), ("filters_admitted", ctypes.c_uint32),
                ("filters_pending", ctypes.c_uint32), ("mean_wave_gpu_ms", ctypes.c_double),
                ("launch_host_s", ctypes.c_double)]


REQ_INSERT, REQ_QUERY = 0, 1

# name -> (argtypes, restype)
_VP, _U64, _I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
_SIGS = {
    "blowchoc_create": ([ctypes.POINTER(blowchoc_params), _VP, ctypes.POINTER(_VP)], _I),
    "blowchoc_insert": ([_VP, _VP, _U64, _VP], _I),
    "blowchoc_insert_noalloc": ([_VP, _VP, _U64, _VP], _I),
    "blowchoc_query": ([_VP, _VP, _U64, _VP, _VP], _I),
    "blowchoc_stats": ([_VP, ctypes.POINTER(blowchoc_filter_stats)], _I),
    "blowchoc_stats_async": ([_VP, _VP, _VP], _I),
    "blowchoc_stats_decode": ([_VP, _VP, ctypes.POINTER(blowchoc_filter_stats)], _I),
    "blowchoc_destroy": ([_VP], _I),
    "blowchoc_words": ([_VP, ctypes.POINTER(_VP), ctypes.POINTER(_U64)], _I),
    "blowchoc_multipliers": ([_VP, _VP, _VP], _I),
    "blowchoc_read_words": ([_VP, _U64, _U64, _VP], _I),
    "blowchoc_write_words": ([_VP, _U64, _U64, _VP], _I),
    "blowchoc_clear": ([_VP, _VP], _I),
    "blowchoc_set_cost_table": ([_VP, _VP], _I),
    "blowchoc_cost_ranks": ([ctypes.c_int, ctypes.c_double, ctypes.c_uint32, _VP, ctypes.c_uint64], _I),
    "blowchoc_fpr_estimate": ([_VP, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _VP], _I),
    "blowchoc_derive_multipliers": ([_VP, _VP, _VP], _I),
    "blowchoc_l2_residency": ([_VP, ctypes.c_double, _VP], _I),
    "blowchoc_last_error": ([], ctypes.c_char_p),
    "blowchoc_launch_count": ([], ctypes.c_uint64),
    "blowchoc_cluster_ctas": ([_VP, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint32)], _I),
    "blowchoc_query_count": ([_VP, _VP, ctypes.c_uint64, _VP, _VP], _I),
    "blowchoc_insert_host": ([_VP, _VP, ctypes.c_uint64, _VP], _I),
    "blowchoc_query_host": ([_VP, _VP, ctypes.c_uint64, _VP, _VP], _I),
    "blowchoc_generate_keys": ([_VP, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _VP], _I),
    "blowchoc_batch_create": ([ctypes.POINTER(_VP)], _I),
    "blowchoc_batch_destroy": ([_VP], _I),
    "blowchoc_insert_many": ([_VP, ctypes.POINTER(blowchoc_work), ctypes.c_uint32, _VP], _I),
    "blowchoc_query_many": ([_VP, ctypes.POINTER(blowchoc_work), ctypes.c_uint32, _VP], _I),
    "blowchoc_batch_record": ([_VP, ctypes.POINTER(blowchoc_work), ctypes.c_uint32,
                               ctypes.POINTER(blowchoc_work), ctypes.c_uint32], _I),
    "blowchoc_batch_replay": ([_VP, _VP], _I),
    "blowchoc_batch_get_tuning": ([_VP, ctypes.POINTER(blowchoc_tuning)], _I),
    "blowchoc_batch_set_tuning": ([_VP, ctypes.POINTER(blowchoc_tuning)], _I),
    "blowchoc_batch_autotune": ([_VP, ctypes.POINTER(blowchoc_work), ctypes.c_uint32,
                                 ctypes.POINTER(blowchoc_work), ctypes.c_uint32, _VP,
                                 ctypes.POINTER(blowchoc_tuning)], _I),
    "blowchoc_shard_layout": ([_U64, ctypes.c_uint32, _U64, ctypes.POINTER(_U64), ctypes.POINTER(_U64),
                               ctypes.POINTER(_U64)], _I),
    "blowchoc_shard_partition_scratch": ([_U64, ctypes.c_uint32, ctypes.POINTER(_U64)], _I),
    "blowchoc_shard_partition": ([_VP, _U64, ctypes.c_uint32, _U64, _VP, _VP, _VP, _VP, _U64, _VP], _I),
    "blowchoc_shard_unpermute": ([_VP, _VP, _VP, _U64, ctypes.c_uint32, _VP, _VP], _I),
    "blowchoc_batch_size_class": ([_VP, _U64, ctypes.POINTER(ctypes.c_uint32)], _I),
    "blowchoc_batch_get_class_tuning": ([_VP, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.POINTER(blowchoc_class_tuning), ctypes.POINTER(ctypes.c_uint32)], _I),
    "blowchoc_batch_set_class_tuning": ([_VP, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.POINTER(blowchoc_class_tuning)], _I),
    "blowchoc_batch_clear_class_tuning": ([_VP], _I),
    "blowchoc_server_create": ([ctypes.POINTER(blowchoc_server_config), ctypes.POINTER(_VP)], _I),
    "blowchoc_server_add_filter": ([_VP, ctypes.POINTER(blowchoc_params), ctypes.POINTER(ctypes.c_uint32)], _I),
    "blowchoc_server_remove_filter": ([_VP, ctypes.c_uint32], _I),
    "blowchoc_server_submit": ([_VP, ctypes.c_uint32, ctypes.c_uint32, _VP, _U64, _VP, ctypes.c_double,
                                ctypes.POINTER(_U64)], _I),
    "blowchoc_server_start": ([_VP], _I),
    "blowchoc_server_set_tuning": ([_VP, ctypes.POINTER(blowchoc_tuning)], _I),
    "blowchoc_server_wait": ([_VP, ctypes.c_double], _I),
    "blowchoc_server_request_times": ([_VP, _U64, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], _I),
    "blowchoc_server_stats": ([_VP, ctypes.POINTER(blowchoc_server_summary)], _I),
    "blowchoc_server_filter": ([_VP, ctypes.c_uint32, ctypes.POINTER(_VP)], _I),
    "blowchoc_server_destroy": ([_VP], _I),
    "blowchoc_mlp_create": ([ctypes.c_uint32, _U64, ctypes.POINTER(_VP)], _I),
    "blowchoc_mlp_destroy": ([_VP], _I),
    "blowchoc_mlp_param_count": ([], ctypes.c_uint32),
    "blowchoc_mlp_get_params": ([_VP, _VP, _VP], _I),
    "blowchoc_mlp_set_params": ([_VP, _VP], _I),
    "blowchoc_mlp_forward": ([_VP, _VP, _VP], _I),
    "blowchoc_mlp_backward": ([_VP, _VP, ctypes.c_uint32, _VP, _VP], _I),
    "blowchoc_mlp_adam_step": ([_VP, ctypes.c_float, _VP], _I),
    "blowchoc_insert_sampled": ([_VP, _VP, _U64, _VP, ctypes.c_float, _U64, _VP, _VP, _VP], _I),
    "blowchoc_barrier_selftest": ([ctypes.c_uint32, ctypes.c_double, _VP], _I),
    "blowchoc_gather_probe": ([_VP, _U64, _U64, _U64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                               _VP, _VP], _I),
    "blowchoc_get_tuning": ([_VP, ctypes.POINTER(blowchoc_tuning)], _I),
    "blowchoc_set_tuning": ([_VP, ctypes.POINTER(blowchoc_tuning)], _I),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libblowchoc.so (built by the package's build step)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing: run __graft_entry__.build() "
                           "(there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    """Names the binding expects the library to export."""
    return sorted(_SIGS)


def _check(rc):
    if rc != BLOWCHOC_OK:
        raise BlowChocError(rc, load_library().blowchoc_last_error().decode())


def _dev_ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if x.element_size() != 8 or not x.is_contiguous():
            raise ValueError("expected a contiguous tensor of 8-byte elements")
        return x.data_ptr()
    raise TypeError("expected a torch CUDA tensor or an integer device address")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def blowchoc_create(params: blowchoc_params, stream=None):
    h = _VP()
    _check(load_library().blowchoc_create(ctypes.byref(params), _stream(stream), ctypes.byref(h)))
    return h


def blowchoc_insert(f, d_keys, n: int, stream=None):
    _check(load_library().blowchoc_insert(f, _dev_ptr(d_keys), int(n), _stream(stream)))


def blowchoc_insert_noalloc(f, d_keys, n: int, stream=None):
    _check(load_library().blowchoc_insert_noalloc(f, _dev_ptr(d_keys), int(n), _stream(stream)))


def blowchoc_query(f, d_keys, n: int, d_bitmap, stream=None):
    _check(load_library().blowchoc_query(f, _dev_ptr(d_keys), int(n), _dev_ptr(d_bitmap),
                                         _stream(stream)))


def blowchoc_stats(f) -> blowchoc_filter_stats:
    out = blowchoc_filter_stats()
    _check(load_library().blowchoc_stats(f, ctypes.byref(out)))
    return out


STATS_RAW_WORDS = 516


def blowchoc_stats_async(f, h_raw, stream=None):
    """Queue the histogram and the copy of the raw counters into h_raw (host,
    STATS_RAW_WORDS uint64; pinned for an asynchronous copy) on `stream`."""
    n = h_raw.numel() if hasattr(h_raw, "numel") else h_raw.size
    if n < STATS_RAW_WORDS:
        raise ValueError("h_raw holds %d words; the counters need %d" % (n, STATS_RAW_WORDS))
    _check(load_library().blowchoc_stats_async(f, _host_ptr(h_raw), _stream(stream)))


def blowchoc_stats_decode(f, h_raw) -> blowchoc_filter_stats:
    n = h_raw.numel() if hasattr(h_raw, "numel") else h_raw.size
    if n < STATS_RAW_WORDS:
        raise ValueError("h_raw holds %d words; the counters need %d" % (n, STATS_RAW_WORDS))
    out = blowchoc_filter_stats()
    _check(load_library().blowchoc_stats_decode(f, _host_ptr(h_raw), ctypes.byref(out)))
    return out


def blowchoc_destroy(f):
    _check(load_library().blowchoc_destroy(f))


def blowchoc_words(f):
    p, n = _VP(), _U64()
    _check(load_library().blowchoc_words(f, ctypes.byref(p), ctypes.byref(n)))
    return p.value, n.value


def blowchoc_multipliers(f):
    a_block = (ctypes.c_uint64 * 3)()
    a_bit = (ctypes.c_uint64 * 32)()
    _check(load_library().blowchoc_multipliers(f, a_block, a_bit))
    return list(a_block), list(a_bit)


def blowchoc_derive_multipliers(nblocks: int, k: int, choices: int, hash_seed: int, bitsel: int = 0):
    """The multipliers (a_block[:choices], a_bit[:k]) a filter with these
    parameters will use; host-only."""
    p = blowchoc_params(nblocks=int(nblocks), k=int(k), choices=int(choices), cost=COST_EXP, bitsel=int(bitsel),
                        cost_param=(1 + 5 ** 0.5) / 2, hash_seed=int(hash_seed), batch=1)
    a_block = (ctypes.c_uint64 * 3)()
    a_bit = (ctypes.c_uint64 * 32)()
    _check(load_library().blowchoc_derive_multipliers(ctypes.byref(p), a_block, a_bit))
    return list(a_block)[:int(choices)], list(a_bit)[:int(k)]


def blowchoc_read_words(f, first: int, count: int, h_dst):
    """h_dst: a writable host buffer (numpy uint64 array) of >= count words."""
    _check(load_library().blowchoc_read_words(f, int(first), int(count), h_dst.ctypes.data))


def blowchoc_write_words(f, first: int, count: int, h_src):
    _check(load_library().blowchoc_write_words(f, int(first), int(count), h_src.ctypes.data))


def blowchoc_set_cost_table(f, costs):
    """costs: numpy float64 array of 513 * (k + 1) values, costs[L * (k + 1) + a]."""
    import numpy as np
    c = np.ascontiguousarray(costs, dtype=np.float64)
    _check(load_library().blowchoc_set_cost_table(f, c.ctypes.data))


def blowchoc_cost_ranks(cost: int, cost_param: float, k: int):
    """The host-side rank table of the costs (numpy uint16, 513 * (k + 1)
    entries, index L * (k + 1) + a; 0xFFFF where L + a > 512)."""
    import numpy as np
    out = np.empty(513 * (int(k) + 1), dtype=np.uint16)
    _check(load_library().blowchoc_cost_ranks(int(cost), float(cost_param), int(k), out.ctypes.data, out.size))
    return out


def blowchoc_fpr_estimate(hist, k: int, choices: int, bitsel: int = 0) -> float:
    """The histogram FPR estimate of blowchoc_stats for a host histogram of
    513 block counts (index = load)."""
    import numpy as np
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    assert h.shape == (513,)
    out = ctypes.c_double()
    _check(load_library().blowchoc_fpr_estimate(h.ctypes.data, int(k), int(choices), int(bitsel),
                                                 ctypes.byref(out)))
    return float(out.value)


def blowchoc_l2_residency(f, fraction, stream):
    _check(load_library().blowchoc_l2_residency(f, float(fraction), _stream(stream)))


def blowchoc_clear(f, stream=None):
    _check(load_library().blowchoc_clear(f, _stream(stream)))


def _host_ptr(a):
    """Address of a host uint64 buffer: a numpy array or a CPU torch tensor."""
    if hasattr(a, "data_ptr"):
        assert not a.is_cuda and a.is_contiguous() and a.element_size() == 8
        return a.data_ptr()
    import numpy as np
    assert isinstance(a, np.ndarray) and a.dtype.itemsize == 8 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def blowchoc_insert_host(f, h_keys, n: int, stream=None):
    _check(load_library().blowchoc_insert_host(f, _host_ptr(h_keys), int(n), _stream(stream)))


def blowchoc_query_host(f, h_keys, n: int, h_bitmap, stream=None):
    _check(load_library().blowchoc_query_host(f, _host_ptr(h_keys), int(n), _host_ptr(h_bitmap),
                                              _stream(stream)))


def blowchoc_query_count(f, d_keys, n: int, d_count, stream=None):
    _check(load_library().blowchoc_query_count(f, d_keys, int(n), d_count, _stream(stream)))


def blowchoc_generate_keys(d_out, n: int, seed: int, start: int = 0, stream=None):
    _check(load_library().blowchoc_generate_keys(d_out, int(n), int(seed) & 0xFFFFFFFFFFFFFFFF, int(start),
                                                 _stream(stream)))


def generate_keys(n: int, seed: int, start: int = 0, out=None, stream=None):
    """n splitmix64 keys of `seed` from stream position `start`, generated on
    the current CUDA device into `out` (an int64 tensor) or a new tensor."""
    import torch
    if out is None:
        out = torch.empty(int(n), dtype=torch.int64, device="cuda")
    assert out.dtype == torch.int64 and out.is_cuda and out.is_contiguous() and out.numel() >= n
    blowchoc_generate_keys(out.data_ptr(), n, seed, start, stream)
    return out


def blowchoc_cluster_ctas(f, n: int) -> int:
    out = ctypes.c_uint32()
    _check(load_library().blowchoc_cluster_ctas(f, int(n), ctypes.byref(out)))
    return int(out.value)


def blowchoc_get_tuning(f) -> blowchoc_tuning:
    out = blowchoc_tuning()
    _check(load_library().blowchoc_get_tuning(f, ctypes.byref(out)))
    return out


def blowchoc_set_tuning(f, t: blowchoc_tuning):
    _check(load_library().blowchoc_set_tuning(f, ctypes.byref(t)))


def blowchoc_gather_probe(d_words, nblocks: int, nreads: int, seed: int, lanes: int,
                          ctas_per_sm: int, d_sink, stream=None, inflight: int = 1):
    _check(load_library().blowchoc_gather_probe(_dev_ptr(d_words), int(nblocks), int(nreads),
                                                int(seed), int(lanes), int(ctas_per_sm), int(inflight),
                                                _dev_ptr(d_sink), _stream(stream)))


def _works(items):
    """items: list of (filter handle or Filter, keys tensor/ptr, n, bitmap or None)."""
    arr = (blowchoc_work * max(len(items), 1))()
    for i, (f, keys, n, bm) in enumerate(items):
        h = f.handle if hasattr(f, "handle") else f
        arr[i].filter = h.value if hasattr(h, "value") else h
        arr[i].d_keys = _dev_ptr(keys) if n else None
        arr[i].n = int(n)
        arr[i].d_bitmap = _dev_ptr(bm) if bm is not None else None
    return arr, len(items)


def blowchoc_batch_create():
    h = _VP()
    _check(load_library().blowchoc_batch_create(ctypes.byref(h)))
    return h


def blowchoc_batch_destroy(b):
    _check(load_library().blowchoc_batch_destroy(b))


def blowchoc_insert_many(b, items, stream=None):
    arr, n = _works(items)
    _check(load_library().blowchoc_insert_many(b, arr, n, _stream(stream)))


def blowchoc_query_many(b, items, stream=None):
    arr, n = _works(items)
    _check(load_library().blowchoc_query_many(b, arr, n, _stream(stream)))


def blowchoc_batch_record(b, ins, qry):
    a1, n1 = _works(ins)
    a2, n2 = _works(qry)
    _check(load_library().blowchoc_batch_record(b, a1, n1, a2, n2))


def blowchoc_batch_replay(b, stream=None):
    _check(load_library().blowchoc_batch_replay(b, _stream(stream)))


def blowchoc_batch_get_tuning(b) -> blowchoc_tuning:
    out = blowchoc_tuning()
    _check(load_library().blowchoc_batch_get_tuning(b, ctypes.byref(out)))
    return out


def blowchoc_batch_set_tuning(b, t: blowchoc_tuning):
    _check(load_library().blowchoc_batch_set_tuning(b, ctypes.byref(t)))


def blowchoc_batch_autotune(b, ins, qry, stream=None) -> blowchoc_tuning:
    a1, n1 = _works(ins)
    a2, n2 = _works(qry)
    out = blowchoc_tuning()
    _check(load_library().blowchoc_batch_autotune(b, a1, n1, a2, n2, _stream(stream),
                                                  ctypes.byref(out)))
    return out


def blowchoc_shard_layout(nblocks: int, T: int, hash_seed: int):
    """(a_0, blocks per sub-array, hash seed of the sub-arrays) of a filter of
    nblocks blocks split into T sub-arrays (host-only)."""
    a0, ms, seed = _U64(), _U64(), _U64()
    _check(load_library().blowchoc_shard_layout(int(nblocks), int(T), int(hash_seed) & 0xFFFFFFFFFFFFFFFF,
                                                ctypes.byref(a0), ctypes.byref(ms), ctypes.byref(seed)))
    return a0.value, ms.value, seed.value


def blowchoc_shard_partition_scratch(n: int, T: int) -> int:
    out = _U64()
    _check(load_library().blowchoc_shard_partition_scratch(int(n), int(T), ctypes.byref(out)))
    return out.value


def blowchoc_shard_partition(d_keys, n: int, T: int, a0: int, d_out_keys, d_out_index, d_offsets, d_scratch,
                             scratch_words: int, stream=None):
    _check(load_library().blowchoc_shard_partition(_dev_ptr(d_keys), int(n), int(T), int(a0), _dev_ptr(d_out_keys),
                                                   _dev_ptr(d_out_index), _dev_ptr(d_offsets), _dev_ptr(d_scratch),
                                                   int(scratch_words), _stream(stream)))


def blowchoc_shard_unpermute(d_seg_bits, d_offsets, d_index, n: int, T: int, d_bitmap, stream=None):
    _check(load_library().blowchoc_shard_unpermute(_dev_ptr(d_seg_bits), _dev_ptr(d_offsets), _dev_ptr(d_index),
                                                   int(n), int(T), _dev_ptr(d_bitmap), _stream(stream)))


CLASS_CACHE, CLASS_L2, CLASS_SPILL, CLASS_HBM = 0, 1, 2, 3
ROUTE_WORKLIST, ROUTE_DIRECT, ROUTE_SORTED = 0, 1, 2


def blowchoc_batch_size_class(b, nblocks: int) -> int:
    out = ctypes.c_uint32()
    _check(load_library().blowchoc_batch_size_class(b, int(nblocks), ctypes.byref(out)))
    return out.value


def blowchoc_batch_get_class_tuning(b, cls: int, k: int, c: int):
    """(blowchoc_class_tuning, is_set) of (size class, k, c)."""
    out = blowchoc_class_tuning()
    is_set = ctypes.c_uint32()
    _check(load_library().blowchoc_batch_get_class_tuning(b, int(cls), int(k), int(c), ctypes.byref(out),
                                                          ctypes.byref(is_set)))
    return out, bool(is_set.value)


def blowchoc_batch_set_class_tuning(b, cls: int, k: int, c: int, t: blowchoc_class_tuning):
    _check(load_library().blowchoc_batch_set_class_tuning(b, int(cls), int(k), int(c), ctypes.byref(t)))


def blowchoc_batch_clear_class_tuning(b):
    _check(load_library().blowchoc_batch_clear_class_tuning(b))


class Batch:
    """Owning handle of a many-filter batch object."""

    def __init__(self):
        self.handle = blowchoc_batch_create()

    def close(self):
        if self.handle is not None and self.handle.value:
            blowchoc_batch_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def insert_many(self, items, stream=None):
        blowchoc_insert_many(self.handle, items, stream)

    def query_many(self, items, stream=None):
        blowchoc_query_many(self.handle, items, stream)

    def record(self, ins, qry):
        blowchoc_batch_record(self.handle, ins, qry)

    def replay(self, stream=None):
        blowchoc_batch_replay(self.handle, stream)

    def tuning(self):
        return blowchoc_batch_get_tuning(self.handle)

    def set_tuning(self, **kw):
        t = blowchoc_batch_get_tuning(self.handle)
        for k, v in kw.items():
            setattr(t, k, int(v))
        blowchoc_batch_set_tuning(self.handle, t)

    def autotune(self, ins, qry, stream=None):
        return blowchoc_batch_autotune(self.handle, ins, qry, stream)

    def size_class(self, nblocks):
        return blowchoc_batch_size_class(self.handle, nblocks)

    def class_tuning(self, cls, k, c):
        """(fields as a dict, is_set) of (size class, k, c)."""
        t, is_set = blowchoc_batch_get_class_tuning(self.handle, cls, k, c)
        return {name: int(getattr(t, name)) for name, _ in t._fields_}, is_set

    def set_class_tuning(self, cls, k, c, **kw):
        t, _ = blowchoc_batch_get_class_tuning(self.handle, cls, k, c)
        for name, v in kw.items():
            setattr(t, name, int(v))
        blowchoc_batch_set_class_tuning(self.handle, cls, k, c, t)

    def clear_class_tuning(self):
        blowchoc_batch_clear_class_tuning(self.handle)


class Server:
    """Request-serving loop (blowchoc_server_*). Host key and bitmap buffers
    are numpy uint64 arrays (pinned torch tensors also work via .numpy());
    the caller keeps them alive until wait() returns."""

    def __init__(self, hbm_budget_bytes, staging_bytes=1 << 30, streams=4, max_wave_requests=64):
        cfg = blowchoc_server_config(hbm_budget_bytes=int(hbm_budget_bytes),
                                     staging_bytes=int(staging_bytes), streams=int(streams),
                                     max_wave_requests=int(max_wave_requests))
        h = _VP()
        _check(load_library().blowchoc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self._keep = []

    def add_filter(self, nblocks, k, choices, cost, cost_param, hash_seed, batch):
        p = blowchoc_params(nblocks=int(nblocks), k=int(k), choices=int(choices), cost=int(cost),
                            bitsel=0, cost_param=float(cost_param), hash_seed=int(hash_seed),
                            batch=int(batch))
        out = ctypes.c_uint32()
        _check(load_library().blowchoc_server_add_filter(self.handle, ctypes.byref(p), ctypes.byref(out)))
        return out.value

    def remove_filter(self, fid):
        _check(load_library().blowchoc_server_remove_filter(self.handle, int(fid)))

    def submit(self, fid, kind, h_keys, h_bitmap=None, arrival_s=0.0):
        rid = _U64()
        self._keep.append((h_keys, h_bitmap))
        _check(load_library().blowchoc_server_submit(
            self.handle, int(fid), int(kind), h_keys.ctypes.data, len(h_keys),
            h_bitmap.ctypes.data if h_bitmap is not None else None, float(arrival_s), ctypes.byref(rid)))
        return rid.value

    def set_tuning(self, **kw):
        """Launch configuration for the server's filters and many-filter
        calls (before start): the filter defaults with the given fields."""
        probe = Filter(1, 1, 1)
        try:
            t = blowchoc_get_tuning(probe.handle)
        finally:
            probe.close()
        for k, v in kw.items():
            setattr(t, k, int(v))
        _check(load_library().blowchoc_server_set_tuning(self.handle, ctypes.byref(t)))

    def start(self):
        _check(load_library().blowchoc_server_start(self.handle))

    def wait(self, timeout_s=600.0):
        _check(load_library().blowchoc_server_wait(self.handle, float(timeout_s)))

    def request_times(self, rid):
        a, l, d = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(load_library().blowchoc_server_request_times(self.handle, int(rid), ctypes.byref(a),
                                                            ctypes.byref(l), ctypes.byref(d)))
        return a.value, l.value, d.value

    def stats(self):
        out = blowchoc_server_summary()
        _check(load_library().blowchoc_server_stats(self.handle, ctypes.byref(out)))
        return out

    def filter_handle(self, fid):
        h = _VP()
        _check(load_library().blowchoc_server_filter(self.handle, int(fid), ctypes.byref(h)))
        return h

    def words_host(self, fid):
        import numpy as np
        h = self.filter_handle(fid)
        if not h.value:
            return None
        _, n = blowchoc_words(h)
        out = np.empty(n, dtype=np.uint64)
        blowchoc_read_words(h, 0, n, out)
        return out

    def close(self):
        if self.handle is not None and self.handle.value:
            load_library().blowchoc_server_destroy(self.handle)
        self.handle = None
        self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """The learned-cost network (blowchoc_mlp_*)."""

    def __init__(self, k, seed):
        h = _VP()
        _check(load_library().blowchoc_mlp_create(int(k), int(seed), ctypes.byref(h)))
        self.handle = h
        self.k = int(k)
        self.nparams = int(load_library().blowchoc_mlp_param_count())

    def params(self):
        import numpy as np
        p = np.empty(self.nparams, dtype=np.float32)
        _check(load_library().blowchoc_mlp_get_params(self.handle, p.ctypes.data, None))
        return p

    def grad(self):
        import numpy as np
        g = np.empty(self.nparams, dtype=np.float64)
        _check(load_library().blowchoc_mlp_get_params(self.handle, None, g.ctypes.data))
        return g

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(load_library().blowchoc_mlp_set_params(self.handle, p.ctypes.data))

    def forward(self, d_table, stream=None):
        _check(load_library().blowchoc_mlp_forward(self.handle, _dev_ptr_any(d_table), _stream(stream)))

    def backward(self, d_w, d_scales, stream=None):
        """d_w: device float32 rows x 513 (k + 1); d_scales: device float64 rows."""
        rows = d_scales.numel()
        _check(load_library().blowchoc_mlp_backward(self.handle, _dev_ptr_any(d_w), int(rows),
                                                    _dev_ptr_any(d_scales), _stream(stream)))

    def adam_step(self, lr, stream=None):
        _check(load_library().blowchoc_mlp_adam_step(self.handle, float(lr), _stream(stream)))

    def close(self):
        if self.handle is not None and self.handle.value:
            load_library().blowchoc_mlp_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dev_ptr_any(x):
    """Device address of a contiguous CUDA tensor of any dtype (or an int)."""
    if isinstance(x, int):
        return x
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return x.data_ptr()


def blowchoc_insert_sampled(f, d_keys, n, d_table, tau, seed, d_w, d_choice=None, stream=None):
    _check(load_library().blowchoc_insert_sampled(
        f, _dev_ptr(d_keys), int(n), _dev_ptr_any(d_table), float(tau), int(seed), _dev_ptr_any(d_w),
        _dev_ptr_any(d_choice) if d_choice is not None else None, _stream(stream)))


def blowchoc_barrier_selftest(ctas=8, seconds=0.5, stream=None) -> int:
    """Runs the bounded-barrier diagnostic; returns the library's code
    (BLOWCHOC_ETIMEOUT when the bound worked)."""
    return int(load_library().blowchoc_barrier_selftest(int(ctas), float(seconds), _stream(stream)))


def blowchoc_launch_count() -> int:
    return int(load_library().blowchoc_launch_count())


def blowchoc_last_error() -> str:
    return load_library().blowchoc_last_error().decode()


class _CudaArray:
    """Minimal __cuda_array_interface__ holder for a zero-copy torch view."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i8", "data": (ptr, False),
                                         "version": 3, "strides": None}


class Filter:
    """Owning handle around blowchoc_create/destroy with tensor conveniences."""

    def __init__(self, nblocks, k, choices, cost=COST_EXP, cost_param=(1 + 5 ** 0.5) / 2,
                 hash_seed=0, batch=1, stream=None, bitsel=0):
        self.params = blowchoc_params(nblocks=int(nblocks), k=int(k), choices=int(choices),
                                      cost=int(cost), bitsel=int(bitsel), cost_param=float(cost_param),
                                      hash_seed=int(hash_seed), batch=int(batch))
        self.handle = blowchoc_create(self.params, stream)

    def close(self):
        if self.handle is not None and self.handle.value:
            blowchoc_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def insert(self, keys, stream=None):
        blowchoc_insert(self.handle, keys, keys.numel(), stream)

    def query(self, keys, bitmap=None, stream=None):
        import torch
        n = keys.numel()
        if bitmap is None:
            bitmap = torch.empty(max((n + 63) // 64, 1), dtype=torch.int64, device=keys.device)
        blowchoc_query(self.handle, keys, n, bitmap, stream)
        return bitmap[: (n + 63) // 64]

    def stats(self):
        return blowchoc_stats(self.handle)

    def stats_async(self, h_raw, stream=None):
        """Queue the statistics into h_raw (pinned host int64 tensor or numpy
        uint64 array of STATS_RAW_WORDS) on `stream`; decode them with
        stats_decode once the stream has completed."""
        blowchoc_stats_async(self.handle, h_raw, stream)
        return h_raw

    def stats_decode(self, h_raw):
        return blowchoc_stats_decode(self.handle, h_raw)

    def words_view(self):
        """Zero-copy torch int64 view of the filter words (device)."""
        import torch
        p, n = blowchoc_words(self.handle)
        return torch.as_tensor(_CudaArray(p, n), device="cuda")

    def words_host(self):
        import numpy as np
        _, n = blowchoc_words(self.handle)
        out = np.empty(n, dtype=np.uint64)
        blowchoc_read_words(self.handle, 0, n, out)
        return out

    def multipliers(self):
        return blowchoc_multipliers(self.handle)

    def clear(self, stream=None):
        blowchoc_clear(self.handle, stream)

    def set_cost_table(self, costs):
        blowchoc_set_cost_table(self.handle, costs)

    def l2_residency(self, fraction, stream):
        blowchoc_l2_residency(self.handle, fraction, stream)

    def cluster_ctas(self, n):
        return blowchoc_cluster_ctas(self.handle, n)

    def insert_host(self, keys, stream=None):
        """Insert host keys (numpy uint64/int64 array or CPU tensor; pinned
        memory overlaps the copies with the kernels). Ordered on `stream`:
        keep `keys` unchanged until the stream completes."""
        n = keys.numel() if hasattr(keys, "numel") else len(keys)
        blowchoc_insert_host(self.handle, keys, n, stream)

    def query_host(self, keys, bitmap=None, stream=None):
        """Query host keys into a host bitmap (numpy uint64, ceil(n/64)
        words; allocated if None). Complete once `stream` completes."""
        import numpy as np
        n = keys.numel() if hasattr(keys, "numel") else len(keys)
        if bitmap is None:
            bitmap = np.zeros(max(1, (n + 63) // 64), dtype=np.uint64)
        blowchoc_query_host(self.handle, keys, n, bitmap, stream)
        return bitmap

    def query_count(self, keys, count=None, stream=None):
        """Number of `keys` (int64 CUDA tensor) reported present. With a
        one-element int64 CUDA tensor `count`, adds to it asynchronously and
        returns it; otherwise synchronises and returns an int."""
        import torch
        assert keys.dtype == torch.int64 and keys.is_cuda and keys.is_contiguous()
        own = count is None
        if own:
            count = torch.zeros(1, dtype=torch.int64, device=keys.device)
        blowchoc_query_count(self.handle, keys.data_ptr(), keys.numel(), count.data_ptr(), stream)
        if own:
            return int(count.item())
        return count

    def tuning(self):
        return blowchoc_get_tuning(self.handle)

    def set_tuning(self, **kw):
        t = blowchoc_get_tuning(self.handle)
        for k, v in kw.items():
            setattr(t, k, int(v))
        blowchoc_set_tuning(self.handle, t)
