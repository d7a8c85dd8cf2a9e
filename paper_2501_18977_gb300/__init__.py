"""GB300 (sm_103a) Blocked Bloom filters with choices (arXiv 2501.18977).

The filter lives in device memory and every operation runs in hand-written
CUDA kernels behind the C ABI of include/blowchoc.h; this package is the
Python binding of that ABI and its build step.
"""
from .binding import (  # noqa: F401
    BLOWCHOC_OK, BLOWCHOC_EINVAL, BLOWCHOC_ENOMEM, BLOWCHOC_ECUDA, BLOWCHOC_ETIMEOUT,
    BLOWCHOC_EBUDGET, COST_MIX, COST_LA, COST_EXP, BlowChocError, Filter,
    blowchoc_params, blowchoc_filter_stats, blowchoc_create, blowchoc_insert,
    blowchoc_insert_noalloc, blowchoc_query,
    blowchoc_stats, blowchoc_stats_async, blowchoc_stats_decode, STATS_RAW_WORDS,
    blowchoc_destroy, blowchoc_words, blowchoc_multipliers,
    blowchoc_read_words, blowchoc_write_words, blowchoc_clear, blowchoc_set_cost_table, blowchoc_cost_ranks,
    blowchoc_fpr_estimate, blowchoc_derive_multipliers,
    blowchoc_cluster_ctas,
    blowchoc_query_count, blowchoc_generate_keys, generate_keys, blowchoc_insert_host, blowchoc_query_host,
    blowchoc_l2_residency, blowchoc_last_error, blowchoc_launch_count,
    blowchoc_tuning, blowchoc_get_tuning, blowchoc_set_tuning, blowchoc_gather_probe,
    blowchoc_work, Batch, blowchoc_batch_create, blowchoc_batch_destroy, blowchoc_insert_many,
    blowchoc_query_many, blowchoc_batch_record, blowchoc_batch_replay, blowchoc_batch_get_tuning,
    blowchoc_batch_set_tuning, blowchoc_batch_autotune, Server, blowchoc_server_config,
    blowchoc_class_tuning, blowchoc_batch_size_class, blowchoc_batch_get_class_tuning,
    blowchoc_batch_set_class_tuning, blowchoc_batch_clear_class_tuning, CLASS_CACHE, CLASS_L2, CLASS_SPILL,
    CLASS_HBM, ROUTE_WORKLIST, ROUTE_DIRECT, ROUTE_SORTED, blowchoc_shard_layout,
    blowchoc_shard_partition_scratch, blowchoc_shard_partition, blowchoc_shard_unpermute,
    blowchoc_server_summary, REQ_INSERT, REQ_QUERY, Mlp, blowchoc_insert_sampled,
    blowchoc_barrier_selftest,
    load_library, exported_symbols, LIB_PATH)
