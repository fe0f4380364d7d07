"""GB300-native (sm_103a) UTF-8 / UTF-16LE validation and transcoding.

The work runs in the CUDA library built from ``csrc/`` (C ABI: ``include/gbutf.h``);
``binding`` is a thin ctypes layer over it.
"""
from .binding import (  # noqa: F401
    OP_CODE, OPS, REQ_DISCARD_OUTPUT, Arena, GbuBatchConfig, GbuCompletion, GbuRequest, GbuServerConfig, GbuServerStats, Graph,
    Server, gbu_server_cancel, gbu_server_copy_output, gbu_server_create, gbu_server_default_config, gbu_server_destroy,
    gbu_server_get_stats, gbu_server_now_ns, gbu_server_poll, gbu_server_release, gbu_server_submit, gbu_convert_utf16le_to_utf8_batched,
    gbu_convert_utf8_to_utf16le_batched, gbu_exclusive_scan_u64, gbu_get_batch_config,
    gbu_graph_begin, gbu_graph_destroy, gbu_graph_end, gbu_graph_kernels, gbu_graph_launch,
    gbu_set_batch_config, gbu_tune_batched, gbu_utf16_length_from_utf8_batched,
    gbu_utf8_length_from_utf16le_batched, gbu_validate_utf16le_batched, gbu_validate_utf8_batched,
    NOALLOC_MAX_UNITS, STATUS, STATUS_CODE, Codec, GbuError, GbuResult, gbu_convert_utf16le_to_utf8,
    convert_utf8_to_utf16le_noalloc, gbu_convert_utf8_to_utf16le,
    gbu_convert_utf8_to_utf16le_noalloc, gbu_create, gbu_debug_skip_publish, gbu_destroy,
    gbu_launch_config, gbu_launch_count, gbu_reset, gbu_set_wait_limit, gbu_utf16_length_from_utf8,
    gbu_utf8_length_from_utf16le, gbu_validate_utf16le, gbu_validate_utf8, lib, library_path,
    result_tuple, shard_cuts_host, combine_shards, gbu_set_early_exit, Chunked, Pipe)
