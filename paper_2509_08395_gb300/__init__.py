"""GB300 (sm_103a) implementation of SINDI's sparse MIPS search hot path (arXiv 2509.08395).

The computation lives in hand-written CUDA kernels behind the C ABI of
``include/sindi.h`` (``lib/libsindi.so``); ``sindi`` is its Python binding.
"""
from .sindi import (  # noqa: F401
    ACCUMS,
    DTYPES,
    MODES,
    PRUNES,
    SINDI_SCAN_PIPELINED,
    Index,
    Plan,
    Server,
    SindiError,
    load,
    sindi_build,
    sindi_check,
    sindi_get_stats,
    sindi_index_export,
    sindi_index_free,
    sindi_index_info,
    sindi_index_load,
    sindi_index_save,
    sindi_merge_topk,
    sindi_plan_create,
    sindi_plan_free,
    sindi_plan_launch,
    sindi_reset_stats,
    sindi_search,
    sindi_search_noalloc,
    sindi_server_create,
    sindi_server_destroy,
    sindi_server_poll,
    sindi_server_stats,
    sindi_server_submit,
    sindi_set_timing,
    sindi_version,
)
