"""GB300 (sm_103a) RAK label propagation and modularity.

RAK / LPA label propagation as studied by Sahu, arXiv 2301.09125 (Sec. 3.2:
weighted label adoption with strict / non-strict ties and a tolerance test;
Sec. 3.3: COPRA and the asynchronous update; Sec. 3.4: SLPA; Sec. 1:
modularity), implemented as CUDA kernels behind the C ABI of ``include/lp.h``
(``liblp.so``).  This package is the thin Python binding of that ABI; build
the library with ``paper_2301_09125_gb300.build.build()``.
"""
from ._binding import (  # noqa: F401
    LP_ASYNC, LP_EINVAL, LP_ECUDA, LP_ENOMEM, LP_ENOTREADY, LP_ETIMEOUT, LP_FLAG_BORROW,
    LP_FLAG_CHECK_SYMMETRIC, LP_FLAG_DEVICE_PTRS, LP_OK, LP_SYNC, SIGNATURES, Graph, LPError,
    load, lp_batch_autotune, lp_batch_create, lp_batch_destroy, lp_batch_labels_get,
    lp_batch_modularity, lp_batch_run, lp_batch_set_buckets, lp_graph_autotune,
    lp_graph_create, lp_graph_set_buckets, lp_graph_destroy, lp_graph_info, lp_labels_get,
    lp_last_error, lp_launch_count, lp_modularity, lp_profile_enable, lp_profile_read,
    lp_profile_reset, lp_rak_history, lp_rak_params, lp_selftest_barrier_timeout,
    lp_rak_params_default, lp_rak_result, lp_rak_run, lp_rak_sweep_noalloc, lp_serve_result,
    lp_copra_params, lp_copra_run, lp_copra_sets_get, lp_probe_gather, lp_slpa_memory_get,
    lp_slpa_params, lp_slpa_run, lp_split_communities,
    lp_server_config, lp_server_config_default, lp_server_create, lp_server_destroy,
    lp_server_drain, lp_server_poll, lp_server_stats, lp_server_submit, lp_tune_result,
    make_params)
