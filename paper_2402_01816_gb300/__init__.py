"""GB300-native stable mergesort after the greeNsort method (arXiv 2402.01816).

The sorting runs in the CUDA library ``_build/libgns.so`` (sources in
``csrc/``, C ABI in ``include/gns.h``); this package only builds it
(``build.build()``) and binds it (``_native``): the Python functions carry the
C entry points' names and do argument marshalling only.  ``inputs`` holds the
seeded synthetic workloads.
"""
from ._native import (ASCENDING, DESCENDING, GNS_ERR_CUDA, GNS_ERR_INVALID, GNS_ERR_OOM,  # noqa: F401
                      GNS_ERR_TIMEOUT, GNS_ERR_UNSUPPORTED, GNS_OK, GnsError, gns_debug_skip_publish,
                      gns_launch_count, gns_profile_enable, gns_profile_read, gns_segmented_release,
                      gns_segmented_schedule, gns_segmented_sort, gns_sort_noalloc,
                      gns_set_wait_limit_ns, gns_sort, gns_sort_host, gns_sort_symmetric,
                      FROGSORT1, GECKOSORT1, SQUIDSORT1, gns_stream_status, gns_version,
                      gns_learned_sort, gns_learned_half_plan_ok, gns_mlp_forward, gns_mlp_init_params, gns_mlp_loss_grad, gns_mlp_train,
                      gns_workspace_bytes, gns_release_workspace_cache, GNS_ERR_INTERNAL, strerror, lib,
                      gns_debug_learned_fault, gns_debug_jitter, gns_debug_merge_partition,
                      gns_debug_ordered_segments, FAULT_NONE, FAULT_BUCKETS_SWAPPED,
                      FAULT_GARBAGE_WEIGHTS, FAULT_SPLITTERS_REVERSED)
