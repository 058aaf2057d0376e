"""GB300 (sm_103a) Count Sketch halo finder: the hot path of arXiv:1711.00975.

The compute lives in libhalosketch.so (hand-written CUDA behind the C ABI of
include/halosketch.h); `halosketch` is its thin ctypes binding.
"""
from .halosketch import (MLP, Batch, HSError, Learned, Sketch, exact_counts, hs_last_error, hs_measure_red_rate, lib, make_params,
                         sketch_counters, sketch_create, sketch_destroy, sketch_flush, sketch_info,
                         sketch_load_counters, sketch_merge, sketch_query, sketch_reset, sketch_seek,
                         sketch_stats, sketch_synchronize, sketch_update, topk_extract)

__all__ = ["MLP", "Batch", "HSError", "Learned", "Sketch", "exact_counts", "hs_last_error", "hs_measure_red_rate", "lib", "make_params",
           "sketch_counters", "sketch_create", "sketch_destroy", "sketch_flush", "sketch_info",
           "sketch_load_counters", "sketch_merge", "sketch_query", "sketch_reset", "sketch_seek", "sketch_stats",
           "sketch_synchronize", "sketch_update", "topk_extract"]
