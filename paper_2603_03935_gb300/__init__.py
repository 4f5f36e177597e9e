"""GB300-native DISC per-frame integration step (arxiv 2603.03935).

The compute path is libdisc.so: hand-written sm_103a CUDA kernels behind the C
ABI of include/disc.h.  This package is a thin ctypes binding with the same
names; it only marshals arguments.  There is no CPU fallback: when the library
is missing, loading fails loudly.
"""
from .binding import (DiscError, DiscGroup, DiscMap, DiscServer, config_default, device_frame, host_frame, lib, pack_key,
                      query_heatmap, status_str, token_stats_static)

__all__ = ["DiscError", "DiscGroup", "DiscMap", "DiscServer", "config_default", "device_frame", "host_frame", "lib",
           "pack_key", "query_heatmap", "status_str", "token_stats_static"]
