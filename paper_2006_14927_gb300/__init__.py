"""GB300 (sm_103a) Cherenkov photon-bunch generation and propagation.

The hot path of the paper's CERENK/RAYBND/TELOUT chain as one C-ABI CUDA
library (``libcher.so``, header ``include/cher.h``) with a thin ctypes
binding.  Build the library with :func:`build`.
"""
from ._binding import (CHER_FP32_BULK, CHER_FP64, NSTATS, STAT_NAMES, CherError, Context,
                       HitBuffers, build_curved_tables_host, build_sensitivity_host, build_tables_host,
                       device_tracks, lib,
                       LIB_PATH, SIGNATURES)
from .build import build

__all__ = ["CHER_FP32_BULK", "CHER_FP64", "NSTATS", "STAT_NAMES", "CherError", "Context",
           "HitBuffers", "build_curved_tables_host", "build_sensitivity_host", "build_tables_host", "device_tracks", "lib", "build", "LIB_PATH",
           "SIGNATURES"]
