"""GB300-native per-pixel weighted reservoir sampling for foveated frame streams.

The reservoir update and resolve of "Enhancing Foveated Rendering with
Weighted Reservoir Sampling" (arXiv 2510.03964) as hand-written sm_103a CUDA
kernels behind the C-ABI of include/wrs.h (libwrs.so). This package is the
thin Python face of that library: torch supplies device memory and streams,
the library does all of the work, and nothing falls back to the CPU: without
the built library every call raises.
"""
from ._lib import WrsError, header_functions, load
from .wrs import (Batch, Foveation, HostPipeline, Stream, foveate, make_config, mip_build, mip_layout, mip_levels,
                  state_bytes, state_layout, unpack_state)

__all__ = ["Batch", "Stream", "make_config", "state_bytes", "state_layout", "unpack_state", "WrsError",
           "load", "header_functions", "Foveation", "HostPipeline", "foveate", "mip_build", "mip_layout", "mip_levels"]


def kernel_source_hash() -> str:
    """Hash of the CUDA sources and the public header: ties recorded profiler
    counters to the kernel they were taken on."""
    import glob
    import hashlib
    import os
    from .build import CSRC, INCLUDE
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(CSRC, "*"))) + [os.path.join(INCLUDE, "wrs.h")]:
        if os.path.isfile(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]
