"""abx: BVH-driven DBSCAN / friends-of-friends clustering on one GB300 GPU.

A thin Python binding over the C-ABI library ``libabx.so`` (declared in
``include/abx.h``).  Every step of the clustering runs in the library's CUDA
kernels; this package only marshals arguments (torch tensors for device
memory, the current torch stream).  There is no CPU fallback: if the library
is missing or fails to load, every call raises.
"""
from .binding import (  # noqa: F401
    ABX_EBUSY, ABX_ECANCELLED, ABX_ECUDA, ABX_EINTERNAL, ABX_EINVAL, ABX_ENOMEM, ABX_ENOMEM_BUDGET,
    ABX_ENONFINITE, ABX_ETIMEOUT, ABX_OK, AbxError, BVH, Params, Server, ServeConfig, dbscan, dbscan_batch,
    dbscan_host,
    device_status, launch_count, lib, profile_enable, profile_read, status_str,
)
