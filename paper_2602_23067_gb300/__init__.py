"""GB300 AES-GCM for FITS data units (the data path of "GpuFitsCrypt").

The computation lives in ``libgcmgpu.so`` (C ABI: ``include/gcmgpu.h``); the
``api`` module is a thin binding that turns tensors, numpy arrays and
``bytes`` into pointers and lengths.  PyTorch is used only for device memory
and streams.  The native library is loaded on first use of the API, and its
absence raises ImportError: there is no fallback implementation.
"""
from __future__ import annotations

_API_NAMES = {
    "Context", "GcmError", "GCM_OK", "GCM_ERR_AUTH", "GCM_MEM_DEVICE", "GCM_MEM_HOST",
    "gcm_ctx_create", "gcm_ctx_destroy", "gcm_encrypt", "gcm_decrypt_verify", "last_error",
    "FitsResult", "GFC_AAD_HEADER", "GFC_AAD_STRUCTURAL", "Server", "HostBuffer", "BatchPlan",
}


def __getattr__(name):
    if name in _API_NAMES:
        from . import api

        return getattr(api, name)
    raise AttributeError(name)
