"""GB300 AES-GCM for FITS data units (the data path of "GpuFitsCrypt").

The computation lives in ``libgcmgpu.so`` (C ABI: ``include/gcmgpu.h``).  This
package is a thin binding: it turns tensors, numpy arrays and ``bytes`` into
pointers and lengths and maps status codes to exceptions.  PyTorch is used
only for device memory and streams.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

from ._native import (GCM_ERR_AUTH, GCM_MEM_DEVICE, GCM_MEM_HOST, GCM_OK, GcmError, check,
                      gcm_ctx_create, gcm_ctx_destroy, gcm_decrypt_verify, gcm_encrypt, last_error)

__all__ = [
    "Context", "GcmError", "GCM_OK", "GCM_ERR_AUTH", "GCM_MEM_DEVICE", "GCM_MEM_HOST",
    "gcm_ctx_create", "gcm_ctx_destroy", "gcm_encrypt", "gcm_decrypt_verify", "last_error",
]


def _host_buf(data) -> Tuple[int, int, object]:
    """(pointer, length, keepalive) for bytes / bytearray / numpy / CPU tensors."""
    if data is None:
        return 0, 0, None
    if isinstance(data, (bytes, bytearray, memoryview)):
        b = ctypes.create_string_buffer(bytes(data), max(1, len(data)))
        return ctypes.addressof(b), len(data), b
    if hasattr(data, "ctypes") and hasattr(data, "nbytes"):  # numpy
        if not data.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return data.ctypes.data, int(data.nbytes), data
    if hasattr(data, "data_ptr"):  # torch CPU tensor (e.g. pinned)
        if data.is_cuda:
            raise ValueError("expected a host buffer")
        if not data.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return data.data_ptr(), data.numel() * data.element_size(), data
    raise TypeError("unsupported host buffer type %r" % type(data))


def _dev_buf(t) -> Tuple[int, int]:
    if t is None:
        return 0, 0
    if not hasattr(t, "data_ptr") or not t.is_cuda:
        raise TypeError("device mode expects CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return t.data_ptr(), t.numel() * t.element_size()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Context:
    """A library session on one GPU (the paper's gfc_context_create /
    gfc_context_destroy pair)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = device
        self.handle = gcm_ctx_create(device, hbm_budget_bytes)

    def close(self) -> None:
        if self.handle:
            gcm_ctx_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- device-resident data (torch CUDA uint8 tensors) -------------------
    def encrypt_device(self, key: bytes, iv: bytes, aad, pt, ct=None, tag=None, stream=None):
        """Enqueue GCM-AE on device tensors; returns (ct, tag) tensors."""
        import torch

        if ct is None:
            ct = torch.empty_like(pt)
        if tag is None:
            tag = torch.empty(16, dtype=torch.uint8, device=pt.device)
        kp, kl, kk = _host_buf(key)
        ip, il, ik = _host_buf(iv)
        ap, al = _dev_buf(aad)
        pp, pl = _dev_buf(pt)
        cp, cl = _dev_buf(ct)
        tp, tl = _dev_buf(tag)
        if cl < pl or tl < 16:
            raise ValueError("output buffers too small")
        check(gcm_encrypt(self.handle, kp, kl, ip, il, ap, al, pp, pl, cp, tp, GCM_MEM_DEVICE,
                          _stream_handle(stream)))
        return ct, tag

    def decrypt_verify_device(self, key: bytes, iv: bytes, aad, ct, tag, pt=None, stream=None):
        """GCM-AD on device tensors.  Raises GcmError(GCM_ERR_AUTH) on a tag
        mismatch, after the output has been zero-filled on the device."""
        import torch

        if pt is None:
            pt = torch.empty_like(ct)
        kp, kl, kk = _host_buf(key)
        ip, il, ik = _host_buf(iv)
        ap, al = _dev_buf(aad)
        cp, cl = _dev_buf(ct)
        tp, tl = _dev_buf(tag)
        pp, pl = _dev_buf(pt)
        if pl < cl or tl < 16:
            raise ValueError("buffers too small")
        check(gcm_decrypt_verify(self.handle, kp, kl, ip, il, ap, al, cp, cl, tp, pp, GCM_MEM_DEVICE,
                                 _stream_handle(stream)))
        return pt

    # -- host-resident data (bytes / numpy / pinned CPU tensors) ------------
    def encrypt_host(self, key: bytes, iv: bytes, aad, pt, ct=None, stream=0) -> Tuple[object, bytes]:
        """GCM-AE of host data, staged through the device; returns (ct, tag)."""
        import numpy as np

        kp, kl, kk = _host_buf(key)
        ip, il, ik = _host_buf(iv)
        ap, al, ak = _host_buf(aad)
        pp, pl, pk = _host_buf(pt)
        if ct is None:
            ct = np.empty(pl, dtype=np.uint8)
        cp, cl, ck = _host_buf(ct)
        if cl < pl:
            raise ValueError("ct too small")
        tag = ctypes.create_string_buffer(16)
        check(gcm_encrypt(self.handle, kp, kl, ip, il, ap, al, pp, pl, cp, ctypes.addressof(tag),
                          GCM_MEM_HOST, stream))
        return ct, tag.raw

    def decrypt_verify_host(self, key: bytes, iv: bytes, aad, ct, tag: bytes, pt=None, stream=0):
        import numpy as np

        kp, kl, kk = _host_buf(key)
        ip, il, ik = _host_buf(iv)
        ap, al, ak = _host_buf(aad)
        cp, cl, ck = _host_buf(ct)
        tp, tl, tk = _host_buf(tag)
        if pt is None:
            pt = np.empty(cl, dtype=np.uint8)
        pp, pl, pk = _host_buf(pt)
        if pl < cl or tl != 16:
            raise ValueError("bad buffer sizes")
        check(gcm_decrypt_verify(self.handle, kp, kl, ip, il, ap, al, cp, cl, tp, pp, GCM_MEM_HOST, stream))
        return pt
