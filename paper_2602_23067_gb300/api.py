"""GB300 AES-GCM for FITS data units (the data path of "GpuFitsCrypt").

The computation lives in ``libgcmgpu.so`` (C ABI: ``include/gcmgpu.h``).  This
package is a thin binding: it turns tensors, numpy arrays and ``bytes`` into
pointers and lengths and maps status codes to exceptions.  PyTorch is used
only for device memory and streams.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

from ._native import (GCM_ERR_AUTH, GCM_MEM_DEVICE, GCM_MEM_HOST, GCM_OK, GFC_AAD_HEADER, GFC_AAD_STRUCTURAL,
                      GcmError, GcmMsg, GfcResult, check, gcm_ctx_create, gcm_ctx_destroy, gcm_decrypt_verify,
                      gcm_encrypt, last_error, lib)

__all__ = [
    "Context", "GcmError", "GCM_OK", "GCM_ERR_AUTH", "GCM_MEM_DEVICE", "GCM_MEM_HOST",
    "gcm_ctx_create", "gcm_ctx_destroy", "gcm_encrypt", "gcm_decrypt_verify", "last_error",
    "FitsResult", "GFC_AAD_HEADER", "GFC_AAD_STRUCTURAL", "Server", "HostBuffer", "BatchPlan",
]


class FitsResult:
    """A processed FITS file (the paper's FitsOperationResult): ``data`` is a
    uint8 CUDA tensor (device calls) or numpy array (host calls) holding the
    header in clear and the processed data unit; ``warning_code`` is 2 when
    the payload was suppressed after a tag mismatch."""

    def __init__(self, data, error_code: int, warning_code: int, message: str, iv: bytes = b"", tag: bytes = b"",
                 datasum: Optional[int] = None):
        self.data = data
        self.error_code = error_code
        self.warning_code = warning_code
        self.message = message
        self.iv = iv
        self.tag = tag
        # FITS DATASUM of the encrypted data unit (None when not computed)
        self.datasum = datasum


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


def _key_arg(b) -> Tuple[object, int]:
    """A host key or IV for a direct library call: bytes objects are passed
    as they are (ctypes hands over a pointer to their immutable buffer for
    the duration of the call), anything else through _host_buf."""
    if type(b) is bytes:
        return b, len(b)
    p, n, _ = _host_buf(b)
    return p, n


def _dev_buf(t) -> Tuple[int, int]:
    if t is None:
        return 0, 0
    try:
        cuda, contig = t.is_cuda, t.is_contiguous()
    except AttributeError:
        raise TypeError("device mode expects CUDA tensors") from None
    if not cuda:
        raise TypeError("device mode expects CUDA tensors")
    if not contig:
        raise ValueError("tensors must be contiguous")
    return t.data_ptr(), t.nbytes


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
        if ct is None or tag is None:
            import torch

            if ct is None:
                ct = torch.empty_like(pt)
            if tag is None:
                tag = torch.empty(16, dtype=torch.uint8, device=pt.device)
        kp, kl = _key_arg(key)
        ip, il = _key_arg(iv)
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
        if pt is None:
            import torch

            pt = torch.empty_like(ct)
        kp, kl = _key_arg(key)
        ip, il = _key_arg(iv)
        ap, al = _dev_buf(aad)
        cp, cl = _dev_buf(ct)
        tp, tl = _dev_buf(tag)
        pp, pl = _dev_buf(pt)
        if pl < cl or tl < 16:
            raise ValueError("buffers too small")
        check(gcm_decrypt_verify(self.handle, kp, kl, ip, il, ap, al, cp, cl, tp, pp, GCM_MEM_DEVICE,
                                 _stream_handle(stream)))
        return pt

    def set_key_cache(self, entries: int) -> None:
        """gcm_ctx_set_key_cache: keys kept set up on the device (0 = off)."""
        check(lib.gcm_ctx_set_key_cache(self.handle, entries))

    def set_tile_log2(self, tile_log2: int) -> None:
        """gcm_ctx_set_tile_log2: force tiles of 2^tile_log2 blocks (0 = default)."""
        check(lib.gcm_ctx_set_tile_log2(self.handle, tile_log2))

    def set_aes_impl(self, impl: int) -> None:
        """gcm_ctx_set_aes_impl: GCM_AES_TABLES (0) or GCM_AES_BITSLICED (1)."""
        check(lib.gcm_ctx_set_aes_impl(self.handle, impl))

    def autotune(self, key_len: int = 32, max_bytes: int = 256 << 20) -> bytes:
        """gcm_ctx_autotune: returns the 64-entry table (tile log2 per size class)."""
        buf = ctypes.create_string_buffer(64)
        check(lib.gcm_ctx_autotune(self.handle, key_len, max_bytes, ctypes.addressof(buf)))
        return buf.raw

    def set_tuning(self, table: Optional[bytes]) -> None:
        """gcm_ctx_set_tuning: install a saved table (None clears it)."""
        if table is None:
            check(lib.gcm_ctx_set_tuning(self.handle, None))
            return
        buf = ctypes.create_string_buffer(bytes(table), 64)
        check(lib.gcm_ctx_set_tuning(self.handle, ctypes.addressof(buf)))

    def sync(self, stream=None) -> None:
        """gcm_sync: wait for the work enqueued on `stream` (default: torch's
        current stream) and raise GcmError on an asynchronous CUDA error."""
        check(lib.gcm_sync(self.handle, _stream_handle(stream)))

    def ctr_xor_device(self, key: bytes, iv: bytes, inp, out=None, stream=None):
        """Enqueue the CTR keystream XOR alone (gcm_ctr_xor); returns out."""
        import torch

        if out is None:
            out = torch.empty_like(inp)
        kp, kl, kk = _host_buf(key)
        ip, il, ik = _host_buf(iv)
        sp, sl = _dev_buf(inp)
        op, ol = _dev_buf(out)
        if ol < sl:
            raise ValueError("output buffer too small")
        check(lib.gcm_ctr_xor(self.handle, kp, kl, ip, il, sp, sl, op, _stream_handle(stream)))
        return out

    def ghash_device(self, key: bytes, aad, data, out=None, stream=None):
        """Enqueue GHASH_H(aad, data) alone (gcm_ghash); returns a 16-byte tensor."""
        import torch

        if out is None:
            out = torch.empty(16, dtype=torch.uint8, device=data.device)
        kp, kl, kk = _host_buf(key)
        ap, al = _dev_buf(aad)
        dp, dl = _dev_buf(data)
        op, ol = _dev_buf(out)
        if ol < 16:
            raise ValueError("output buffer too small")
        check(lib.gcm_ghash(self.handle, kp, kl, ap, al, dp, dl, op, _stream_handle(stream)))
        return out

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

    # -- many messages (gcm_batch) ------------------------------------------
    def set_host_access(self, mode: int) -> None:
        """0 auto (direct kernel access to host memory when the device supports
        it), 1 require direct, 2 always stage through device buffers."""
        check(lib.gcm_ctx_set_host_access(self.handle, mode))

    def set_streaming(self, chunk_bytes: int, n_buffers: int = 3) -> None:
        check(lib.gcm_ctx_set_streaming(self.handle, chunk_bytes, n_buffers))

    def batch(self, msgs, decrypt: bool = False, stream=None):
        """gcm_batch over a list of dicts with keys key, iv (bytes) and aad,
        inp, out, tag: CUDA tensors (device batch: one persistent launch) or
        host buffers (numpy / pinned tensors: the streamed pipeline).  All
        messages must live in the same memory space.  Returns the list of
        per-message status codes (0 or GCM_ERR_AUTH)."""
        n = len(msgs)
        arr = (GcmMsg * max(1, n))()
        keep = []
        device = None
        for i, m in enumerate(msgs):
            dev = hasattr(m["inp"], "is_cuda") and m["inp"].is_cuda
            if device is None:
                device = dev
            elif device != dev:
                raise ValueError("all messages of a batch must be in the same memory space")
            arr[i] = _gcm_msg(m, dev, keep)
        status = (ctypes.c_int32 * max(1, n))()
        mem = GCM_MEM_DEVICE if device else GCM_MEM_HOST
        st = _stream_handle(stream) if device else 0
        check(lib.gcm_batch(self.handle, arr, n, 1 if decrypt else 0, status, mem, st))
        return [int(status[i]) for i in range(n)]

    def batch_plan(self, msgs, decrypt: bool = False) -> "BatchPlan":
        """gcm_batch_plan_create over device messages (dicts as for ``batch``):
        the batch prepared once and replayed as a CUDA graph."""
        return BatchPlan(self, msgs, decrypt)

    # -- key cache and serving ----------------------------------------------
    def key_register(self, key: bytes) -> int:
        """gcm_key_register: builds the key's material once on the device."""
        kp, kl, kk = _host_buf(key)
        h = ctypes.c_uint32()
        check(lib.gcm_key_register(self.handle, kp, kl, ctypes.byref(h)))
        return h.value

    def server(self, hbm_budget_bytes: int = 0, max_wave_msgs: int = 4096, max_inflight: int = 3) -> "Server":
        return Server(self, hbm_budget_bytes, max_wave_msgs, max_inflight)

    # -- FITS files (header in clear, data unit encrypted) ------------------
    def _fits_common(self, decrypt, key, fits, iv, tag, aad_mode, stream):
        import numpy as np

        kp, kl, kk = _host_buf(key)
        device = hasattr(fits, "is_cuda") and fits.is_cuda
        if device:
            fp, fl = _dev_buf(fits)
            mem, st = GCM_MEM_DEVICE, _stream_handle(stream)
        else:
            fp, fl, fk = _host_buf(fits)
            mem, st = GCM_MEM_HOST, (stream or 0)
        res = GfcResult()
        iv_out = ctypes.create_string_buffer(12)
        tag_out = ctypes.create_string_buffer(16)
        ivb = ctypes.create_string_buffer(bytes(iv), 12) if iv is not None else None
        if decrypt:
            tb = ctypes.create_string_buffer(bytes(tag), 16)
            rc = lib.gfc_fits_decrypt_verify(self.handle, kp, kl, fp, fl, ctypes.addressof(ivb),
                                             ctypes.addressof(tb), aad_mode, mem, st, ctypes.byref(res))
        else:
            rc = lib.gfc_fits_encrypt(self.handle, kp, kl, fp, fl, ctypes.addressof(ivb) if ivb is not None else None,
                                      ctypes.addressof(iv_out), ctypes.addressof(tag_out), aad_mode, mem, st,
                                      ctypes.byref(res))
        msg = res.error_message.decode("utf-8", "replace")
        data = None
        if res.data_buffer:
            n = res.buffer_size
            if device:
                data = _dev_tensor_copy(res.data_buffer, n, fits.device)
            else:
                data = np.ctypeslib.as_array((ctypes.c_uint8 * n).from_address(res.data_buffer)).copy()
        datasum = int(res.datasum) if res.datasum_valid else None
        warning = res.warning_code
        if res.data_buffer:
            lib.gfc_result_free(self.handle, ctypes.byref(res))
        if rc not in (GCM_OK, GCM_ERR_AUTH):
            raise GcmError(rc, msg)
        return FitsResult(data, rc, warning, msg, iv_out.raw if not decrypt else bytes(iv),
                          tag_out.raw if not decrypt else bytes(tag), datasum)

    def _take_result(self, rc, res, device, like):
        import numpy as np

        msg = res.error_message.decode("utf-8", "replace")
        data = None
        if res.data_buffer:
            n = res.buffer_size
            if device:
                data = _dev_tensor_copy(res.data_buffer, n, like.device)
            else:
                data = np.ctypeslib.as_array((ctypes.c_uint8 * n).from_address(res.data_buffer)).copy()
        datasum = int(res.datasum) if res.datasum_valid else None
        warning = res.warning_code
        if res.data_buffer:
            lib.gfc_result_free(self.handle, ctypes.byref(res))
        if rc != GCM_OK:
            raise GcmError(rc, msg)
        return FitsResult(data, rc, warning, msg, datasum=datasum)

    def container_encrypt(self, key_h: bytes, key_d: bytes, fits, nonce_h: Optional[bytes] = None,
                          nonce_d: Optional[bytes] = None, stream=None) -> "FitsResult":
        """gfc_container_encrypt: the paper's two-HDU dual-key container of a
        FITS image (bytes/numpy on the host or a CUDA uint8 tensor)."""
        device = hasattr(fits, "is_cuda") and fits.is_cuda
        if device:
            fp, fl = _dev_buf(fits)
            mem, st = GCM_MEM_DEVICE, _stream_handle(stream)
        else:
            fp, fl, fk = _host_buf(fits)
            mem, st = GCM_MEM_HOST, (stream or 0)
        hp, hl, hk = _host_buf(key_h)
        dp, dl, dk = _host_buf(key_d)
        nh = ctypes.create_string_buffer(bytes(nonce_h), 12) if nonce_h is not None else None
        nd = ctypes.create_string_buffer(bytes(nonce_d), 12) if nonce_d is not None else None
        res = GfcResult()
        rc = lib.gfc_container_encrypt(self.handle, hp, hl, dp, dl, fp, fl,
                                       ctypes.addressof(nh) if nh is not None else None,
                                       ctypes.addressof(nd) if nd is not None else None, mem, st, ctypes.byref(res))
        return self._take_result(rc, res, device, fits)

    def decrypt_frame(self, container, key_h: Optional[bytes], key_d: Optional[bytes], stream=None) -> "FitsResult":
        """gfc_decrypt_frame: the FITS file of a container, with the paper's
        warning codes (0 full access, 1 header fallback, 2 payload suppressed)."""
        device = hasattr(container, "is_cuda") and container.is_cuda
        if device:
            cp, cl = _dev_buf(container)
            mem, st = GCM_MEM_DEVICE, _stream_handle(stream)
        else:
            cp, cl, ck = _host_buf(container)
            mem, st = GCM_MEM_HOST, (stream or 0)
        hp, hl, hk = _host_buf(key_h) if key_h is not None else (None, 0, None)
        dp, dl, dk = _host_buf(key_d) if key_d is not None else (None, 0, None)
        res = GfcResult()
        rc = lib.gfc_decrypt_frame(self.handle, cp, cl, hp, hl, dp, dl, mem, st, ctypes.byref(res))
        return self._take_result(rc, res, device, container)

    def fits_encrypt_raw(self, key: bytes, fits, iv: bytes, aad_mode: int = GFC_AAD_HEADER, stream=None):
        """gfc_fits_encrypt on a CUDA tensor without copying the result: returns
        (GfcResult, tag).  The result buffer belongs to the library until
        ``release(result)``."""
        kp, kl, kk = _host_buf(key)
        fp, fl = _dev_buf(fits)
        res = GfcResult()
        ivb = ctypes.create_string_buffer(bytes(iv), 12)
        iv_out, tag_out = ctypes.create_string_buffer(12), ctypes.create_string_buffer(16)
        rc = lib.gfc_fits_encrypt(self.handle, kp, kl, fp, fl, ctypes.addressof(ivb), ctypes.addressof(iv_out),
                                  ctypes.addressof(tag_out), aad_mode, GCM_MEM_DEVICE, _stream_handle(stream),
                                  ctypes.byref(res))
        if rc != GCM_OK:
            raise GcmError(rc, res.error_message.decode("utf-8", "replace"))
        return res, tag_out.raw

    def fits_decrypt_verify_raw(self, key: bytes, enc_ptr: int, enc_len: int, iv: bytes, tag: bytes,
                                aad_mode: int = GFC_AAD_HEADER, stream=None):
        """gfc_fits_decrypt_verify on a device buffer (e.g. a raw encryption
        result) without copying: returns the GfcResult (raises on errors other
        than a tag mismatch)."""
        kp, kl, kk = _host_buf(key)
        res = GfcResult()
        ivb = ctypes.create_string_buffer(bytes(iv), 12)
        tb = ctypes.create_string_buffer(bytes(tag), 16)
        rc = lib.gfc_fits_decrypt_verify(self.handle, kp, kl, enc_ptr, enc_len, ctypes.addressof(ivb),
                                         ctypes.addressof(tb), aad_mode, GCM_MEM_DEVICE, _stream_handle(stream),
                                         ctypes.byref(res))
        if rc not in (GCM_OK, GCM_ERR_AUTH):
            raise GcmError(rc, res.error_message.decode("utf-8", "replace"))
        return res

    def release(self, res) -> None:
        """gfc_result_free for a raw result."""
        lib.gfc_result_free(self.handle, ctypes.byref(res))

    @staticmethod
    def result_view(res, offset: int = 0, length: Optional[int] = None, device=None):
        """A uint8 tensor viewing (not copying) a raw device result."""
        import torch

        n = (res.buffer_size - offset) if length is None else length
        return torch.as_tensor(_DevView(res.data_buffer + offset, n), device=device or "cuda")

    def fits_encrypt(self, key: bytes, fits, iv: Optional[bytes] = None, aad_mode: int = GFC_AAD_HEADER,
                     stream=None) -> "FitsResult":
        """gfc_fits_encrypt.  ``fits`` is bytes/numpy (host) or a CUDA uint8
        tensor (device).  iv=None draws a random 96-bit IV."""
        return self._fits_common(False, key, fits, iv, None, aad_mode, stream)

    def fits_decrypt_verify(self, key: bytes, fits_enc, iv: bytes, tag: bytes, aad_mode: int = GFC_AAD_HEADER,
                            stream=None) -> "FitsResult":
        """gfc_fits_decrypt_verify.  A tag mismatch does not raise: the
        result has error_code GCM_ERR_AUTH, warning_code 2 and a zeroed data
        unit (payload suppression)."""
        return self._fits_common(True, key, fits_enc, iv, tag, aad_mode, stream)


class HostBuffer:
    """Page-locked host memory of exactly ``nbytes`` from gcm_host_alloc, for
    GCM_MEM_HOST calls, host batches and the server.  ``ptr`` is the address
    and ``tensor`` a uint8 CPU tensor over it (valid until ``free``)."""

    def __init__(self, nbytes: int, device: int = 0):
        import torch

        p = ctypes.c_void_p()
        check(lib.gcm_host_alloc(device, nbytes, ctypes.byref(p)))
        self.ptr = int(p.value)
        self.nbytes = nbytes
        self.tensor = torch.frombuffer((ctypes.c_uint8 * nbytes).from_address(self.ptr), dtype=torch.uint8)

    def free(self) -> None:
        if self.ptr:
            self.tensor = None
            check(lib.gcm_host_free(ctypes.c_void_p(self.ptr)))
            self.ptr = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()


class _Raw:
    pass


class _DevView:
    """Exposes a library-owned device buffer to torch (CUDA array interface)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "|u1", "data": (ptr, False), "version": 3,
                                         "strides": None}


def _dev_tensor_copy(ptr: int, n: int, device):
    """Copies n bytes at a library-owned device pointer into a new tensor."""
    import torch

    torch.cuda.synchronize(device)
    view = torch.as_tensor(_DevView(ptr, n), device=device)
    out = view.clone()
    torch.cuda.synchronize(device)
    return out


def _gcm_msg(m, dev: bool, keep: list) -> GcmMsg:
    """One gcm_msg from a dict with keys key, iv (bytes) and aad, inp, out,
    tag (CUDA tensors when dev, else host buffers); optional len."""
    kp, kl, kk = _host_buf(m["key"])
    ip, il, ik = _host_buf(m["iv"])
    keep += [kk, ik]
    if dev:
        ap, al = _dev_buf(m.get("aad"))
        pp, pl = _dev_buf(m["inp"])
        op, ol = _dev_buf(m["out"])
        tp, tl = _dev_buf(m["tag"])
    else:
        ap, al, ak = _host_buf(m.get("aad"))
        pp, pl, pk = _host_buf(m["inp"])
        op, ol, ok = _host_buf(m["out"])
        tp, tl, tk = _host_buf(m["tag"])
        keep += [ak, pk, ok, tk]
    n_bytes = m.get("len", pl)
    if ol < n_bytes or tl < 16:
        raise ValueError("output or tag buffer too small")
    return GcmMsg(kp, kl, ip, il, ap or None, al, pp or None, op or None, n_bytes, tp)


class BatchPlan:
    """A device batch replayed as a CUDA graph (gcm_batch_plan_*): ``set``
    swaps a message's key, IV and buffers (same lengths), ``launch`` enqueues
    one run, ``wait`` returns its per-message statuses."""

    def __init__(self, ctx: "Context", msgs, decrypt: bool):
        self.ctx = ctx
        self.n = len(msgs)
        keep = []
        arr = (GcmMsg * max(1, self.n))()
        for i, m in enumerate(msgs):
            if not (hasattr(m["inp"], "is_cuda") and m["inp"].is_cuda):
                raise ValueError("a batch plan takes device (CUDA tensor) messages")
            arr[i] = _gcm_msg(m, True, keep)
        h = ctypes.c_void_p()
        check(lib.gcm_batch_plan_create(ctx.handle, arr, self.n, 1 if decrypt else 0, ctypes.byref(h)))
        self.handle = h.value
        self._status = (ctypes.c_int32 * max(1, self.n))()

    def set(self, i: int, msg) -> None:
        self.set_many(i, [msg])

    def set_many(self, first: int, msgs) -> None:
        """Replaces messages first .. first + len(msgs) - 1 in one call."""
        keep = []
        arr = (GcmMsg * max(1, len(msgs)))()
        for k, m in enumerate(msgs):
            arr[k] = _gcm_msg(m, True, keep)
        check(lib.gcm_batch_plan_set(self.handle, first, arr, len(msgs)))

    def launch(self, stream=None) -> None:
        check(lib.gcm_batch_plan_launch(self.handle, _stream_handle(stream)))

    def wait(self):
        check(lib.gcm_batch_plan_wait(self.handle, self._status))
        return [int(self._status[i]) for i in range(self.n)]

    def run(self, stream=None):
        self.launch(stream)
        return self.wait()

    def close(self) -> None:
        if self.handle:
            lib.gcm_batch_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """The continuous-batching server (gcm_server_*).  Requests reference host
    buffers that must stay alive until their completion is polled."""

    def __init__(self, ctx: Context, hbm_budget_bytes: int, max_wave_msgs: int, max_inflight: int):
        from ._native import GcmCompletion

        self.ctx = ctx
        h = ctypes.c_void_p()
        check(lib.gcm_server_create(ctx.handle, hbm_budget_bytes, max_wave_msgs, max_inflight, ctypes.byref(h)))
        self.handle = h.value
        self._keep = {}
        self._buf = (GcmCompletion * 4096)()

    def submit(self, op: int, key_handle: int, iv: bytes, aad, inp, out, tag, arrival_ns: int = 0,
               user: int = 0) -> int:
        """Queues a request on host buffers (bytes/numpy/pinned tensors); the
        tag buffer receives the tag (op 0) or holds the expected tag (op 1)."""
        from ._native import GcmRequest

        ivp, ivl, ivk = _host_buf(iv)
        ap, al, ak = _host_buf(aad)
        pp, pl, pk = _host_buf(inp)
        op_, ol, ok = _host_buf(out)
        tp, tl, tk = _host_buf(tag)
        req = GcmRequest(op, key_handle, ivp, ivl, ap or None, al, pp or None, op_ or None, pl, tp, arrival_ns, user)
        t = ctypes.c_uint64()
        check(lib.gcm_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = (ivk, ak, pk, ok, tk)
        return t.value

    def poll(self):
        """Returns a list of (ticket, status, arrival_ns, complete_ns, user)."""
        n = lib.gcm_server_poll(self.handle, self._buf, len(self._buf))
        out = []
        for i in range(n):
            c = self._buf[i]
            self._keep.pop(c.ticket, None)
            out.append((c.ticket, c.status, c.arrival_ns, c.complete_ns, c.user))
        return out

    def stats(self):
        w, m, q, b = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_size_t(), ctypes.c_size_t()
        rc = lib.gcm_server_stats(self.handle, ctypes.byref(w), ctypes.byref(m), ctypes.byref(q), ctypes.byref(b))
        bud, peak, waits = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_uint64()
        check(lib.gcm_server_admission(self.handle, ctypes.byref(bud), ctypes.byref(peak), ctypes.byref(waits)))
        return {"waves": w.value, "messages": m.value, "queued": q.value, "bytes_in_flight": b.value, "error": rc,
                "budget": bud.value, "peak_bytes_in_flight": peak.value, "budget_waits": waits.value}

    def close(self) -> None:
        if self.handle:
            lib.gcm_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
