"""ctypes binding of ``libgcmgpu.so`` (the C ABI in ``include/gcmgpu.h``).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  If the library has not been built, importing this module
raises; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgcmgpu.so")

GCM_OK = 0
GCM_ERR_INVALID_ARG = -1
GCM_ERR_LENGTH_LIMIT = -2
GCM_ERR_AUTH = -3
GCM_ERR_NO_MEMORY = -4
GCM_ERR_CUDA = -5
GCM_ERR_TIMEOUT = -6
GCM_ERR_ALIGNMENT = -7
GCM_ERR_BUSY = -8

GCM_MEM_DEVICE = 0
GCM_MEM_HOST = 1
GCM_AES_TABLES = 0
GCM_AES_BITSLICED = 1

STATUS_NAMES = {
    GCM_OK: "GCM_OK",
    GCM_ERR_INVALID_ARG: "GCM_ERR_INVALID_ARG",
    GCM_ERR_LENGTH_LIMIT: "GCM_ERR_LENGTH_LIMIT",
    GCM_ERR_AUTH: "GCM_ERR_AUTH",
    GCM_ERR_NO_MEMORY: "GCM_ERR_NO_MEMORY",
    GCM_ERR_CUDA: "GCM_ERR_CUDA",
    GCM_ERR_TIMEOUT: "GCM_ERR_TIMEOUT",
    GCM_ERR_ALIGNMENT: "GCM_ERR_ALIGNMENT",
    GCM_ERR_BUSY: "GCM_ERR_BUSY",
}

GFC_AAD_HEADER = 0
GFC_AAD_STRUCTURAL = 1


class GfcLayout(ctypes.Structure):
    _fields_ = [("header_bytes", ctypes.c_size_t), ("data_bytes", ctypes.c_size_t),
                ("data_padded_bytes", ctypes.c_size_t), ("bitpix", ctypes.c_int), ("naxis", ctypes.c_int),
                ("naxes", ctypes.c_int64 * 16)]


class GfcResult(ctypes.Structure):
    _fields_ = [("data_buffer", ctypes.c_void_p), ("buffer_size", ctypes.c_size_t), ("error_code", ctypes.c_int),
                ("warning_code", ctypes.c_int), ("error_message", ctypes.c_char * 200), ("mem", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("datasum", ctypes.c_uint32), ("datasum_valid", ctypes.c_int)]


class GcmMsg(ctypes.Structure):
    _fields_ = [("key", ctypes.c_void_p), ("key_len", ctypes.c_size_t), ("iv", ctypes.c_void_p),
                ("iv_len", ctypes.c_size_t), ("aad", ctypes.c_void_p), ("aad_len", ctypes.c_size_t),
                ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("len", ctypes.c_size_t),
                ("tag", ctypes.c_void_p)]


class GcmRequest(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("key", ctypes.c_uint32), ("iv", ctypes.c_void_p), ("iv_len", ctypes.c_size_t),
                ("aad", ctypes.c_void_p), ("aad_len", ctypes.c_size_t), ("in_", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("len", ctypes.c_size_t), ("tag", ctypes.c_void_p),
                ("arrival_ns", ctypes.c_uint64), ("user", ctypes.c_uint64)]


class GcmCompletion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("arrival_ns", ctypes.c_uint64),
                ("complete_ns", ctypes.c_uint64), ("user", ctypes.c_uint64)]


# Every symbol the header declares, with its ctypes signature.
_VP = ctypes.c_void_p
_SZ = ctypes.c_size_t
SIGNATURES = {
    "gcm_ctx_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, _SZ]),
    "gcm_ctx_destroy": (None, [_VP]),
    "gcm_last_error": (ctypes.c_char_p, []),
    "gcm_encrypt": (ctypes.c_int, [_VP, _VP, _SZ, _VP, _SZ, _VP, _SZ, _VP, _SZ, _VP, _VP, ctypes.c_int, _VP]),
    "gcm_decrypt_verify": (ctypes.c_int, [_VP, _VP, _SZ, _VP, _SZ, _VP, _SZ, _VP, _SZ, _VP, _VP, ctypes.c_int, _VP]),
    "gcm_profile_enable": (ctypes.c_int, [_VP, ctypes.c_int]),
    "gcm_profile_read": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "gcm_encrypt_noalloc": (ctypes.c_int, [_VP, _SZ, _VP, _SZ, _VP, _SZ, _VP, _SZ, _VP, _VP, _VP]),
    "gcm_sync": (ctypes.c_int, [_VP, _VP]),
    "gcm_ctx_set_key_cache": (ctypes.c_int, [_VP, _SZ]),
    "gcm_ctx_set_tile_log2": (ctypes.c_int, [_VP, ctypes.c_int]),
    "gcm_ctx_set_aes_impl": (ctypes.c_int, [_VP, ctypes.c_int]),
    "gcm_ctx_autotune": (ctypes.c_int, [_VP, _SZ, _SZ, _VP]),
    "gcm_ctx_set_tuning": (ctypes.c_int, [_VP, _VP]),
    "gcm_ctr_xor": (ctypes.c_int, [_VP, _VP, _SZ, _VP, _SZ, _VP, _SZ, _VP, _VP]),
    "gcm_ghash": (ctypes.c_int, [_VP, _VP, _SZ, _VP, _SZ, _VP, _SZ, _VP, _VP]),
    "gfc_fits_layout": (ctypes.c_int, [_VP, _SZ, ctypes.POINTER(GfcLayout)]),
    "gcm_batch": (ctypes.c_int, [_VP, ctypes.POINTER(GcmMsg), _SZ, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                 ctypes.c_int, _VP]),
    "gcm_ctx_set_streaming": (ctypes.c_int, [_VP, _SZ, ctypes.c_int]),
    "gcm_ctx_set_host_access": (ctypes.c_int, [_VP, ctypes.c_int]),
    "gcm_key_register": (ctypes.c_int, [_VP, _VP, _SZ, ctypes.POINTER(ctypes.c_uint32)]),
    "gcm_server_create": (ctypes.c_int, [_VP, _SZ, _SZ, ctypes.c_int, ctypes.POINTER(_VP)]),
    "gcm_server_submit": (ctypes.c_int, [_VP, ctypes.POINTER(GcmRequest), ctypes.POINTER(ctypes.c_uint64)]),
    "gcm_server_poll": (ctypes.c_size_t, [_VP, ctypes.POINTER(GcmCompletion), _SZ]),
    "gcm_server_submit_batch": (ctypes.c_int, [_VP, _VP, _SZ, ctypes.POINTER(ctypes.c_uint64)]),
    "gcm_server_stats": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "gcm_server_destroy": (None, [_VP]),
    "gcm_server_timing": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "gcm_server_admission": (ctypes.c_int, [_VP, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ),
                                            ctypes.POINTER(ctypes.c_uint64)]),
    "gcm_now_ns": (ctypes.c_uint64, []),
    "gcm_batch_timed": (ctypes.c_int, [_VP, ctypes.POINTER(GcmMsg), _SZ, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_uint64), _VP]),
    "gfc_fits_encrypt": (ctypes.c_int, [_VP, _VP, _SZ, _VP, _SZ, _VP, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP,
                                        ctypes.POINTER(GfcResult)]),
    "gfc_fits_decrypt_verify": (ctypes.c_int, [_VP, _VP, _SZ, _VP, _SZ, _VP, _VP, ctypes.c_int, ctypes.c_int,
                                               _VP, ctypes.POINTER(GfcResult)]),
    "gfc_result_free": (None, [_VP, ctypes.POINTER(GfcResult)]),
    "gfc_container_encrypt": (ctypes.c_int, [_VP, _VP, _SZ, _VP, _SZ, _VP, _SZ, _VP, _VP, ctypes.c_int, _VP,
                                             ctypes.POINTER(GfcResult)]),
    "gfc_decrypt_frame": (ctypes.c_int, [_VP, _VP, _SZ, _VP, _SZ, _VP, _SZ, ctypes.c_int, _VP,
                                         ctypes.POINTER(GfcResult)]),
    "gcm_noalloc_last_error": (ctypes.c_char_p, []),
    "gcm_host_alloc": (ctypes.c_int, [ctypes.c_int, _SZ, ctypes.POINTER(_VP)]),
    "gcm_host_free": (ctypes.c_int, [_VP]),
    "gcm_batch_plan_create": (ctypes.c_int, [_VP, ctypes.POINTER(GcmMsg), _SZ, ctypes.c_int, ctypes.POINTER(_VP)]),
    "gcm_batch_plan_set": (ctypes.c_int, [_VP, _SZ, ctypes.POINTER(GcmMsg), _SZ]),
    "gcm_batch_plan_launch": (ctypes.c_int, [_VP, _VP]),
    "gcm_batch_plan_wait": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32)]),
    "gcm_batch_plan_destroy": (None, [_VP]),
}


class GcmError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(code, "?"), code, message))
        self.code = code


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            "libgcmgpu.so is not built (expected at %s); run "
            "`python -c 'import __graft_entry__ as g; g.build()'` first" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def last_error() -> str:
    msg = lib.gcm_last_error()
    return msg.decode("utf-8", "replace") if msg else ""


def check(rc: int) -> int:
    if rc != GCM_OK:
        raise GcmError(rc, last_error())
    return rc


def gcm_ctx_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    h = _VP()
    check(lib.gcm_ctx_create(ctypes.byref(h), device, hbm_budget_bytes))
    return h.value


def gcm_ctx_destroy(ctx: Optional[int]) -> None:
    lib.gcm_ctx_destroy(ctx)


def gcm_encrypt(ctx, key_ptr, key_len, iv_ptr, iv_len, aad_ptr, aad_len, pt_ptr, length, ct_ptr, tag_ptr,
                mem, stream) -> int:
    """Raw call: pointers are integers (host or device per ``mem``).  Returns
    the status code without raising."""
    return lib.gcm_encrypt(ctx, key_ptr, key_len, iv_ptr, iv_len, aad_ptr, aad_len, pt_ptr, length,
                           ct_ptr, tag_ptr, mem, stream)


def gcm_decrypt_verify(ctx, key_ptr, key_len, iv_ptr, iv_len, aad_ptr, aad_len, ct_ptr, length, tag_ptr,
                       pt_ptr, mem, stream) -> int:
    return lib.gcm_decrypt_verify(ctx, key_ptr, key_len, iv_ptr, iv_len, aad_ptr, aad_len, ct_ptr, length,
                                  tag_ptr, pt_ptr, mem, stream)


def gcm_profile_enable(ctx, enable: bool) -> None:
    check(lib.gcm_profile_enable(ctx, 1 if enable else 0))


def gcm_profile_read(ctx, reset: bool = False):
    """Returns dict(fused_ms, fused_launches, fused_bytes, launches)."""
    ms, nl, nb, la = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    check(lib.gcm_profile_read(ctx, 1 if reset else 0, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(nb),
                               ctypes.byref(la)))
    return {"fused_ms": ms.value, "fused_launches": nl.value, "fused_bytes": nb.value, "launches": la.value}


def gcm_encrypt_noalloc(key_ptr, key_len, iv_ptr, iv_len, aad_ptr, aad_len, pt_ptr, length, ct_ptr, tag_ptr,
                        stream) -> int:
    """Raw call of the allocation-free encryption (device pointers for aad,
    pt, ct, tag; host pointers for key and iv).  Returns the status code."""
    return lib.gcm_encrypt_noalloc(key_ptr, key_len, iv_ptr, iv_len, aad_ptr, aad_len, pt_ptr, length, ct_ptr,
                                   tag_ptr, stream)


def noalloc_last_error() -> str:
    msg = lib.gcm_noalloc_last_error()
    return msg.decode("utf-8", "replace") if msg else ""


def gfc_fits_layout(fits: bytes) -> GfcLayout:
    buf = ctypes.create_string_buffer(bytes(fits), max(1, len(fits)))
    out = GfcLayout()
    check(lib.gfc_fits_layout(ctypes.addressof(buf), len(fits), ctypes.byref(out)))
    return out
