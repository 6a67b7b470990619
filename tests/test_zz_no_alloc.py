"""gcm_encrypt_noalloc: the allocation-free encryption entry point.

Callers that cannot allocate device memory at call time (their HBM is owned
by another allocator, or they must avoid the device-wide synchronisation a
cudaMalloc/cudaFree can cause) use this entry point; its scratch is a fixed
array inside the library.  This file checks, through the C ABI, that two
calls in a row give exactly the ciphertext and tag of the regular pooled
entry point (gcm_encrypt), and that the calls leave free device memory
unchanged.  It is named so that pytest collects it after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2602_23067_gb300 import workloads

pytestmark = pytest.mark.gpu


def _cases():
    r = workloads.rng(99)
    return [
        {  # AES-256, 96-bit IV, one FITS header record as AAD, ragged payload
            "key": r.integers(0, 256, 32, dtype=np.uint8).tobytes(),
            "iv": r.integers(0, 256, 12, dtype=np.uint8).tobytes(),
            "aad": workloads.fits_header(99, -32, [1024, 768]),
            "pt": workloads.random_bytes(991, 3 * (1 << 20) + 5).tobytes(),
        },
        {  # AES-128, 60-byte IV (GHASH(IV) path), short AAD
            "key": r.integers(0, 256, 16, dtype=np.uint8).tobytes(),
            "iv": r.integers(0, 256, 60, dtype=np.uint8).tobytes(),
            "aad": r.integers(0, 256, 20, dtype=np.uint8).tobytes(),
            "pt": workloads.random_bytes(992, 1 << 20).tobytes(),
        },
    ]


def test_noalloc_matches_the_pooled_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_23067_gb300 import Context, _native

    torch.cuda.set_device(0)
    cases = _cases()
    dev = []
    for c in cases:
        dev.append({
            "aad": torch.frombuffer(bytearray(c["aad"]), dtype=torch.uint8).cuda(),
            "pt": torch.frombuffer(bytearray(c["pt"]), dtype=torch.uint8).cuda(),
            "ct": torch.empty(len(c["pt"]), dtype=torch.uint8, device="cuda"),
            "tag": torch.empty(16, dtype=torch.uint8, device="cuda"),
        })
    # expected values from the existing entry point
    expected = []
    with Context(0) as ctx:
        for c, d in zip(cases, dev):
            ct, tag = ctx.encrypt_device(c["key"], c["iv"], d["aad"], d["pt"])
            torch.cuda.synchronize()
            expected.append((bytes(ct.cpu().numpy()), bytes(tag.cpu().numpy())))
            del ct, tag
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream().cuda_stream
    free = []
    for c, d, (ect, etag) in zip(cases, dev, expected):
        kb = ctypes.create_string_buffer(c["key"], len(c["key"]))
        ib = ctypes.create_string_buffer(c["iv"], len(c["iv"]))
        rc = _native.gcm_encrypt_noalloc(ctypes.addressof(kb), len(c["key"]), ctypes.addressof(ib), len(c["iv"]),
                                         d["aad"].data_ptr(), d["aad"].numel(), d["pt"].data_ptr(),
                                         d["pt"].numel(), d["ct"].data_ptr(), d["tag"].data_ptr(), stream)
        assert rc == 0, _native.noalloc_last_error()
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert bytes(d["tag"].cpu().numpy()) == etag
        assert bytes(d["ct"].cpu().numpy()) == ect
    # the second call allocated nothing
    assert free[1] == free[0]


def test_noalloc_rejects_requests_beyond_its_scratch():
    pytest.importorskip("torch")
    from paper_2602_23067_gb300 import _native

    key, iv = ctypes.create_string_buffer(16), ctypes.create_string_buffer(12)
    fake = 1 << 40  # never dereferenced: the size check comes first
    rc = _native.gcm_encrypt_noalloc(ctypes.addressof(key), 16, ctypes.addressof(iv), 12, None, 0, fake,
                                     (8 << 30) + 16, fake, fake, None)
    assert rc == _native.GCM_ERR_LENGTH_LIMIT
    assert "8 GiB" in _native.noalloc_last_error()
    iv300 = ctypes.create_string_buffer(300)
    rc = _native.gcm_encrypt_noalloc(ctypes.addressof(key), 16, ctypes.addressof(iv300), 300, None, 0, fake, 16,
                                     fake, fake, None)
    assert rc == _native.GCM_ERR_LENGTH_LIMIT
