"""gcm_encrypt_noalloc: the allocation-free encryption entry point.

Callers that cannot allocate device memory at call time use this entry
point: a process whose HBM is owned by another allocator (a framework's
caching pool, a memory-capped serving process), or a latency-critical loop
that must not risk the device-wide synchronisation of cudaMalloc/cudaFree.
Its scratch is a fixed array inside the library.

Checked here, through the C ABI:
  * every call's ciphertext and tag equal the oracle's (whole messages):
    AES-128/192/256; 96-bit IVs and IVs of 1, 60 and 256 bytes; an empty
    message with no AAD (no tile at all) and one with AAD only; payloads
    small enough for tiles below 2^16 blocks; a payload + AAD of exactly
    2^29 blocks (8 GiB: 8192 tiles, every partial slot and the last tree
    slot of the fixed array in use), checked with the oracle run chunk by
    chunk on all host cores;
  * every call also equals the regular pooled entry point (gcm_encrypt);
  * calls in a row leave free device memory unchanged;
  * requests beyond the fixed array are refused before any GPU work.
It is named so that pytest collects it after every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import mapreduce
from paper_2602_23067_gb300 import workloads

pytestmark = pytest.mark.gpu

BIG = 1 << 33  # payload + AAD of the largest case: 2^29 blocks


def _cases():
    r = workloads.rng(99)

    def b(n):
        return r.integers(0, 256, n, dtype=np.uint8).tobytes()

    return [
        {"what": "AES-256, 96-bit IV, FITS header record as AAD, ragged payload",
         "key": b(32), "iv": b(12), "aad": workloads.fits_header(99, -32, [1024, 768]),
         "pt": workloads.random_bytes(991, 3 * (1 << 20) + 5).tobytes()},
        {"what": "AES-128, 60-byte IV (GHASH(IV) path), short AAD",
         "key": b(16), "iv": b(60), "aad": b(20), "pt": workloads.random_bytes(992, 1 << 20).tobytes()},
        {"what": "empty payload, no AAD (no tile)", "key": b(16), "iv": b(12), "aad": b"", "pt": b""},
        {"what": "empty payload, AAD only", "key": b(32), "iv": b(12), "aad": b(100), "pt": b""},
        {"what": "AES-192, 1-byte IV, 1000-byte payload (smallest tiles)",
         "key": b(24), "iv": b(1), "aad": b(7), "pt": b(1000)},
        {"what": "AES-128, 256-byte IV (the limit), 70000-byte payload",
         "key": b(16), "iv": b(256), "aad": b(33), "pt": b(70000)},
    ]


def _dev(torch, data: bytes, n=None):
    n = len(data) if n is None else n
    t = torch.empty(max(16, n), dtype=torch.uint8, device="cuda")
    if data:
        t[:len(data)].copy_(torch.frombuffer(bytearray(data), dtype=torch.uint8))
    return t


def _noalloc(native, key, iv, aad_t, aad_len, pt_t, n, ct_t, tag_t, stream):
    kb = ctypes.create_string_buffer(key, len(key))
    ib = ctypes.create_string_buffer(iv, len(iv))
    return native.gcm_encrypt_noalloc(ctypes.addressof(kb), len(key), ctypes.addressof(ib), len(iv),
                                      aad_t.data_ptr() if aad_len else None, aad_len,
                                      pt_t.data_ptr() if n else None, n, ct_t.data_ptr() if n else None,
                                      tag_t.data_ptr(), stream)


def test_noalloc_matches_the_oracle_and_the_pooled_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_23067_gb300 import Context, _native

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    cases = _cases()
    # expected values from the existing pooled entry point
    pooled = []
    with Context(0) as ctx:
        for c in cases:
            aad = torch.frombuffer(bytearray(c["aad"]), dtype=torch.uint8).cuda() if c["aad"] else None
            pt = torch.frombuffer(bytearray(c["pt"]), dtype=torch.uint8).cuda() if c["pt"] else \
                torch.empty(0, dtype=torch.uint8, device="cuda")
            ct, tag = ctx.encrypt_device(c["key"], c["iv"], aad, pt)
            torch.cuda.synchronize()
            pooled.append((bytes(ct.cpu().numpy()), bytes(tag.cpu().numpy())))
    torch.cuda.synchronize()

    bufs = [(_dev(torch, c["aad"]), _dev(torch, c["pt"]), _dev(torch, b"", len(c["pt"])),
             torch.empty(16, dtype=torch.uint8, device="cuda")) for c in cases]
    torch.cuda.synchronize()
    free = []
    for c, (aad_t, pt_t, ct_t, tag_t), (pct, ptag) in zip(cases, bufs, pooled):
        n = len(c["pt"])
        rc = _noalloc(_native, c["key"], c["iv"], aad_t, len(c["aad"]), pt_t, n, ct_t, tag_t, stream)
        assert rc == 0, (c["what"], _native.noalloc_last_error())
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        ref_ct, ref_tag = oracle.gcm_encrypt(c["key"], c["iv"], c["aad"], c["pt"])
        got_ct, got_tag = bytes(ct_t[:n].cpu().numpy()), bytes(tag_t.cpu().numpy())
        assert got_tag == ref_tag, c["what"]
        assert got_ct == ref_ct, c["what"]
        assert (got_ct, got_tag) == (pct, ptag), c["what"]
    # the calls after the first allocated nothing
    assert len(set(free)) == 1, free


def test_noalloc_at_its_largest_size_against_the_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_23067_gb300 import Context, _native

    torch.cuda.set_device(0)
    torch.cuda.empty_cache()
    if torch.cuda.mem_get_info()[0] < 3 * BIG + (8 << 30):
        pytest.skip("needs %d GB of free device memory" % ((3 * BIG + (8 << 30)) // 10**9))
    r = workloads.rng(98)
    key = r.integers(0, 256, 32, dtype=np.uint8).tobytes()
    iv = r.integers(0, 256, 12, dtype=np.uint8).tobytes()
    aad = workloads.fits_header(98, -32, [65536, 32768])
    n = BIG - len(aad)  # payload + AAD = 2^29 blocks: 8192 tiles of 2^16
    assert (len(aad) + 15) // 16 + (n + 15) // 16 == 1 << 29
    stream = torch.cuda.current_stream().cuda_stream
    aad_t = _dev(torch, aad)
    pt = torch.empty(n, dtype=torch.uint8, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(98)
    for o in range(0, n, 1 << 30):
        k = min(1 << 30, n - o)
        pt[o:o + k].copy_(torch.randint(0, 256, (k,), dtype=torch.uint8, device="cuda", generator=g))
    ct = torch.empty_like(pt)
    ct_first = torch.empty_like(pt)
    tag_t = torch.empty(16, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    free = []
    for _ in range(2):  # two calls in a row: same output, no allocation
        ct.zero_()
        rc = _noalloc(_native, key, iv, aad_t, len(aad), pt, n, ct, tag_t, stream)
        assert rc == 0, _native.noalloc_last_error()
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        if len(free) == 1:
            first_tag = bytes(tag_t.cpu().numpy())
            ct_first.copy_(ct)
    assert free[0] == free[1], free
    assert bytes(tag_t.cpu().numpy()) == first_tag
    assert torch.equal(ct, ct_first)
    del ct_first
    # the pooled entry point on the same message
    with Context(0) as ctx:
        ct2, tag2 = ctx.encrypt_device(key, iv, aad_t[:len(aad)], pt)
        torch.cuda.synchronize()
        assert bytes(tag2.cpu().numpy()) == first_tag
        assert torch.equal(ct2, ct)
        del ct2
    # the oracle, chunk by chunk on the host cores
    chunk = 64 << 20
    with mapreduce.HostInput(n) as src:
        torch.from_numpy(src.array).copy_(pt)
        (ref_dg, ref_tag), = mapreduce.gcm_encrypt_digests(
            [{"key": key, "iv": iv, "aad": aad, "off": 0, "len": n}], src, chunk_bytes=chunk)
    assert first_tag == ref_tag
    host = ct.cpu()
    assert mapreduce.digests(host.numpy(), chunk) == ref_dg
    del host, pt, ct
    torch.cuda.empty_cache()


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
