"""GPU path vs the CPU oracle, bit for bit (GCM is deterministic in key, IV,
AAD and payload, so there is exactly one correct ciphertext and tag).

Every call goes through the C ABI (ctypes binding of libgcmgpu.so).
"""
import random

import numpy as np
import pytest

import oracle
from paper_2602_23067_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    from paper_2602_23067_gb300 import Context

    c = Context(0)
    yield c
    c.close()


def rnd(r, n):
    return bytes(r.getrandbits(8) for _ in range(n))


def to_dev(torch, b: bytes):
    t = torch.empty(max(len(b), 0), dtype=torch.uint8, device="cuda")
    if len(b):
        t.copy_(torch.frombuffer(bytearray(b), dtype=torch.uint8))
    return t


def to_bytes(t) -> bytes:
    return bytes(t.cpu().numpy().tobytes())


def gpu_encrypt(torch, ctx, key, iv, aad, pt):
    a = to_dev(torch, aad) if aad else None
    p = to_dev(torch, pt)
    ct, tag = ctx.encrypt_device(key, iv, a, p)
    torch.cuda.synchronize()
    return to_bytes(ct), to_bytes(tag)


def gpu_decrypt(torch, ctx, key, iv, aad, ct, tag):
    from paper_2602_23067_gb300 import GcmError

    a = to_dev(torch, aad) if aad else None
    c = to_dev(torch, ct)
    t = to_dev(torch, tag)
    out = torch.full_like(c, 0xA5)
    try:
        ctx.decrypt_verify_device(key, iv, a, c, t, pt=out)
        ok = True
    except GcmError as e:
        assert e.code == -3, e
        ok = False
    torch.cuda.synchronize()
    return ok, to_bytes(out)


def check_case(torch, ctx, key, iv, aad, pt):
    ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, aad, pt)
    ct, tag = gpu_encrypt(torch, ctx, key, iv, aad, pt)
    assert tag == ref_tag, "tag mismatch (len=%d aad=%d iv=%d key=%d)" % (len(pt), len(aad), len(iv), len(key))
    assert ct == ref_ct, "ciphertext mismatch (len=%d)" % len(pt)
    ok, back = gpu_decrypt(torch, ctx, key, iv, aad, ct, tag)
    assert ok and back == pt


def test_plain_single_message_aes128_1mib(torch_cuda, ctx):
    """1 MiB of seeded uniform bytes, 96-bit IV, 20-byte AAD, AES-128."""
    r = workloads.rng(1)
    key = r.integers(0, 256, 16, dtype=np.uint8).tobytes()
    iv = r.integers(0, 256, 12, dtype=np.uint8).tobytes()
    aad = r.integers(0, 256, 20, dtype=np.uint8).tobytes()
    pt = workloads.random_bytes(11, 1 << 20).tobytes()
    check_case(torch_cuda, ctx, key, iv, aad, pt)


@pytest.mark.parametrize("key_len", [16, 24, 32])
def test_lengths_sweep(torch_cuda, ctx, key_len):
    r = random.Random(key_len)
    for n in (0, 1, 15, 16, 17, 31, 32, 33, 63, 64, 65, 255, 256, 257, 1000, 4095, 4096, 4097):
        key, iv = rnd(r, key_len), rnd(r, 12)
        aad = rnd(r, r.choice((0, 1, 13, 16, 20, 33)))
        check_case(torch_cuda, ctx, key, iv, aad, rnd(r, n))


@pytest.mark.parametrize("aad_len", [0, 1, 15, 16, 17, 20, 255, 2880, 2881, 16 * 1024 + 3])
def test_aad_lengths(torch_cuda, ctx, aad_len):
    r = random.Random(1000 + aad_len)
    key, iv = rnd(r, 32), rnd(r, 12)
    for n in (0, 5, 48, 5000):
        check_case(torch_cuda, ctx, key, iv, rnd(r, aad_len), rnd(r, n))


@pytest.mark.parametrize("iv_len", [1, 7, 8, 11, 13, 16, 17, 60, 128, 300])
def test_iv_lengths(torch_cuda, ctx, iv_len):
    r = random.Random(2000 + iv_len)
    for key_len in (16, 32):
        key, iv = rnd(r, key_len), rnd(r, iv_len)
        check_case(torch_cuda, ctx, key, iv, rnd(r, 9), rnd(r, 777))


def test_many_tiles_with_ragged_tail(torch_cuda, ctx):
    # Enough blocks for tens of tiles at the smallest tile size, plus a
    # partial final block and an AAD that straddles a tile boundary.
    r = random.Random(3000)
    for n, a in ((16 * 1024 * 70 + 9, 3000), (16 * 1024 * 5 + 16, 0), (16 * 1024 * 600 + 1, 17)):
        key, iv = rnd(r, 32), rnd(r, 12)
        pt = workloads.random_bytes(3000 + n, n).tobytes()
        check_case(torch_cuda, ctx, key, iv, rnd(r, a), pt)


def test_counter_wrap(torch_cuda, ctx):
    # non-96-bit IV whose J0 low word is near 2^32: inc32 wraps mid-message
    import ctypes

    r = random.Random(4000)
    key = rnd(r, 16)
    h, _, _ = oracle.h_j0(key, bytes(12))
    hb = ctypes.create_string_buffer(h, 16)
    out = ctypes.create_string_buffer(16)
    nblocks = 1 << 16
    for _ in range(1 << 24):
        iv = rnd(r, 16)
        ivb = ctypes.create_string_buffer(iv, 16)
        oracle.lib().oracle_j0(ctypes.addressof(hb), ctypes.addressof(ivb), 16, ctypes.addressof(out))
        low = int.from_bytes(out.raw[12:16], "big")
        if (1 << 32) - nblocks + 100 <= low:
            break
    pt = workloads.random_bytes(4001, 16 * nblocks - 3).tobytes()
    check_case(torch_cuda, ctx, key, iv, b"wrap", pt)


def test_tamper_rejected_and_zero_filled(torch_cuda, ctx):
    r = random.Random(5000)
    key, iv, aad = rnd(r, 32), rnd(r, 12), rnd(r, 40)
    pt = rnd(r, 3000)
    ct, tag = oracle.gcm_encrypt(key, iv, aad, pt)
    for which in ("ct", "aad", "tag"):
        for _ in range(6):
            args = {"ct": bytearray(ct), "aad": bytearray(aad), "tag": bytearray(tag)}
            buf = args[which]
            bit = r.randrange(8 * len(buf))
            buf[bit // 8] ^= 1 << (bit % 8)
            ok, out = gpu_decrypt(torch_cuda, ctx, key, iv, bytes(args["aad"]), bytes(args["ct"]),
                                  bytes(args["tag"]))
            assert not ok
            assert out == bytes(len(ct))


def test_in_place(torch_cuda, ctx):
    torch = torch_cuda
    r = random.Random(6000)
    key, iv, aad, pt = rnd(r, 16), rnd(r, 12), rnd(r, 3), rnd(r, 100000)
    ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, aad, pt)
    buf = to_dev(torch, pt)
    a = to_dev(torch, aad)
    _, tag = ctx.encrypt_device(key, iv, a, buf, ct=buf)
    torch.cuda.synchronize()
    assert to_bytes(buf) == ref_ct and to_bytes(tag) == ref_tag
    ctx.decrypt_verify_device(key, iv, a, buf, tag, pt=buf)
    torch.cuda.synchronize()
    assert to_bytes(buf) == pt


@pytest.mark.parametrize("host_access", [0, 2])
def test_host_mode(torch_cuda, ctx, host_access):
    ctx.set_host_access(host_access)
    r = random.Random(7000)
    key, iv, aad = rnd(r, 32), rnd(r, 12), rnd(r, 2880)
    pt = workloads.random_bytes(7001, 300000).tobytes()
    ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, aad, pt)
    ct, tag = ctx.encrypt_host(key, iv, aad, np.frombuffer(pt, dtype=np.uint8).copy())
    assert ct.tobytes() == ref_ct and tag == ref_tag
    back = ctx.decrypt_verify_host(key, iv, aad, ct, tag)
    assert back.tobytes() == pt
    from paper_2602_23067_gb300 import GcmError

    bad = bytearray(tag)
    bad[0] ^= 1
    out = np.full(len(pt), 7, np.uint8)
    with pytest.raises(GcmError):
        ctx.decrypt_verify_host(key, iv, aad, ct, bytes(bad), pt=out)
    assert not out.any()  # payload suppressed in host memory
    ctx.set_host_access(0)


@pytest.mark.parametrize("host_access", [0, 2])
def test_host_mode_page_locked(torch_cuda, ctx, host_access):
    # Buffers from gcm_host_alloc (exact size, page-locked), in place: the
    # kernels on the host memory directly (0) and the staged copy pipeline (2).
    from paper_2602_23067_gb300 import HostBuffer

    torch = torch_cuda
    ctx.set_host_access(host_access)
    r = random.Random(7100 + host_access)
    key, iv, aad = rnd(r, 16), rnd(r, 60), rnd(r, 100)
    n = 1000003
    pt = workloads.random_bytes(7101, n).tobytes()
    ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, aad, pt)
    with HostBuffer(n) as hb:
        assert hb.tensor.numel() == n and hb.ptr % 16 == 0
        hb.tensor.copy_(torch.frombuffer(bytearray(pt), dtype=torch.uint8))
        _, tag = ctx.encrypt_host(key, iv, aad, hb.tensor, ct=hb.tensor)
        assert tag == ref_tag and bytes(hb.tensor.numpy()) == ref_ct
        ctx.decrypt_verify_host(key, iv, aad, hb.tensor, tag, pt=hb.tensor)
        assert bytes(hb.tensor.numpy()) == pt
    ctx.set_host_access(0)


def test_fits_shaped_file(torch_cuda, ctx):
    # header records in clear as AAD, 2880-padded data unit as payload
    f = workloads.fits_file_host(8, 300, 200, n_sources=20)
    header, data, _ = oracle.fits_split(f)
    key, iv = bytes(range(32)), bytes(range(12))
    check_case(torch_cuda, ctx, key, iv, header, data)


def test_invalid_arguments(torch_cuda, ctx):
    from paper_2602_23067_gb300 import GcmError

    torch = torch_cuda
    p = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(GcmError) as e:
        ctx.encrypt_device(bytes(15), bytes(12), None, p)
    assert e.value.code == -1
    with pytest.raises(GcmError) as e:
        ctx.encrypt_device(bytes(16), b"", None, p)
    assert e.value.code == -1
    with pytest.raises(GcmError) as e:
        ctx.encrypt_device(bytes(16), bytes(12), None, p[1:33], ct=torch.zeros(32, dtype=torch.uint8, device="cuda"))
    assert e.value.code == -7


def test_hbm_budget_refuses_scratch(torch_cuda):
    # An allocation failure made on the host side: a context whose HBM
    # budget cannot hold one call's scratch refuses the call with
    # GCM_ERR_NO_MEMORY (-4) and stays usable; an unlimited context then
    # gives the oracle's result for the same inputs.
    from paper_2602_23067_gb300 import Context, GcmError

    torch = torch_cuda
    key, iv = bytes(range(16)), bytes(12)
    pt = workloads.random_bytes(77, 1 << 16).tobytes()
    p = torch.frombuffer(bytearray(pt), dtype=torch.uint8).cuda()
    with Context(0, hbm_budget_bytes=4096) as small:
        for _ in range(2):
            with pytest.raises(GcmError) as e:
                small.encrypt_device(key, iv, None, p)
            assert e.value.code == -4
    with Context(0) as ctx:
        ct, tag = ctx.encrypt_device(key, iv, None, p)
        torch.cuda.synchronize()
        ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, b"", pt)
        assert bytes(ct.cpu().numpy()) == ref_ct and bytes(tag.cpu().numpy()) == ref_tag
