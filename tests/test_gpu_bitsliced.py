"""The bitsliced AES engine (gcm_ctx_set_aes_impl(ctx, GCM_AES_BITSLICED)) of
the fused pass against the CPU oracle, bit for bit: GCM ciphertexts and tags,
decrypt-verify with the validation gate, the CTR-only pass, every tile size
(so whole-payload segments of 32 .. 4096 blocks, windows of 1024 blocks that
end inside a segment), ragged tails, AAD, 96-bit and other IVs, and a
counter that wraps (inc32) inside a bitsliced window.  Every call goes
through the C ABI."""
import ctypes
import random

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
    from paper_2602_23067_gb300._native import GCM_AES_BITSLICED

    c = Context(0)
    c.set_aes_impl(GCM_AES_BITSLICED)
    yield c
    c.close()


def rnd(r, n):
    return bytes(r.getrandbits(8) for _ in range(n))


def dev(torch, b: bytes):
    t = torch.empty(max(1, len(b)), dtype=torch.uint8, device="cuda")
    if b:
        t[: len(b)].copy_(torch.frombuffer(bytearray(b), dtype=torch.uint8))
    return t[: len(b)]


def host(t) -> bytes:
    return bytes(t.cpu().numpy().tobytes())


def roundtrip(torch, ctx, key, iv, aad, pt):
    from paper_2602_23067_gb300 import GcmError

    ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, aad, pt)
    a = dev(torch, aad) if aad else None
    ct, tag = ctx.encrypt_device(key, iv, a, dev(torch, pt))
    torch.cuda.synchronize()
    assert host(tag) == ref_tag, "tag (len %d, aad %d, iv %d, key %d)" % (len(pt), len(aad), len(iv), len(key))
    assert host(ct) == ref_ct, "ciphertext (len %d)" % len(pt)
    back = ctx.decrypt_verify_device(key, iv, a, ct, tag)
    torch.cuda.synchronize()
    assert host(back) == pt
    if pt:
        bad = tag.clone()
        bad[0] ^= 1
        out = torch.full_like(ct, 0x5A)
        with pytest.raises(GcmError):
            ctx.decrypt_verify_device(key, iv, a, ct, bad, pt=out)
        torch.cuda.synchronize()
        assert not bool(out.any()), "output not zero-filled after a failed tag check"


def test_rejects_unknown_engine(ctx):
    from paper_2602_23067_gb300 import GcmError

    with pytest.raises(GcmError):
        ctx.set_aes_impl(7)


@pytest.mark.parametrize("key_len", [16, 24, 32])
def test_gcm_matches_oracle(torch_cuda, ctx, key_len):
    r = random.Random(12000 + key_len)
    cases = ((16 * 1024 * 70 + 9, 3000), (16 * 1024 * 5 + 16, 0), (1 << 20, 20), (16 * 4096 * 3, 2880),
             (16 * 1500, 0), (1, 0), (0, 33))
    for n, a in cases:
        key, iv = rnd(r, key_len), rnd(r, r.choice((12, 12, 12, 16, 60)))
        pt = workloads.random_bytes(12000 + n, n).tobytes()
        roundtrip(torch_cuda, ctx, key, iv, rnd(r, a), pt)


@pytest.mark.parametrize("tile_log2", list(range(9, 17)))
def test_every_tile_size(torch_cuda, tile_log2):
    from paper_2602_23067_gb300 import Context
    from paper_2602_23067_gb300._native import GCM_AES_BITSLICED

    r = random.Random(12100 + tile_log2)
    with Context(0) as c:
        c.set_aes_impl(GCM_AES_BITSLICED)
        c.set_tile_log2(tile_log2)
        for n, a in ((3 * (1 << 20) + 7, 2880), (16 * 1000 + 3, 17), (1 << 18, 0)):
            key, iv = rnd(r, 32), rnd(r, 12)
            pt = workloads.random_bytes(12100 + n, n).tobytes()
            roundtrip(torch_cuda, c, key, iv, rnd(r, a), pt)


@pytest.mark.parametrize("key_len", [16, 32])
def test_ctr_alone_matches_oracle(torch_cuda, ctx, key_len):
    r = random.Random(12200 + key_len)
    for n in (16 * 1024 * 70 + 9, 16 * 4096 * 4, 4097):
        key, iv = rnd(r, key_len), rnd(r, r.choice((12, 7)))
        pt = workloads.random_bytes(12200 + n, n).tobytes()
        ref_ct, _ = oracle.gcm_encrypt(key, iv, b"", pt)
        y = ctx.ctr_xor_device(key, iv, dev(torch_cuda, pt))
        torch_cuda.cuda.synchronize()
        assert host(y) == ref_ct, n


def test_counter_wrap_inside_a_window(torch_cuda, ctx):
    # A non-96-bit IV whose J0 low word is a little below 2^32: the counter
    # wraps (low 32 bits only) in the middle of the message.
    r = random.Random(12300)
    key = rnd(r, 32)
    h, _, _ = oracle.h_j0(key, bytes(12))
    hb = ctypes.create_string_buffer(h, 16)
    out = ctypes.create_string_buffer(16)
    nblocks = 1 << 16
    for _ in range(1 << 24):
        iv = rnd(r, 16)
        ivb = ctypes.create_string_buffer(iv, 16)
        oracle.lib().oracle_j0(ctypes.addressof(hb), ctypes.addressof(ivb), 16, ctypes.addressof(out))
        low = int.from_bytes(out.raw[12:16], "big")
        if (1 << 32) - nblocks + 1000 <= low <= (1 << 32) - 2000:
            break
    pt = workloads.random_bytes(12301, 16 * nblocks).tobytes()
    roundtrip(torch_cuda, ctx, key, iv, b"", pt)


def test_same_result_as_the_table_engine_on_a_large_message(torch_cuda):
    # 256 MiB + a ragged tail: both engines through the same API must agree
    # byte for byte; sampled blocks are checked against the oracle's
    # keystream (C_j = P_j xor E_K(inc32^(j+1)(J0))).
    from paper_2602_23067_gb300 import Context
    from paper_2602_23067_gb300._native import GCM_AES_BITSLICED, GCM_AES_TABLES

    torch = torch_cuda
    r = random.Random(12400)
    key, iv, aad = rnd(r, 32), rnd(r, 12), rnd(r, 2880)
    n = (256 << 20) + 13
    g = torch.Generator(device="cuda")
    g.manual_seed(12400)
    pt = torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda", generator=g)
    a = dev(torch, aad)
    outs = {}
    with Context(0) as c:
        for impl in (GCM_AES_TABLES, GCM_AES_BITSLICED):
            c.set_aes_impl(impl)
            ct, tag = c.encrypt_device(key, iv, a, pt)
            torch.cuda.synchronize()
            outs[impl] = (ct, host(tag))
    assert outs[GCM_AES_TABLES][1] == outs[GCM_AES_BITSLICED][1]
    assert torch.equal(outs[GCM_AES_TABLES][0], outs[GCM_AES_BITSLICED][0])
    _, j0, _ = oracle.h_j0(key, iv)
    ct = outs[GCM_AES_BITSLICED][0]
    for j in [0, 1, 31, 32, 1023, 1024, 4095, 4096, 65535, 65536] + [r.randrange(n // 16) for _ in range(40)]:
        ks = oracle.keystream_block(key, j0, j + 1)  # data block j (0-based) uses inc32^(j+1)(J0)
        p = host(pt[16 * j: 16 * j + 16])
        want = bytes(x ^ y for x, y in zip(p, ks))
        assert host(ct[16 * j: 16 * j + 16]) == want, j
