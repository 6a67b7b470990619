"""The context's device key cache (gcm_ctx_set_key_cache): results with a
cached key (only J0 / E_K(J0) derived per call), after replacements in a
small cache, across two streams, and with the cache off are all the oracle's,
bit for bit."""
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


def rnd(r, n):
    return bytes(r.getrandbits(8) for _ in range(n))


def dev(torch, b):
    t = torch.empty(max(1, len(b)), dtype=torch.uint8, device="cuda")
    if b:
        t[: len(b)].copy_(torch.frombuffer(bytearray(b), dtype=torch.uint8))
    return t[: len(b)]


def enc_check(torch, ctx, key, iv, aad, pt, stream=None):
    ct, tag = ctx.encrypt_device(key, iv, dev(torch, aad) if aad else None, dev(torch, pt), stream=stream)
    return ct, tag, oracle.gcm_encrypt(key, iv, aad, pt)


def test_repeated_key_hits(torch_cuda):
    from paper_2602_23067_gb300 import Context

    torch = torch_cuda
    r = random.Random(9100)
    with Context(0) as ctx:
        key = rnd(r, 32)
        for iv_len in (12, 12, 7, 16, 60, 12):
            iv, aad = rnd(r, iv_len), rnd(r, r.choice((0, 20, 2880)))
            pt = workloads.random_bytes(r.randrange(1 << 30), r.choice((0, 17, 4096, 300001))).tobytes()
            ct, tag, (rc, rt) = enc_check(torch, ctx, key, iv, aad, pt)
            torch.cuda.synchronize()
            assert bytes(tag.cpu().numpy()) == rt and bytes(ct.cpu().numpy()) == rc
            back = ctx.decrypt_verify_device(key, iv, dev(torch, aad) if aad else None, ct, tag)
            assert bytes(back.cpu().numpy()) == pt


def test_small_cache_replacement(torch_cuda):
    from paper_2602_23067_gb300 import Context

    torch = torch_cuda
    r = random.Random(9200)
    with Context(0) as ctx:
        ctx.set_key_cache(2)
        keys = [rnd(r, r.choice((16, 24, 32))) for _ in range(5)]
        pending = []
        for rep in range(4):
            for key in keys:
                iv, aad = rnd(r, 12), rnd(r, 5)
                pt = workloads.random_bytes(rep * 10 + len(pending), 5000 + rep).tobytes()
                pending.append(enc_check(torch, ctx, key, iv, aad, pt))
        torch.cuda.synchronize()
        for ct, tag, (rc, rt) in pending:
            assert bytes(tag.cpu().numpy()) == rt and bytes(ct.cpu().numpy()) == rc
        ctx.set_key_cache(0)
        key, iv = keys[0], rnd(r, 12)
        ct, tag, (rc, rt) = enc_check(torch, ctx, key, iv, b"", b"cache off" * 100)
        torch.cuda.synchronize()
        assert bytes(tag.cpu().numpy()) == rt and bytes(ct.cpu().numpy()) == rc


def test_same_key_two_streams(torch_cuda):
    from paper_2602_23067_gb300 import Context

    torch = torch_cuda
    r = random.Random(9300)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with Context(0) as ctx:
        key = rnd(r, 16)
        pending = []
        for i in range(12):
            st = s1 if i % 2 == 0 else s2
            iv, aad = rnd(r, 12), rnd(r, 20)
            pt = workloads.random_bytes(9300 + i, (1 << 20) + i).tobytes()
            a, p = dev(torch, aad), dev(torch, pt)
            torch.cuda.synchronize()
            with torch.cuda.stream(st):
                ct, tag = ctx.encrypt_device(key, iv, a, p, stream=st)
            pending.append((ct, tag, oracle.gcm_encrypt(key, iv, aad, pt), a, p))
        torch.cuda.synchronize()
        for ct, tag, (rc, rt), _, _ in pending:
            assert bytes(tag.cpu().numpy()) == rt and bytes(ct.cpu().numpy()) == rc
