"""The two halves of the fused pass on their own (gcm_ctr_xor, gcm_ghash)
vs the oracle, bit for bit.

CTR alone must give exactly the GCM ciphertext (SP 800-38D GCTR from
inc32(J0)); GHASH alone must give the serial GHASH of
A || pad || C || pad || [len(A)]_64 || [len(C)]_64, and xoring it with
E_K(J0) must give the GCM tag of the same (A, C)."""
import random

import pytest

import oracle
from paper_2602_23067_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_23067_gb300 import Context

    c = Context(0)
    yield torch, c
    c.close()


def rnd(r, n):
    return bytes(r.getrandbits(8) for _ in range(n))


def dev(torch, b):
    t = torch.empty(len(b), dtype=torch.uint8, device="cuda")
    if b:
        t.copy_(torch.frombuffer(bytearray(b), dtype=torch.uint8))
    return t


def ghash_input(aad, c):
    def pad(x):
        return x + bytes(-len(x) % 16)

    return pad(aad) + pad(c) + (8 * len(aad)).to_bytes(8, "big") + (8 * len(c)).to_bytes(8, "big")


LENGTHS = (1, 15, 16, 17, 255, 256, 257, 4097, 16 * 1024 * 70 + 9, 16 * 1024 * 600 + 1)


@pytest.mark.parametrize("key_len", [16, 24, 32])
def test_ctr_alone_is_the_gcm_ciphertext(env, key_len):
    torch, ctx = env
    r = random.Random(8100 + key_len)
    for n in LENGTHS:
        key, iv = rnd(r, key_len), rnd(r, r.choice((12, 12, 7, 16, 60)))
        pt = workloads.random_bytes(8100 + n, n).tobytes()
        ref_ct, _ = oracle.gcm_encrypt(key, iv, b"", pt)
        x = dev(torch, pt)
        y = ctx.ctr_xor_device(key, iv, x)
        ctx.sync()  # gcm_sync on torch's current stream
        assert bytes(y.cpu().numpy()) == ref_ct, n
        # involution, in place
        ctx.ctr_xor_device(key, iv, y, out=y)
        torch.cuda.synchronize()
        assert bytes(y.cpu().numpy()) == pt


@pytest.mark.parametrize("aad_len", [0, 1, 16, 20, 2880, 2881])
def test_ghash_alone_matches_serial_ghash(env, aad_len):
    torch, ctx = env
    r = random.Random(8200 + aad_len)
    for n in (0, 1, 16, 17, 4096, 16 * 1024 * 70 + 9, 16 * 1024 * 600 + 1):
        key = rnd(r, r.choice((16, 32)))
        aad = rnd(r, aad_len)
        c = workloads.random_bytes(8200 + n, n).tobytes()
        h, _, _ = oracle.h_j0(key, bytes(12))
        ref = oracle.ghash(h, ghash_input(aad, c))
        s = ctx.ghash_device(key, dev(torch, aad) if aad else None, dev(torch, c))
        torch.cuda.synchronize()
        assert bytes(s.cpu().numpy()) == ref, (n, aad_len)


def test_ghash_xor_ej0_is_the_tag(env):
    torch, ctx = env
    r = random.Random(8300)
    key, iv, aad = rnd(r, 32), rnd(r, 12), rnd(r, 2880)
    pt = workloads.random_bytes(8301, 1 << 20).tobytes()
    ct, tag = oracle.gcm_encrypt(key, iv, aad, pt)
    _, _, ej0 = oracle.h_j0(key, iv)
    s = ctx.ghash_device(key, dev(torch, aad), dev(torch, ct))
    torch.cuda.synchronize()
    assert bytes(a ^ b for a, b in zip(bytes(s.cpu().numpy()), ej0)) == tag
