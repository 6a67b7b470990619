"""Parity at the largest message GCM allows: 2^36 - 32 bytes of plaintext
(2^39 - 256 bits, SP 800-38D Sec. 5.2.1.1).  Its 2^32 - 2 blocks use every
value of the 32-bit counter word that a 96-bit IV leaves for data (the last
block is encrypted under counter word 2^32 - 1), and with a 2900-byte AAD
the GHASH sequence spans 65,537 tiles of 2^16 blocks, so the tree combine
runs 17 levels through its global-memory levels before the shared-memory
ones.

The oracle cannot hash 68.7 GB in test time; GHASH is linear in the
ciphertext, so a ciphertext that is zero except at chosen blocks has a tag
the oracle evaluates in closed form from a few powers of H:
  * decrypt-verify of that sparse ciphertext with the closed-form tag must
    accept, and sampled plaintext blocks must equal C_j xor
    E_K(inc32^(j+1)(J0)) (the oracle's keystream, block by block, including
    the last counters);
  * re-encrypting the plaintext must give back the same tag and exactly the
    sparse ciphertext (sampled blocks, and the count of nonzero words over
    the whole buffer);
  * one block more than the limit, or one byte more, is refused before any
    device work (GCM_ERR_LENGTH_LIMIT).
One device buffer of 2^36 - 16 bytes is used in place throughout.
"""
import random

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

MAXLEN = (1 << 36) - 32
AAD_LEN = 2900  # 181 whole blocks and a 4-byte tail


@pytest.fixture(scope="module")
def big():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < MAXLEN + (8 << 30):
        pytest.skip("needs %.0f GB of free device memory, %.0f GB free" % ((MAXLEN + (8 << 30)) / 1e9, free / 1e9))
    from paper_2602_23067_gb300 import Context

    ctx = Context(0)
    buf = torch.zeros(MAXLEN + 16, dtype=torch.uint8, device="cuda")
    yield torch, ctx, buf
    del buf
    ctx.close()
    torch.cuda.empty_cache()


def _sample(n, seed, k=240):
    r = random.Random(seed)
    idx = {0, 1, 2, n - 1, n - 2, n - 3}
    for t in range(1, 6):  # tile edges (tiles of 2^16 blocks end at the sequence end)
        for d in (-1, 0, 1):
            idx.add(n - t * (1 << 16) + d)
    while len(idx) < k:
        idx.add(r.randrange(n))
    return sorted(idx)


def test_one_past_the_limit_is_refused(big):
    torch, ctx, buf = big
    from paper_2602_23067_gb300 import GcmError
    from paper_2602_23067_gb300._native import GCM_ERR_LENGTH_LIMIT

    key, iv = bytes(range(16)), bytes(12)
    for n in (MAXLEN + 16, MAXLEN + 1):
        view = buf[:n]
        with pytest.raises(GcmError) as e:
            ctx.encrypt_device(key, iv, None, view, ct=view)
        assert e.value.code == GCM_ERR_LENGTH_LIMIT
        t = torch.zeros(16, dtype=torch.uint8, device="cuda")
        with pytest.raises(GcmError) as e:
            ctx.decrypt_verify_device(key, iv, None, view, t, pt=view)
        assert e.value.code == GCM_ERR_LENGTH_LIMIT
    torch.cuda.synchronize()
    assert int(torch.count_nonzero(buf[-(1 << 20):]).item()) == 0  # nothing was written


def test_max_length_sparse_ciphertext(big):
    torch, ctx, buf = big
    n = MAXLEN // 16
    assert n == (1 << 32) - 2
    r = np.random.default_rng(40)
    key = r.integers(0, 256, 32, dtype=np.uint8).tobytes()
    iv = r.integers(0, 256, 12, dtype=np.uint8).tobytes()
    aad = r.integers(0, 256, AAD_LEN, dtype=np.uint8).tobytes()
    aad_dev = torch.frombuffer(bytearray(aad), dtype=torch.uint8).cuda()
    h, j0, ej0 = oracle.h_j0(key, iv)

    idx = _sample(n, 41)
    pr = random.Random(42)
    vals = [bytes(pr.getrandbits(8) for _ in range(16)) for _ in idx]
    data = buf[:MAXLEN]
    blocks = data.view(-1, 16)
    ii = torch.tensor(idx, dtype=torch.int64, device="cuda")
    blocks.index_copy_(0, ii, torch.tensor(np.frombuffer(b"".join(vals), dtype=np.uint8).reshape(-1, 16),
                                           device="cuda"))

    # GHASH of A || 0pad || C || [len A]_64 || [len C]_64 with C zero except at idx:
    # the AAD part times H^(n+1), block j (0-based) times H^(n+1-j), the length block times H.
    apad = aad + bytes(-len(aad) % 16)
    g = oracle.gf_mul(oracle.ghash(h, apad), oracle.gf_pow(h, n + 1))
    for v, j in zip(vals, idx):
        g = oracle.xor16(g, oracle.gf_mul(v, oracle.gf_pow(h, n + 1 - j)))
    lb = (8 * AAD_LEN).to_bytes(8, "big") + (8 * MAXLEN).to_bytes(8, "big")
    g = oracle.xor16(g, oracle.gf_mul(lb, h))
    expected_tag = oracle.xor16(ej0, g)

    t = torch.tensor(list(expected_tag), dtype=torch.uint8, device="cuda")
    ctx.decrypt_verify_device(key, iv, aad_dev, data, t, pt=data)  # raises GcmError if the tag differs
    torch.cuda.synchronize()

    zeros_at = sorted(set(random.Random(43).randrange(n) for _ in range(60)) - set(idx))
    check = idx + zeros_at
    got = blocks.index_select(0, torch.tensor(check, dtype=torch.int64, device="cuda")).cpu().numpy()
    cval = dict(zip(idx, vals))
    for k, j in enumerate(check):
        ks = oracle.keystream_block(key, j0, j + 1)
        c = cval.get(j, bytes(16))
        assert bytes(got[k]) == oracle.xor16(c, ks), j

    _, tag = ctx.encrypt_device(key, iv, aad_dev, data, ct=data)
    torch.cuda.synchronize()
    assert bytes(tag.cpu().numpy().tobytes()) == expected_tag
    got = blocks.index_select(0, torch.tensor(check, dtype=torch.int64, device="cuda")).cpu().numpy()
    for k, j in enumerate(check):
        assert bytes(got[k]) == cval.get(j, bytes(16)), j
    words = data.view(torch.int64)
    nonzero = 0
    step = 1 << 27
    for s in range(0, words.numel(), step):
        nonzero += int(torch.count_nonzero(words[s:s + step]).item())
    expected_nonzero = sum((v[:8] != bytes(8)) + (v[8:] != bytes(8)) for v in vals)
    assert nonzero == expected_nonzero
