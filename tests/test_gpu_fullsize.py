"""Full-size parity for the single large message (AES-256, a 32768 x 32768
float32 FITS image: 4,294,969,920 bytes of record-padded data unit behind a
2880-byte header used as AAD), in the same launch configuration the
benchmark times.

The oracle cannot run 4 GiB in test time, so the checks are ones it can make
one item at a time or that hold at any size:
  * sampled ciphertext blocks equal P_j xor E_K(inc32^j(J0)), block by block;
  * decrypt-verify of the ciphertext returns the plaintext;
  * GHASH is linear in C: for a ciphertext that is zero except at chosen
    blocks, the tag has a closed form the oracle evaluates with a few powers
    of H (so the tree combine, tile placement and length block are checked
    at full scale), and changing chosen blocks of the real ciphertext
    changes its tag by the same closed form.
"""
import random

import numpy as np
import pytest

import oracle
from paper_2602_23067_gb300 import workloads

pytestmark = pytest.mark.gpu

N1 = N2 = 32768
DATA_BYTES = N1 * N2 * 4
PADDED = workloads.padded_len(DATA_BYTES)


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_23067_gb300 import Context

    ctx = Context(0)
    r = workloads.rng(2)
    key = r.integers(0, 256, 32, dtype=np.uint8).tobytes()
    iv = r.integers(0, 256, 12, dtype=np.uint8).tobytes()
    header = workloads.fits_header(2, -32, [N1, N2], ncards=36)
    assert len(header) == 2880 and PADDED == 4294969920
    pt = torch.empty(PADDED, dtype=torch.uint8, device="cuda")
    workloads.sky_image_device(2, N1, N2, out=pt)
    aad = torch.frombuffer(bytearray(header), dtype=torch.uint8).cuda()
    ct, tag = ctx.encrypt_device(key, iv, aad, pt)
    torch.cuda.synchronize()
    yield torch, ctx, key, iv, header, aad, pt, ct, bytes(tag.cpu().numpy().tobytes())
    del pt, ct
    ctx.close()
    torch.cuda.empty_cache()


def blocks_at(torch, t, idx):
    ii = torch.tensor(idx, dtype=torch.int64, device=t.device)
    return t.view(-1, 16).index_select(0, ii).cpu().numpy()


def sample_indices(nblocks, seed, k=1500):
    r = random.Random(seed)
    idx = {0, 1, nblocks - 1, nblocks - 2}
    for m in (1 << 16, 1 << 15, 1 << 10):  # tile edges at several tile sizes
        for t in range(1, 8):
            for d in (-1, 0, 1):
                v = nblocks - t * m + d
                if 0 <= v < nblocks:
                    idx.add(v)
    while len(idx) < k:
        idx.add(r.randrange(nblocks))
    return sorted(idx)


def test_sampled_ciphertext_blocks(setup):
    torch, ctx, key, iv, header, aad, pt, ct, tag = setup
    n = PADDED // 16
    idx = sample_indices(n, 1)
    p = blocks_at(torch, pt, idx)
    c = blocks_at(torch, ct, idx)
    _, j0, _ = oracle.h_j0(key, iv)
    for k, j in enumerate(idx):
        ks = np.frombuffer(oracle.keystream_block(key, j0, j + 1), dtype=np.uint8)
        assert np.array_equal(c[k], p[k] ^ ks), j


def test_roundtrip(setup):
    torch, ctx, key, iv, header, aad, pt, ct, tag = setup
    t = torch.frombuffer(bytearray(tag), dtype=torch.uint8).cuda()
    out = torch.empty_like(ct)
    ctx.decrypt_verify_device(key, iv, aad, ct, t, pt=out)
    torch.cuda.synchronize()
    assert torch.equal(out, pt)
    del out


def _ghash_terms(h, blocks, positions, n):
    """sum_j C_j * H^(n + 2 - j) over 1-based payload block positions j."""
    acc = oracle.ZERO
    for blk, j in zip(blocks, positions):
        acc = oracle.xor16(acc, oracle.gf_mul(bytes(blk), oracle.gf_pow(h, n + 2 - j)))
    return acc


def test_sparse_ciphertext_closed_form_tag(setup):
    torch, ctx, key, iv, header, aad, pt, ct, tag = setup
    from paper_2602_23067_gb300 import GcmError

    n = PADDED // 16
    h, j0, ej0 = oracle.h_j0(key, iv)
    r = random.Random(3)
    idx = sample_indices(n, 4, k=300)
    vals = [bytes(r.getrandbits(8) for _ in range(16)) for _ in idx]
    sparse = torch.zeros(PADDED, dtype=torch.uint8, device="cuda")
    ii = torch.tensor(idx, dtype=torch.int64, device="cuda")
    sparse.view(-1, 16).index_copy_(0, ii, torch.tensor(np.frombuffer(b"".join(vals), dtype=np.uint8).reshape(-1, 16),
                                                         device="cuda"))
    a_hash = oracle.ghash(h, header)  # 2880 bytes = 180 whole blocks
    g = oracle.gf_mul(a_hash, oracle.gf_pow(h, n + 1))
    g = oracle.xor16(g, _ghash_terms(h, vals, [j + 1 for j in idx], n))
    lb = (8 * len(header)).to_bytes(8, "big") + (8 * PADDED).to_bytes(8, "big")
    g = oracle.xor16(g, oracle.gf_mul(lb, h))
    expected_tag = oracle.xor16(ej0, g)
    out = torch.empty_like(sparse)
    t = torch.frombuffer(bytearray(expected_tag), dtype=torch.uint8).cuda()
    ctx.decrypt_verify_device(key, iv, aad, sparse, t, pt=out)
    torch.cuda.synchronize()
    # plaintext = keystream where the ciphertext is zero
    got = blocks_at(torch, out, idx[:50])
    for k, j in enumerate(idx[:50]):
        ks = oracle.keystream_block(key, j0, j + 1)
        assert bytes(got[k]) == bytes(a ^ b for a, b in zip(vals[k], ks))
    # and a one-bit change of the tag is rejected with the output zero-filled
    bad = bytearray(expected_tag)
    bad[15] ^= 0x80
    tb = torch.frombuffer(bad, dtype=torch.uint8).cuda()
    with pytest.raises(GcmError):
        ctx.decrypt_verify_device(key, iv, aad, sparse, tb, pt=out)
    torch.cuda.synchronize()
    assert int(out.view(torch.int64).abs().sum().item()) == 0
    del sparse, out


def test_tag_shift_under_sparse_edits(setup):
    torch, ctx, key, iv, header, aad, pt, ct, tag = setup
    n = PADDED // 16
    h, _, _ = oracle.h_j0(key, iv)
    r = random.Random(5)
    idx = sample_indices(n, 6, k=64)
    deltas = [bytes(r.getrandbits(8) for _ in range(16)) for _ in idx]
    edited = ct.clone()
    ii = torch.tensor(idx, dtype=torch.int64, device="cuda")
    d = torch.tensor(np.frombuffer(b"".join(deltas), dtype=np.uint8).reshape(-1, 16), device="cuda")
    edited.view(-1, 16).index_copy_(0, ii, edited.view(-1, 16).index_select(0, ii) ^ d)
    new_tag = oracle.xor16(tag, _ghash_terms(h, deltas, [j + 1 for j in idx], n))
    t = torch.frombuffer(bytearray(new_tag), dtype=torch.uint8).cuda()
    out = torch.empty_like(edited)
    ctx.decrypt_verify_device(key, iv, aad, edited, t, pt=out)
    torch.cuda.synchronize()
    del edited, out
