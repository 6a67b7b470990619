"""Full-size parity for the single large message (AES-256, a 32768 x 32768
float32 FITS image: 4,294,969,920 bytes of record-padded data unit behind a
2880-byte header used as AAD), through the call and launch configuration the
benchmark times (gfc_fits_encrypt / gfc_fits_decrypt_verify on the device
FITS file), and through the plain gcm_encrypt.

* The whole ciphertext and the tag against the oracle: the oracle's own
  definitions run chunk by chunk on all host cores (``oracle.mapreduce``:
  GCTR from each chunk's counter, serial GHASH per chunk, partials joined by
  Combine, the length block and E_K(J0)); the ciphertexts are compared by
  the SHA-256 digests of their 64 MiB chunks, the tags byte for byte.
* The DATASUM computed in the cipher pass against the oracle's DATASUM of
  that (oracle-equal) ciphertext.
* Sampled ciphertext blocks against single oracle keystream blocks (tile
  edges at several tile sizes, both ends, random blocks).
* decrypt-verify of the ciphertext gives back the file; a sparse ciphertext
  whose tag the oracle evaluates in closed form (a few powers of H) is
  accepted, and a one-bit change of that tag is rejected with the output
  zero-filled.
"""
import random

import numpy as np
import pytest

import oracle
from oracle import mapreduce
from paper_2602_23067_gb300 import workloads

pytestmark = pytest.mark.gpu

N1 = N2 = 32768
DATA_BYTES = N1 * N2 * 4
PADDED = workloads.padded_len(DATA_BYTES)
CHUNK = 64 << 20


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
    hl = len(header)
    assert hl == 2880 and PADDED == 4294969920
    # the benchmark's FITS file: header records, then the padded data unit
    fits = torch.empty(hl + PADDED, dtype=torch.uint8, device="cuda")
    fits[:hl].copy_(torch.frombuffer(bytearray(header), dtype=torch.uint8))
    workloads.sky_image_device(2, N1, N2, out=fits[hl:])
    pt = fits[hl:]
    stream = torch.cuda.current_stream()
    enc, tag = ctx.fits_encrypt_raw(key, fits, iv, stream=stream)
    torch.cuda.synchronize()
    enc_file = Context.result_view(enc)
    assert enc_file.numel() == hl + PADDED
    aad = fits[:hl]
    ct_plain, tag_plain = ctx.encrypt_device(key, iv, aad, pt)
    torch.cuda.synchronize()
    yield {"torch": torch, "ctx": ctx, "key": key, "iv": iv, "header": header, "aad": aad, "fits": fits, "pt": pt,
           "enc": enc, "enc_file": enc_file, "ct": enc_file[hl:], "tag": tag, "datasum": int(enc.datasum),
           "datasum_valid": bool(enc.datasum_valid), "ct_plain": ct_plain,
           "tag_plain": bytes(tag_plain.cpu().numpy().tobytes())}
    ctx.release(enc)
    del fits, pt, ct_plain
    ctx.close()
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def oracle_ref(setup):
    """Digests and tag of the whole message from the chunked oracle."""
    torch = setup["torch"]
    with mapreduce.HostInput(PADDED) as src:
        torch.from_numpy(src.array).copy_(setup["pt"])
        (dg, tag), = mapreduce.gcm_encrypt_digests(
            [{"key": setup["key"], "iv": setup["iv"], "aad": setup["header"], "off": 0, "len": PADDED}], src,
            chunk_bytes=CHUNK)
    return dg, tag


def host_digests(torch, t):
    host = torch.empty(t.numel(), dtype=torch.uint8)
    host.copy_(t)
    return mapreduce.digests(host.numpy(), CHUNK), host


def test_fits_call_whole_ciphertext_and_tag_against_the_oracle(setup, oracle_ref):
    torch = setup["torch"]
    ref_dg, ref_tag = oracle_ref
    assert len(ref_dg) == (PADDED + CHUNK - 1) // CHUNK
    assert setup["tag"] == ref_tag
    assert torch.equal(setup["enc_file"][:2880], setup["fits"][:2880])  # header stays in clear
    dg, host = host_digests(torch, setup["ct"])
    bad = [i for i, (a, b) in enumerate(zip(dg, ref_dg)) if a != b]
    assert not bad, "ciphertext chunks differing from the oracle: %s" % bad[:10]
    # DATASUM of the encrypted data unit, from the same pass
    assert setup["datasum_valid"]
    assert setup["datasum"] == oracle.datasum_ptr(host.data_ptr(), PADDED)
    del host


def test_plain_call_whole_ciphertext_and_tag_against_the_oracle(setup, oracle_ref):
    torch = setup["torch"]
    ref_dg, ref_tag = oracle_ref
    assert setup["tag_plain"] == ref_tag
    dg, host = host_digests(torch, setup["ct_plain"])
    assert dg == ref_dg
    del host


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
    torch = setup["torch"]
    n = PADDED // 16
    idx = sample_indices(n, 1)
    p = blocks_at(torch, setup["pt"], idx)
    c = blocks_at(torch, setup["ct"], idx)
    _, j0, _ = oracle.h_j0(setup["key"], setup["iv"])
    for k, j in enumerate(idx):
        ks = np.frombuffer(oracle.keystream_block(setup["key"], j0, j + 1), dtype=np.uint8)
        assert np.array_equal(c[k], p[k] ^ ks), j


def test_roundtrip_through_the_fits_call(setup):
    torch, ctx = setup["torch"], setup["ctx"]
    from paper_2602_23067_gb300 import Context

    enc = setup["enc"]
    dec = ctx.fits_decrypt_verify_raw(setup["key"], enc.data_buffer, enc.buffer_size, setup["iv"], setup["tag"],
                                      stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert dec.error_code == 0
    assert torch.equal(Context.result_view(dec), setup["fits"])
    ctx.release(dec)


def _ghash_terms(h, blocks, positions, n):
    """sum_j C_j * H^(n + 2 - j) over 1-based payload block positions j."""
    acc = oracle.ZERO
    for blk, j in zip(blocks, positions):
        acc = oracle.xor16(acc, oracle.gf_mul(bytes(blk), oracle.gf_pow(h, n + 2 - j)))
    return acc


def test_sparse_ciphertext_closed_form_tag(setup):
    torch, ctx = setup["torch"], setup["ctx"]
    key, iv, header, aad = setup["key"], setup["iv"], setup["header"], setup["aad"]
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
