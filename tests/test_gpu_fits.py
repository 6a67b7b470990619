"""The FITS wrapper of the C ABI (gfc_fits_encrypt / gfc_fits_decrypt_verify)
against the oracle's FITS framing + GCM, in host and device memory."""
import numpy as np
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

    ctx = Context(0)
    yield torch, ctx
    ctx.close()


KEY = bytes(range(32))
IV = bytes(range(100, 112))


def _file(seed, n1, n2, bitpix=-32, ncards=36, pad=True):
    hdr = workloads.fits_header(seed, bitpix, [n1, n2], ncards=ncards)
    data = workloads.sky_image_host(seed + 1, n1, n2, bitpix, n_sources=5).tobytes()
    if pad:
        data += bytes(workloads.padded_len(len(data)) - len(data))
    return hdr + data


@pytest.mark.parametrize("where", ["host", "device"])
@pytest.mark.parametrize("shape", [(300, 200, -32, 36), (77, 13, 16, 50), (1024, 1024, -32, 36)])
def test_fits_roundtrip_header_aad(env, where, shape):
    torch, ctx = env
    f = _file(10, *shape)
    ref_enc, ref_tag = oracle.fits_encrypt(KEY, IV, f)
    inp = torch.frombuffer(bytearray(f), dtype=torch.uint8).cuda() if where == "device" else f
    r = ctx.fits_encrypt(KEY, inp, iv=IV)
    got = bytes(r.data.cpu().numpy()) if where == "device" else r.data.tobytes()
    assert r.error_code == 0 and r.tag == ref_tag and r.iv == IV
    assert got == ref_enc
    enc_in = torch.frombuffer(bytearray(got), dtype=torch.uint8).cuda() if where == "device" else got
    d = ctx.fits_decrypt_verify(KEY, enc_in, IV, r.tag)
    back = bytes(d.data.cpu().numpy()) if where == "device" else d.data.tobytes()
    assert d.error_code == 0 and d.warning_code == 0 and back == f
    # FITS DATASUM of the encrypted data unit, from the same pass, both ways
    hdr_len = len(oracle.fits_split(f)[0])
    ds = oracle.datasum(ref_enc[hdr_len:])
    assert r.datasum == ds and d.datasum == ds


def test_unpadded_input_is_zero_padded(env):
    torch, ctx = env
    f = _file(11, 101, 7, pad=False)
    full = f + bytes(workloads.padded_len(len(f) - 2880) - (len(f) - 2880))
    ref_enc, ref_tag = oracle.fits_encrypt(KEY, IV, full)
    r = ctx.fits_encrypt(KEY, f, iv=IV)
    assert r.tag == ref_tag and r.data.tobytes() == ref_enc


@pytest.mark.parametrize("where", ["host", "device"])
def test_structural_aad_mode(env, where):
    torch, ctx = env
    from paper_2602_23067_gb300 import GFC_AAD_STRUCTURAL

    f = _file(12, 256, 256)
    header, padded, _ = oracle.fits_split(f)
    aad = oracle.paper_aad_data(IV, -32, [256, 256])
    ref_ct, ref_tag = oracle.gcm_encrypt(KEY, IV, aad, padded)
    inp = torch.frombuffer(bytearray(f), dtype=torch.uint8).cuda() if where == "device" else f
    r = ctx.fits_encrypt(KEY, inp, iv=IV, aad_mode=GFC_AAD_STRUCTURAL)
    got = bytes(r.data.cpu().numpy()) if where == "device" else r.data.tobytes()
    assert r.tag == ref_tag and got == header + ref_ct
    # header cards outside the structural keywords are not authenticated in this mode
    edited = got.replace(b"TTT3", b"TTT9", 1)
    d = ctx.fits_decrypt_verify(KEY, edited, IV, r.tag, aad_mode=GFC_AAD_STRUCTURAL)
    assert d.error_code == 0
    # but the pixel geometry is
    edited = got.replace(b"NAXIS1  =                  256", b"NAXIS1  =                  128", 1)
    assert edited != got
    from paper_2602_23067_gb300 import GcmError

    try:
        d = ctx.fits_decrypt_verify(KEY, edited, IV, r.tag, aad_mode=GFC_AAD_STRUCTURAL)
        assert d.error_code != 0
    except GcmError:
        pass  # the edited geometry no longer matches the file length


@pytest.mark.parametrize("where", ["host", "device"])
def test_tampered_header_suppresses_payload(env, where):
    torch, ctx = env
    f = _file(13, 300, 100)
    r = ctx.fits_encrypt(KEY, f, iv=IV)
    enc = r.data.tobytes().replace(b"TTT3", b"TTT1", 1)
    inp = torch.frombuffer(bytearray(enc), dtype=torch.uint8).cuda() if where == "device" else enc
    d = ctx.fits_decrypt_verify(KEY, inp, IV, r.tag)
    out = bytes(d.data.cpu().numpy()) if where == "device" else d.data.tobytes()
    assert d.error_code == -3 and d.warning_code == 2
    hl = 2880
    assert out[:hl] == enc[:hl]                      # header returned as is
    assert out[hl:] == bytes(len(out) - hl)          # pixels physically zeroed
    ok, _ = oracle.fits_decrypt(KEY, IV, enc, r.tag)
    assert not ok


def test_random_iv_and_wrong_key(env):
    torch, ctx = env
    f = _file(14, 64, 64)
    r1 = ctx.fits_encrypt(KEY, f)
    r2 = ctx.fits_encrypt(KEY, f)
    assert len(r1.iv) == 12 and r1.iv != r2.iv
    ok, dec = oracle.fits_decrypt(KEY, r1.iv, r1.data.tobytes(), r1.tag)
    assert ok and dec == f
    d = ctx.fits_decrypt_verify(bytes(32), r1.data.tobytes(), r1.iv, r1.tag)
    assert d.warning_code == 2


def test_rejects_multi_hdu_and_non_fits(env):
    torch, ctx = env
    from paper_2602_23067_gb300 import GcmError

    f = _file(15, 10, 10)
    with pytest.raises(GcmError):
        ctx.fits_encrypt(KEY, f + bytes(2880), iv=IV)
    with pytest.raises(GcmError):
        ctx.fits_encrypt(KEY, b"\0" * 5760, iv=IV)


def test_datasum_of_tampered_file_is_reported(env):
    """The DATASUM is taken over the ciphertext as read, so a corrupted file
    shows a DATASUM different from the stored one even though the tag check
    (which rejects it) zero-fills the payload."""
    torch, ctx = env
    f = _file(12, 200, 100)
    r = ctx.fits_encrypt(KEY, f, iv=IV)
    enc = bytearray(r.data.tobytes())
    enc[2880 + 123] ^= 0x10
    d = ctx.fits_decrypt_verify(KEY, bytes(enc), IV, r.tag)
    assert d.error_code == -3 and d.warning_code == 2
    assert d.datasum == oracle.datasum(bytes(enc[2880:])) != r.datasum
