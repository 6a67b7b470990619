"""Pins of the oracle's dual-key container (Sec. 3.2.2) against the
behaviour the paper states for its four access scenarios (Sec. 4.2, Table
"Role-based and temporal access control policies") and the FITS record
rules."""
import random

import pytest

import oracle
from oracle import container as C
from paper_2602_23067_gb300 import workloads

KH, KD = bytes(range(16)), bytes(range(100, 132))
NH, ND = bytes(range(12)), bytes(range(50, 62))


def _file(seed=3, n1=256, n2=256, bitpix=-32):
    hdr = workloads.fits_header(seed, bitpix, [n1, n2], ncards=36)
    data = workloads.sky_image_host(seed + 1, n1, n2, bitpix, n_sources=5).tobytes()
    return hdr + data + bytes(workloads.padded_len(len(data)) - len(data))


def test_record_structure_and_keywords():
    f = _file()
    c = C.container_encrypt(KH, KD, NH, ND, f)
    assert len(c) % 2880 == 0
    p, off = C.parse_header(c, 0)
    x, doff = C.parse_header(c, off)
    assert off % 2880 == 0 and doff % 2880 == 0
    for i in range(0, doff, 80):
        assert all(32 <= b < 127 for b in c[i: i + 80])
    assert p["NAXIS"] == "0" and x["XTENSION"] == "BINTABLE" and x["TFORM1"] == "%dB" % (256 * 256 * 4)
    assert (p["ORIG_BPX"], p["ORIG_NAX"], p["ORIG_NA1"], p["ORIG_NA2"]) == ("-32", "2", "256", "256")
    assert bytes.fromhex(p["NONCE_H"]) == NH and bytes.fromhex(p["NONCE_D"]) == ND
    header, padded, n = oracle.fits_split(f)
    assert len(bytes.fromhex(p["ENCHDR"])) == len(header)
    blob = c[doff: doff + n]
    assert int(x["DATASUM"]) == oracle.datasum(blob)
    # the blob is exactly GCM of the pixels under the data key with AAD_D
    ct, tag = oracle.gcm_encrypt(KD, ND, oracle.paper_aad_data(ND, -32, [256, 256]), padded[:n])
    assert blob == ct and bytes.fromhex(p["AUTHTG_D"]) == tag


def test_full_access_is_bit_exact():
    f = _file()
    out, w = C.decrypt_frame(C.container_encrypt(KH, KD, NH, ND, f), KH, KD)
    assert w == 0 and out == f


def test_metadata_only_suppresses_payload():
    f = _file()
    header, padded, n = oracle.fits_split(f)
    out, w = C.decrypt_frame(C.container_encrypt(KH, KD, NH, ND, f), KH, None)
    assert w == 2 and out[: len(header)] == header and out[len(header):] == bytes(len(padded))


def test_pixels_only_falls_back_to_minimal_header():
    f = _file()
    header, padded, n = oracle.fits_split(f)
    out, w = C.decrypt_frame(C.container_encrypt(KH, KD, NH, ND, f), None, KD)
    mh = C.minimal_header(-32, [256, 256])
    assert w == 1 and out[: len(mh)] == mh and out[len(mh):] == padded
    k, _ = C.parse_header(mh)
    assert k == {"SIMPLE": "T", "BITPIX": "-32", "NAXIS": "2", "NAXIS1": "256", "NAXIS2": "256"}
    # a wrong header key behaves like a missing one
    out2, w2 = C.decrypt_frame(C.container_encrypt(KH, KD, NH, ND, f), bytes(16), KD)
    assert (out2, w2) == (out, w)


def test_tampering_is_detected_per_part():
    f = _file()
    c = bytearray(C.container_encrypt(KH, KD, NH, ND, f))
    p, off = C.parse_header(bytes(c), 0)
    _, doff = C.parse_header(bytes(c), off)
    header, padded, n = oracle.fits_split(f)
    # pixel blob: payload suppressed, header still authenticated
    t = bytearray(c)
    t[doff + 777] ^= 4
    out, w = C.decrypt_frame(bytes(t), KH, KD)
    assert w == 2 and out[: len(header)] == header and out[len(header):] == bytes(len(padded))
    # plaintext structural keyword (context binding through AAD_D)
    t = bytes(c).replace(b"ORIG_NA1=                  256", b"ORIG_NA1=                  255")
    assert t != bytes(c)
    out, w = C.decrypt_frame(t, KH, KD)
    assert w == 2
    # encrypted header: fallback, pixels intact
    i = bytes(c).index(b"ENCHDR  = '") + 11
    t = bytearray(c)
    t[i] = ord("0") if t[i] != ord("0") else ord("1")
    out, w = C.decrypt_frame(bytes(t), KH, KD)
    assert w == 1 and out.endswith(padded)


def test_other_shapes():
    r = random.Random(5)
    for bitpix, n1, n2 in ((16, 77, 13), (16, 5, 5), (-32, 33, 2)):
        f = _file(r.randrange(1000), n1, n2, bitpix)
        out, w = C.decrypt_frame(C.container_encrypt(KH, KD, NH, ND, f), KH, KD)
        assert w == 0 and out == f


def _hdus(c):
    """(header bytes, data bytes) of both HDUs of a container."""
    _, off = C.parse_header(c, 0)
    x, doff = C.parse_header(c, off)
    n = int(x["NAXIS1"])
    return [(c[:off], b""), (c[off:doff], c[doff: doff + n + (-n) % 2880])]


@pytest.mark.parametrize("shape", [(256, 256, -32), (100, 37, 16), (1, 1, 16), (640, 3, -32)])
def test_checksum_closes_every_hdu(shape):
    # The defining property of CHECKSUM (FITS checksum convention, cited in
    # Sec. 3.2.2): with the card in place the HDU sums to -0, and DATASUM is
    # the data unit's own sum ('0' for the data-less primary HDU).
    f = _file(7, shape[0], shape[1], shape[2])
    c = C.container_encrypt(KH, KD, NH, ND, f)
    for hdr, data in _hdus(c):
        keys, _ = C.parse_header(hdr, 0)
        assert int(keys["DATASUM"]) == (oracle.datasum(data) if data else 0)
        assert oracle.datasum(hdr + data) == 0xFFFFFFFF
        v = keys["CHECKSUM"]
        assert len(v) == 16 and v.isalnum() and v.isascii()


def test_checksum_detects_a_flipped_bit():
    f = _file(8)
    c = bytearray(C.container_encrypt(KH, KD, NH, ND, f))
    r = random.Random(81)
    (h0, _), (h1, d1) = _hdus(bytes(c))
    for pos in [r.randrange(len(h0)), len(h0) + r.randrange(len(h1)), len(h0) + len(h1) + r.randrange(len(d1))]:
        t = bytearray(c)
        t[pos] ^= 1 << r.randrange(8)
        sums = [oracle.datasum(h + d) for h, d in _hdus(bytes(t))]
        assert sums.count(0xFFFFFFFF) == 1  # the damaged HDU no longer sums to -0, the other still does


def test_checksum_chars_sum_per_byte_lane():
    # Realigned to words (undo the rotation), the 16 characters add up, byte
    # lane by byte lane, to the encoded value plus 4 * 0x30 in every lane.
    r = random.Random(82)
    values = [0, 1, 0xFFFFFFFF, 0x7FFFFFFF, 0x80000000, 0x3A3A3A3A, 0xE8E8E8E8] + \
        [r.getrandbits(32) for _ in range(3000)]
    for v in values:
        s = C.checksum_chars(v)
        assert s.isalnum() and len(s) == 16
        aligned = (s[1:] + s[:1]).encode("ascii")
        lanes = [sum(aligned[4 * j + i] for j in range(4)) for i in range(4)]
        assert lanes == [((v >> (24 - 8 * i)) & 0xFF) + 4 * 0x30 for i in range(4)], hex(v)
