"""Pins for the CPU oracle (no GPU).

Each test ties the oracle to something other than itself: an independent
library (pyca/cryptography on top of OpenSSL, where installed), an
independent formulation of the same arithmetic (polynomial long division for
GF(2^128)), algebraic identities that a dropped term, a wrong sign/index or a
transposed operand would break, brute force over small cases, and the worked
example the paper prints (Sec. 3.2.3).
"""
import os
import random

import pytest

import oracle
from paper_2602_23067_gb300 import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


def rnd(r, n):
    return bytes(r.getrandbits(8) for _ in range(n))


# --------------------------------------------------------------------------
# AES (FIPS-197)
# --------------------------------------------------------------------------

def test_sbox_is_a_permutation_without_fixed_points():
    s, inv = oracle.sbox()
    assert sorted(s) == list(range(256))
    for x in range(256):
        assert inv[s[x]] == x
        # Design properties of the AES S-box: no fixed points and no
        # "opposite" fixed points.  A wrong affine constant or rotation set
        # breaks them.
        assert s[x] != x
        assert s[x] != x ^ 0xFF


def test_sbox_inverse_relation():
    # FIPS-197 eq. 5.1: S(x) = A(x^-1) xor 0x63 with A linear over GF(2).
    # Undo the inversion (found by search with the oracle's GF(2^8) product)
    # and the constant, and check that what is left is linear.
    s, _ = oracle.sbox()
    inv = {0: 0}
    for a in range(1, 256):
        for b in range(1, 256):
            if oracle.gf8_mul(a, b) == 1:
                inv[a] = b
                break
    aff = [s[inv[x]] ^ 0x63 for x in range(256)]  # = A(x)
    for a in range(256):
        for b in (1, 2, 4, 8, 16, 32, 64, 128):
            assert aff[a ^ b] == aff[a] ^ aff[b]


def test_gf8_field_identities():
    r = random.Random(8)
    for _ in range(300):
        a, b, c = r.randrange(256), r.randrange(256), r.randrange(256)
        m = oracle.gf8_mul
        assert m(a, b) == m(b, a)
        assert m(m(a, b), c) == m(a, m(b, c))
        assert m(a, b ^ c) == m(a, b) ^ m(a, c)
        assert m(a, 1) == a
    # the multiplicative group has order 255 and 0x03 generates it
    x, seen = 1, set()
    for _ in range(255):
        seen.add(x)
        x = oracle.gf8_mul(x, 3)
    assert x == 1 and len(seen) == 255


@pytest.mark.parametrize("key_len", [16, 24, 32])
def test_aes_against_cryptography(key_len):
    pytest.importorskip("cryptography")
    from cryptography.hazmat.primitives.ciphers import Cipher, algorithms, modes

    r = random.Random(key_len)
    for _ in range(40):
        key, blk = rnd(r, key_len), rnd(r, 16)
        enc = Cipher(algorithms.AES(key), modes.ECB()).encryptor()
        assert oracle.aes_encrypt_block(key, blk) == enc.update(blk) + enc.finalize()


@pytest.mark.parametrize("key_len", [16, 24, 32])
def test_aes_inverse_cipher_roundtrip(key_len):
    r = random.Random(100 + key_len)
    for _ in range(40):
        key, blk = rnd(r, key_len), rnd(r, 16)
        c = oracle.aes_encrypt_block(key, blk)
        assert c != blk
        assert oracle.aes_decrypt_block(key, c) == blk


def test_key_expansion_lengths():
    for kl, nr in ((16, 10), (24, 12), (32, 14)):
        w, got = oracle.key_expansion(bytes(kl))
        assert got == nr and len(w) == 16 * (nr + 1)
        assert w[:kl] == bytes(kl)  # the first Nk words are the key itself
    with pytest.raises(ValueError):
        oracle.key_expansion(bytes(20))


# --------------------------------------------------------------------------
# GF(2^128) (SP 800-38D Algorithm 1)
# --------------------------------------------------------------------------

POLY = (1 << 128) | 0x87  # x^128 + x^7 + x^2 + x + 1


def _to_poly(b: bytes) -> int:
    """Block -> integer whose bit i is the coefficient of x^i (bit 0 of the
    block, the MSB of byte 0, is x^0)."""
    v = int.from_bytes(b, "big")
    return int(format(v, "0128b")[::-1], 2)


def _from_poly(p: int) -> bytes:
    return int(format(p, "0128b")[::-1], 2).to_bytes(16, "big")


def _polymul(a: int, b: int) -> int:
    r = 0
    for i in range(128):
        if (a >> i) & 1:
            r ^= b << i
    for d in range(254, 127, -1):
        if (r >> d) & 1:
            r ^= POLY << (d - 128)
    return r


def test_gf128_mul_matches_polynomial_long_division():
    r = random.Random(128)
    for _ in range(200):
        x, y = rnd(r, 16), rnd(r, 16)
        assert oracle.gf_mul(x, y) == _from_poly(_polymul(_to_poly(x), _to_poly(y)))


def test_gf128_field_identities():
    r = random.Random(7)
    one, zero = oracle.ONE, oracle.ZERO
    for _ in range(60):
        a, b, c = rnd(r, 16), rnd(r, 16), rnd(r, 16)
        m, x = oracle.gf_mul, oracle.xor16
        assert m(a, b) == m(b, a)
        assert m(m(a, b), c) == m(a, m(b, c))
        assert m(a, x(b, c)) == x(m(a, b), m(a, c))
        assert m(a, one) == a and m(one, a) == a
        assert m(a, zero) == zero
    # x * x = x^2: the element "x" is 0x40 || 0^120 in the reflected order.
    xe = bytes([0x40]) + bytes(15)
    assert oracle.gf_mul(xe, xe) == bytes([0x20]) + bytes(15)
    # x^127 * x = x^128 = 1 + x + x^2 + x^7 = 0xE1 || 0^120 (the constant R)
    x127 = bytes(15) + b"\x01"
    assert oracle.gf_mul(x127, xe) == bytes([0xE1]) + bytes(15)


def test_gf128_frobenius_and_inverse():
    r = random.Random(11)
    for _ in range(3):
        a = rnd(r, 16)
        y = a
        for _ in range(128):
            y = oracle.gf_mul(y, y)
        assert y == a  # a^(2^128) = a
        inv = oracle.gf_pow(a, (1 << 128) - 2)
        assert oracle.gf_mul(a, inv) == oracle.ONE


def test_gf128_powers_add():
    r = random.Random(12)
    h = rnd(r, 16)
    for i, j in ((0, 5), (3, 4), (17, 33), (100, 1000), (1 << 20, 12345)):
        assert oracle.gf_mul(oracle.gf_pow(h, i), oracle.gf_pow(h, j)) == oracle.gf_pow(h, i + j)
    y = oracle.ONE
    for e in range(1, 20):
        y = oracle.gf_mul(y, h)
        assert y == oracle.gf_pow(h, e)


# --------------------------------------------------------------------------
# GHASH: serial (Eq. 1) versus the paper's tree (Fig. 3b)
# --------------------------------------------------------------------------

def test_ghash_special_cases():
    r = random.Random(13)
    h, x = rnd(r, 16), rnd(r, 16)
    assert oracle.ghash(h, b"") == oracle.ZERO
    assert oracle.ghash(h, x) == oracle.gf_mul(x, h)
    y = rnd(r, 16)
    # two blocks: (X1 * H xor X2) * H = X1 H^2 + X2 H
    assert oracle.ghash(h, x + y) == oracle.xor16(oracle.gf_mul(x, oracle.gf_pow(h, 2)), oracle.gf_mul(y, h))


def test_ghash_tree_equals_serial_for_every_split_small():
    r = random.Random(14)
    h = rnd(r, 16)
    for n in range(1, 13):  # all 2^(n-1) ways to cut n blocks into chunks, n <= 12
        x = rnd(r, 16 * n)
        ref = oracle.ghash(h, x)
        for mask in range(1 << (n - 1)):
            cuts = [i + 1 for i in range(n - 1) if (mask >> i) & 1]
            assert oracle.tree_ghash(h, x, cuts) == ref, (n, cuts)


def test_ghash_tree_equals_serial_random_splits():
    r = random.Random(15)
    h = rnd(r, 16)
    for n in (13, 17, 31, 40):
        x = rnd(r, 16 * n)
        ref = oracle.ghash(h, x)
        for _ in range(6):
            cuts = sorted(r.sample(range(1, n), r.randrange(0, n - 1)))
            assert oracle.tree_ghash(h, x, cuts) == ref


def test_ghash_fig2b_shape():
    r = random.Random(16)
    h = rnd(r, 16)
    for n in (1, 2, 4, 8, 16):
        x = rnd(r, 16 * n)
        assert oracle.tree_ghash_fig2b(h, x) == oracle.ghash(h, x)


def test_ghash_tree_detects_a_wrong_power():
    # Plant a mistake in the combine step (one power of H too many) and
    # check that the identity above would catch it.
    r = random.Random(17)
    h = rnd(r, 16)
    x = rnd(r, 16 * 6)
    blocks = [x[16 * i:16 * i + 16] for i in range(6)]
    left = oracle.chunk_partial(h, blocks[:2])
    right = oracle.chunk_partial(h, blocks[2:])
    good = oracle.combine(h, left, right, 4)
    bad = oracle.xor16(oracle.gf_mul(left, oracle.gf_pow(h, 5)), right)
    assert good == oracle.ghash(h, x)
    assert bad != oracle.ghash(h, x)


# --------------------------------------------------------------------------
# inc32 and GCTR
# --------------------------------------------------------------------------

def test_inc32_wraps_only_the_low_word():
    b = bytes(range(12)) + b"\xff\xff\xff\xff"
    assert oracle.inc32(b) == bytes(range(12)) + b"\x00\x00\x00\x00"
    b = bytes(12) + b"\x00\x00\x00\xff"
    assert oracle.inc32(b) == bytes(12) + b"\x00\x00\x01\x00"


def test_keystream_block_closed_form_matches_repeated_inc32():
    r = random.Random(18)
    key = rnd(r, 16)
    j0 = rnd(r, 12) + b"\xff\xff\xff\xfa"
    cb = j0
    for i in range(1, 12):
        cb = oracle.inc32(cb)
        assert oracle.keystream_block(key, j0, i) == oracle.aes_encrypt_block(key, cb)


def test_gctr_keystream_is_independent_of_the_plaintext():
    r = random.Random(19)
    key, iv = rnd(r, 32), rnd(r, 12)
    p1, p2 = rnd(r, 100), rnd(r, 100)
    c1, _ = oracle.gcm_encrypt(key, iv, b"", p1)
    c2, _ = oracle.gcm_encrypt(key, iv, b"", p2)
    ks1 = bytes(a ^ b for a, b in zip(c1, p1))
    ks2 = bytes(a ^ b for a, b in zip(c2, p2))
    assert ks1 == ks2
    _, j0, _ = oracle.h_j0(key, iv)
    assert j0 == iv + b"\x00\x00\x00\x01"
    for i in range(1, 7):
        assert ks1[16 * (i - 1):16 * i] == oracle.keystream_block(key, j0, i)[: len(ks1[16 * (i - 1):16 * i])]


# --------------------------------------------------------------------------
# Whole GCM
# --------------------------------------------------------------------------

def _crypto_gcm(key, iv, aad, pt):
    from cryptography.hazmat.primitives.ciphers import Cipher, algorithms, modes

    enc = Cipher(algorithms.AES(key), modes.GCM(iv)).encryptor()
    if aad:
        enc.authenticate_additional_data(aad)
    ct = enc.update(pt) + enc.finalize()
    return ct, enc.tag


def test_gcm_against_cryptography_random():
    pytest.importorskip("cryptography")
    r = random.Random(20)
    for case in range(10000):
        key = rnd(r, r.choice((16, 24, 32)))
        iv = rnd(r, 12 if r.random() < 0.6 else r.randrange(8, 129))
        aad = rnd(r, r.choice((0, r.randrange(0, 70), r.randrange(0, 700), r.randrange(0, 4097))))
        pt = rnd(r, r.choice((0, r.randrange(0, 48), r.randrange(0, 3000))))
        ct, tag = oracle.gcm_encrypt(key, iv, aad, pt)
        assert (ct, tag) == _crypto_gcm(key, iv, aad, pt), case
        ok, back = oracle.gcm_decrypt(key, iv, aad, ct, tag)
        assert ok and back == pt


def test_gcm_against_cryptography_long_messages():
    pytest.importorskip("cryptography")
    r = random.Random(21)
    for case in range(100):
        key = rnd(r, r.choice((16, 24, 32)))
        iv = rnd(r, 12 if r.random() < 0.6 else r.randrange(8, 129))
        aad = rnd(r, r.randrange(0, 4097))
        pt = rnd(r, r.randrange(0, 65537))
        ct, tag = oracle.gcm_encrypt(key, iv, aad, pt)
        assert (ct, tag) == _crypto_gcm(key, iv, aad, pt), case


def test_gcm_against_cryptography_aesgcm_96bit():
    pytest.importorskip("cryptography")
    from cryptography.hazmat.primitives.ciphers.aead import AESGCM

    r = random.Random(21)
    for kl in (16, 32):
        key, iv, aad = rnd(r, kl), rnd(r, 12), rnd(r, 20)
        pt = rnd(r, 65536 + 7)
        ct, tag = oracle.gcm_encrypt(key, iv, aad, pt)
        assert ct + tag == AESGCM(key).encrypt(iv, pt, aad)


def test_gcm_counter_wrap_against_cryptography():
    # A non-96-bit IV whose J0 low word sits just below 2^32, so the 32-bit
    # counter wraps inside the message (inc32 never carries into the IV part).
    pytest.importorskip("cryptography")
    import ctypes

    r = random.Random(22)
    key = rnd(r, 16)
    h, _, _ = oracle.h_j0(key, bytes(12))
    hb = ctypes.create_string_buffer(h, 16)
    out = ctypes.create_string_buffer(16)
    nblocks = 4096
    for _ in range(1 << 22):
        iv = rnd(r, 16)
        ivb = ctypes.create_string_buffer(iv, 16)
        oracle.lib().oracle_j0(ctypes.addressof(hb), ctypes.addressof(ivb), 16, ctypes.addressof(out))
        low = int.from_bytes(out.raw[12:16], "big")
        if low >= (1 << 32) - nblocks + 8:
            break
    else:
        pytest.fail("no IV found")
    pt = rnd(r, 16 * nblocks)
    ct, tag = oracle.gcm_encrypt(key, iv, b"hdr", pt)
    assert (ct, tag) == _crypto_gcm(key, iv, b"hdr", pt)


def test_gcm_short_ivs_roundtrip_and_j0_rule():
    # 1..7-byte IVs are outside the range the independent library accepts;
    # check J0 = GHASH(IV || 0-pad || [len(IV)]_64) by composing the serial
    # GHASH with the AES block function, and the round trip.
    r = random.Random(23)
    for ivl in range(1, 8):
        key, iv, pt = rnd(r, 16), rnd(r, ivl), rnd(r, 40)
        h, j0, ej0 = oracle.h_j0(key, iv)
        blk = iv + bytes(16 - ivl) + bytes(8) + (8 * ivl).to_bytes(8, "big")
        assert j0 == oracle.ghash(h, blk)
        assert ej0 == oracle.aes_encrypt_block(key, j0)
        ct, tag = oracle.gcm_encrypt(key, iv, b"A", pt)
        c1 = oracle.inc32(j0)
        assert ct[:16] == bytes(a ^ b for a, b in zip(pt[:16], oracle.aes_encrypt_block(key, c1)))
        ok, back = oracle.gcm_decrypt(key, iv, b"A", ct, tag)
        assert ok and back == pt


def test_tag_definition_by_composition():
    # T = E_K(J0) xor GHASH_H(A || 0 || C || 0 || [len A]_64 || [len C]_64),
    # recomposed from the serial GHASH and the block cipher.
    r = random.Random(24)
    key, iv, aad, pt = rnd(r, 32), rnd(r, 12), rnd(r, 37), rnd(r, 91)
    ct, tag = oracle.gcm_encrypt(key, iv, aad, pt)
    h, j0, ej0 = oracle.h_j0(key, iv)
    s = aad + bytes((-len(aad)) % 16) + ct + bytes((-len(ct)) % 16)
    s += (8 * len(aad)).to_bytes(8, "big") + (8 * len(ct)).to_bytes(8, "big")
    assert tag == oracle.xor16(ej0, oracle.ghash(h, s))


def test_tamper_is_rejected_and_output_zeroed():
    r = random.Random(25)
    key, iv, aad, pt = rnd(r, 16), rnd(r, 12), rnd(r, 5), rnd(r, 21)
    ct, tag = oracle.gcm_encrypt(key, iv, aad, pt)
    # every single bit of ciphertext, AAD and tag
    for which in ("ct", "aad", "tag"):
        src = {"ct": ct, "aad": aad, "tag": tag}[which]
        for bit in range(8 * len(src)):
            mod = bytearray(src)
            mod[bit // 8] ^= 1 << (bit % 8)
            args = {"ct": ct, "aad": aad, "tag": tag}
            args[which] = bytes(mod)
            ok, out = oracle.gcm_decrypt(key, iv, args["aad"], args["ct"], args["tag"])
            assert not ok and out == bytes(len(ct))


def test_empty_message_and_empty_aad():
    pytest.importorskip("cryptography")
    r = random.Random(26)
    key, iv = rnd(r, 16), rnd(r, 12)
    assert oracle.gcm_encrypt(key, iv, b"", b"") == _crypto_gcm(key, iv, b"", b"")
    aad = rnd(r, 33)
    assert oracle.gcm_encrypt(key, iv, aad, b"") == _crypto_gcm(key, iv, aad, b"")


def test_bad_lengths_rejected():
    with pytest.raises(ValueError):
        oracle.gcm_encrypt(bytes(15), bytes(12), b"", b"x")
    with pytest.raises(ValueError):
        oracle.gcm_encrypt(bytes(16), b"", b"", b"x")


# --------------------------------------------------------------------------
# FITS framing (FITS standard 2880-byte records; the paper's AAD, Sec. 3.2.3)
# --------------------------------------------------------------------------

def test_paper_serialize_worked_example():
    with open(os.path.join(HERE, "golden", "serialize_example.txt")) as f:
        rows = [ln.rstrip("\n").split("\t") for ln in f if ln.strip() and not ln.startswith("#")]
    assert rows
    for value, expected in rows:
        assert oracle.serialize_int(int(value)) == expected.encode("ascii")


def test_paper_aad_layout():
    nonce = bytes(range(12))
    aad = oracle.paper_aad_data(nonce, -32, [256, 256])
    assert aad == nonce + b"-32" + b"2" + b"256" + b"256"


def test_fits_split_and_padding():
    for (n1, n2, bitpix) in ((100, 60, -32), (17, 3, 16), (48, 48, -32)):
        f = workloads.fits_file_host(5, n1, n2, bitpix=bitpix, n_sources=3)
        header, data, nbytes = oracle.fits_split(f)
        assert len(header) % 2880 == 0 and header.rstrip(b" ").endswith(b"END")
        assert nbytes == n1 * n2 * abs(bitpix) // 8
        assert len(data) % 2880 == 0 and len(data) - nbytes < 2880
        assert data[nbytes:] == bytes(len(data) - nbytes)
        assert header + data == f


def test_fits_encrypt_roundtrip_and_header_binding():
    f = workloads.fits_file_host(6, 40, 30, n_sources=2)
    key, iv = bytes(range(32)), bytes(range(12))
    enc, tag = oracle.fits_encrypt(key, iv, f)
    header, _, _ = oracle.fits_split(f)
    assert enc[: len(header)] == header  # header stays in clear
    assert enc[len(header):] != f[len(header):]
    ok, dec = oracle.fits_decrypt(key, iv, enc, tag)
    assert ok and dec == f
    # editing a header card (kept in clear) breaks the data tag
    tampered = enc.replace(b"TTT3", b"TTT1", 1)
    assert tampered != enc
    ok, dec = oracle.fits_decrypt(key, iv, tampered, tag)
    assert not ok
