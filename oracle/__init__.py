"""CPU oracle for AES-GCM (test infrastructure only).

This package is the correctness oracle for the GPU library.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it.  The product path never imports it; the two share no code.

* ``gcm_oracle.c`` -- plain byte-at-a-time AES (FIPS-197) and GCM
  (NIST SP 800-38D, Algorithms 1-5), built into ``liboracle.so`` with gcc.
* this module -- a ctypes binding to it, plus plain-Python helpers that
  follow the paper:
    - ``tree_ghash``: the parallel tree form of GHASH (Sec. 3.3.1, Fig. 3b;
      Sec. 5.2.1-5.2.2), used only to pin the regrouping identity that the
      GPU relies on.  Product parity is always checked against the serial
      GHASH of SP 800-38D.
    - ``fits_split`` / ``fits_encrypt`` / ``fits_decrypt``: the FITS framing
      of the data path (header records in clear and authenticated as AAD,
      data unit zero-padded to whole 2880-byte records and encrypted).
    - ``paper_aad_data``: the paper's structural-keyword AAD
      (Sec. 3.2.3, the AAD_Data formula).
* ``mapreduce.py`` -- GCM of multi-GiB messages on many host cores: the same
  C functions applied chunk by chunk (GCTR from each chunk's counter, serial
  GHASH per chunk), the partials joined with ``combine``; it returns the
  tag and SHA-256 digests of the ciphertext chunks.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Iterable, List, Optional, Sequence, Tuple

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gcm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (no CUDA involved)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u8p = ctypes.c_void_p
        L.oracle_aes_key_expansion.argtypes = [u8p, ctypes.c_int, u8p]
        L.oracle_aes_key_expansion.restype = ctypes.c_int
        L.oracle_aes_encrypt_block.argtypes = [u8p, ctypes.c_int, u8p, u8p]
        L.oracle_aes_decrypt_block.argtypes = [u8p, ctypes.c_int, u8p, u8p]
        L.oracle_gf128_mul.argtypes = [u8p, u8p, u8p]
        L.oracle_ghash.argtypes = [u8p, u8p, ctypes.c_size_t, u8p]
        L.oracle_inc32.argtypes = [u8p]
        L.oracle_gctr.argtypes = [u8p, ctypes.c_int, u8p, u8p, ctypes.c_size_t, u8p]
        L.oracle_hash_subkey.argtypes = [u8p, ctypes.c_int, u8p]
        L.oracle_j0.argtypes = [u8p, u8p, ctypes.c_size_t, u8p]
        L.oracle_gcm_encrypt.argtypes = [u8p, ctypes.c_size_t, u8p, ctypes.c_size_t, u8p,
                                         ctypes.c_size_t, u8p, ctypes.c_size_t, u8p, u8p]
        L.oracle_gcm_encrypt.restype = ctypes.c_int
        L.oracle_gcm_decrypt.argtypes = [u8p, ctypes.c_size_t, u8p, ctypes.c_size_t, u8p,
                                         ctypes.c_size_t, u8p, ctypes.c_size_t, u8p, u8p]
        L.oracle_gcm_decrypt.restype = ctypes.c_int
        L.oracle_keystream_block.argtypes = [u8p, ctypes.c_size_t, u8p, ctypes.c_uint64, u8p]
        L.oracle_gcm_h_j0.argtypes = [u8p, ctypes.c_size_t, u8p, ctypes.c_size_t, u8p, u8p, u8p]
        L.oracle_gcm_h_j0.restype = ctypes.c_int
        L.oracle_sbox.argtypes = [u8p, u8p]
        L.oracle_gf8_mul.argtypes = [ctypes.c_uint8, ctypes.c_uint8]
        L.oracle_gf8_mul.restype = ctypes.c_uint8
        L.oracle_datasum.argtypes = [u8p, ctypes.c_size_t]
        L.oracle_datasum.restype = ctypes.c_uint32
        _lib = L
    return _lib


def _buf(data: bytes):
    """A ctypes buffer holding ``data`` (at least one byte so the pointer is valid)."""
    return ctypes.create_string_buffer(bytes(data), max(1, len(data)))


def _ptr(b) -> int:
    return ctypes.addressof(b)


# --------------------------------------------------------------------------
# AES (FIPS-197)
# --------------------------------------------------------------------------

def sbox() -> Tuple[bytes, bytes]:
    out, inv = ctypes.create_string_buffer(256), ctypes.create_string_buffer(256)
    lib().oracle_sbox(_ptr(out), _ptr(inv))
    return out.raw, inv.raw


def gf8_mul(a: int, b: int) -> int:
    return int(lib().oracle_gf8_mul(a, b))


def key_expansion(key: bytes) -> Tuple[bytes, int]:
    w = ctypes.create_string_buffer(240)
    kb = _buf(key)
    nr = lib().oracle_aes_key_expansion(_ptr(kb), len(key), _ptr(w))
    if nr < 0:
        raise ValueError("AES key must be 16, 24 or 32 bytes")
    return w.raw[: 16 * (nr + 1)], nr


def aes_encrypt_block(key: bytes, block: bytes) -> bytes:
    w, nr = key_expansion(key)
    wb, ib, ob = _buf(w), _buf(block), ctypes.create_string_buffer(16)
    lib().oracle_aes_encrypt_block(_ptr(wb), nr, _ptr(ib), _ptr(ob))
    return ob.raw


def aes_decrypt_block(key: bytes, block: bytes) -> bytes:
    w, nr = key_expansion(key)
    wb, ib, ob = _buf(w), _buf(block), ctypes.create_string_buffer(16)
    lib().oracle_aes_decrypt_block(_ptr(wb), nr, _ptr(ib), _ptr(ob))
    return ob.raw


# --------------------------------------------------------------------------
# GF(2^128) and GHASH (SP 800-38D Algorithms 1, 2)
# --------------------------------------------------------------------------

ONE = bytes([0x80]) + bytes(15)  # the multiplicative identity (x^0) in the reflected convention
ZERO = bytes(16)


def gf_mul(x: bytes, y: bytes) -> bytes:
    xb, yb, zb = _buf(x), _buf(y), ctypes.create_string_buffer(16)
    lib().oracle_gf128_mul(_ptr(xb), _ptr(yb), _ptr(zb))
    return zb.raw


def gf_pow(h: bytes, e: int) -> bytes:
    """h^e by square-and-multiply over the oracle's multiplication (h^0 = 1)."""
    if e < 0:
        raise ValueError("negative exponent")
    result, base = ONE, h
    while e:
        if e & 1:
            result = gf_mul(result, base)
        base = gf_mul(base, base)
        e >>= 1
    return result


def xor16(a: bytes, b: bytes) -> bytes:
    return bytes(p ^ q for p, q in zip(a, b))


def ghash(h: bytes, x: bytes) -> bytes:
    """Serial GHASH_H over whole 16-byte blocks (Algorithm 2 / the paper's Eq. 1)."""
    if len(x) % 16:
        raise ValueError("GHASH input must be whole blocks")
    xb, hb, ob = _buf(x), _buf(h), ctypes.create_string_buffer(16)
    lib().oracle_ghash(_ptr(hb), _ptr(xb), len(x) // 16, _ptr(ob))
    return ob.raw


def chunk_partial(h: bytes, blocks: Sequence[bytes]) -> bytes:
    """Horner over one chunk: sum_j X_j * H^(m-j+1), j = 1..m (the map phase
    of the paper's two-phase GHASH, Sec. 5.2.2, with the trailing factor H
    kept inside each partial)."""
    y = ZERO
    for blk in blocks:
        y = gf_mul(xor16(y, blk), h)
    return y


def combine(h: bytes, left: bytes, right: bytes, right_blocks: int) -> bytes:
    """Combine(L, R) = L * H^(#blocks of R) xor R: joins the partials of two
    adjacent segments (the paper's tree step, Fig. 3b, where the power of H
    jumps the gap left by the right-hand segment)."""
    return xor16(gf_mul(left, gf_pow(h, right_blocks)), right)


def tree_ghash(h: bytes, x: bytes, cuts: Iterable[int]) -> bytes:
    """GHASH computed the parallel way: split the block sequence at ``cuts``
    (block indices), Horner inside each chunk, then a balanced pairwise tree
    of ``combine`` steps over the chunk partials (Sec. 3.3.1, Fig. 3b)."""
    n = len(x) // 16
    blocks = [x[16 * i: 16 * i + 16] for i in range(n)]
    edges = [0] + sorted(set(c for c in cuts if 0 < c < n)) + [n]
    level: List[Tuple[bytes, int]] = [
        (chunk_partial(h, blocks[a:b]), b - a) for a, b in zip(edges[:-1], edges[1:])
    ]
    if not level:
        return ZERO
    while len(level) > 1:
        nxt = []
        for i in range(0, len(level) - 1, 2):
            (lp, ln), (rp, rn) = level[i], level[i + 1]
            nxt.append((combine(h, lp, rp, rn), ln + rn))
        if len(level) % 2:
            nxt.append(level[-1])
        level = nxt
    return level[0][0]


def tree_ghash_fig2b(h: bytes, x: bytes) -> bytes:
    """The exact shape drawn in Fig. 3b for a power-of-two block count:
    partials omit the trailing H, level k joins pairs with H^(2^k), and one
    final multiplication by H closes the tree."""
    n = len(x) // 16
    if n == 0:
        return ZERO
    if n & (n - 1):
        raise ValueError("Fig. 3b shape needs a power-of-two block count")
    level = [x[16 * i: 16 * i + 16] for i in range(n)]
    k = 0
    while len(level) > 1:
        stride = gf_pow(h, 1 << k)
        level = [xor16(gf_mul(level[i], stride), level[i + 1]) for i in range(0, len(level), 2)]
        k += 1
    return gf_mul(level[0], h)


# --------------------------------------------------------------------------
# GCM (SP 800-38D Algorithms 3-5)
# --------------------------------------------------------------------------

def inc32(block: bytes) -> bytes:
    b = _buf(block)
    lib().oracle_inc32(_ptr(b))  # b stays referenced until the call returns
    return b.raw[:16]


def h_j0(key: bytes, iv: bytes) -> Tuple[bytes, bytes, bytes]:
    """(H, J0, E_K(J0)) for a key and IV."""
    hb, jb, eb = (ctypes.create_string_buffer(16) for _ in range(3))
    kb, ib = _buf(key), _buf(iv)
    rc = lib().oracle_gcm_h_j0(_ptr(kb), len(key), _ptr(ib), len(iv), _ptr(hb), _ptr(jb), _ptr(eb))
    if rc != 0:
        raise ValueError("bad key or IV length")
    return hb.raw, jb.raw, eb.raw


def keystream_block(key: bytes, j0: bytes, i: int) -> bytes:
    """CIPH_K(inc_32^i(J0)): the keystream XORed into data block i (1-based)."""
    ob = ctypes.create_string_buffer(16)
    kb, jb = _buf(key), _buf(j0)
    lib().oracle_keystream_block(_ptr(kb), len(key), _ptr(jb), i, _ptr(ob))
    return ob.raw


def gcm_encrypt(key: bytes, iv: bytes, aad: bytes, pt: bytes) -> Tuple[bytes, bytes]:
    kb, ib, ab, pb = _buf(key), _buf(iv), _buf(aad), _buf(pt)
    cb, tb = ctypes.create_string_buffer(max(1, len(pt))), ctypes.create_string_buffer(16)
    rc = lib().oracle_gcm_encrypt(_ptr(kb), len(key), _ptr(ib), len(iv), _ptr(ab), len(aad),
                                  _ptr(pb), len(pt), _ptr(cb), _ptr(tb))
    if rc != 0:
        raise ValueError("bad key or IV length")
    return cb.raw[: len(pt)], tb.raw


def gcm_decrypt(key: bytes, iv: bytes, aad: bytes, ct: bytes, tag: bytes) -> Tuple[bool, bytes]:
    """Returns (ok, plaintext); on failure the plaintext is all zero bytes."""
    kb, ib, ab, cb, tb = _buf(key), _buf(iv), _buf(aad), _buf(ct), _buf(tag)
    pb = ctypes.create_string_buffer(b"\xa5" * max(1, len(ct)), max(1, len(ct)))
    rc = lib().oracle_gcm_decrypt(_ptr(kb), len(key), _ptr(ib), len(iv), _ptr(ab), len(aad),
                                  _ptr(cb), len(ct), _ptr(tb), _ptr(pb))
    if rc < 0:
        raise ValueError("bad key or IV length")
    return rc == 0, pb.raw[: len(ct)]


def counter_block(j0: bytes, i: int) -> bytes:
    """inc_32^i(J0): the rightmost 32 bits of J0, read big-endian, plus i
    modulo 2^32; the leftmost 96 bits unchanged (SP 800-38D sec. 6.2 applied
    i times).  Block j (0-based) of a payload is XORed with
    CIPH_K(counter_block(J0, j + 1))."""
    lo = (int.from_bytes(j0[12:16], "big") + i) & 0xFFFFFFFF
    return bytes(j0[:12]) + lo.to_bytes(4, "big")


def gctr_ptr(key: bytes, icb: bytes, src: int, n: int, dst: int) -> None:
    """GCTR_K(ICB, X) (Algorithm 3) from ``n`` bytes at address ``src`` into
    ``dst`` (host addresses, e.g. numpy ``.ctypes.data``)."""
    w, nr = key_expansion(key)
    wb, ib = _buf(w), _buf(icb)
    lib().oracle_gctr(_ptr(wb), nr, _ptr(ib), src, n, dst)


def ghash_ptr(h: bytes, src: int, nblocks: int) -> bytes:
    """Serial GHASH_H (Algorithm 2) over ``nblocks`` whole blocks at host
    address ``src``."""
    hb, ob = _buf(h), ctypes.create_string_buffer(16)
    lib().oracle_ghash(_ptr(hb), src, nblocks, _ptr(ob))
    return ob.raw


def gcm_encrypt_numpy(key: bytes, iv: bytes, aad: bytes, pt_array) -> Tuple["object", bytes]:
    """Oracle encryption of a numpy uint8 array without extra copies."""
    import numpy as np

    pt_array = np.ascontiguousarray(pt_array, dtype=np.uint8)
    ct = np.empty_like(pt_array)
    kb, ib, ab = _buf(key), _buf(iv), _buf(aad)
    tb = ctypes.create_string_buffer(16)
    n = pt_array.size
    dummy = np.zeros(1, np.uint8)
    pp = (pt_array if n else dummy).ctypes.data
    cp = (ct if n else dummy).ctypes.data
    rc = lib().oracle_gcm_encrypt(_ptr(kb), len(key), _ptr(ib), len(iv), _ptr(ab), len(aad),
                                  pp, n, cp, _ptr(tb))
    if rc != 0:
        raise ValueError("bad key or IV length")
    return ct, tb.raw


# --------------------------------------------------------------------------
# FITS framing (FITS standard: 2880-byte records, 80-character cards)
# --------------------------------------------------------------------------

FITS_RECORD = 2880
FITS_CARD = 80


def _card_value(card: bytes) -> Optional[str]:
    if len(card) < 10 or card[8:10] != b"= ":
        return None
    v = card[10:].decode("ascii")
    if "/" in v:
        v = v.split("/", 1)[0]
    return v.strip()


def datasum(data: bytes) -> int:
    """FITS DATASUM: 32-bit ones' complement sum of big-endian words with
    end-around carry (C oracle, word by word)."""
    b = _buf(bytes(data))
    return int(lib().oracle_datasum(_ptr(b), len(data)))


def datasum_ptr(src: int, n: int) -> int:
    """``datasum`` of ``n`` bytes at host address ``src``."""
    return int(lib().oracle_datasum(src, n))


def fits_split(fits: bytes) -> Tuple[bytes, bytes, int]:
    """Split a single-HDU FITS image into (header, padded data unit, data bytes).

    The header is every 2880-byte record up to and including the one that
    holds the END card.  The data unit holds |BITPIX|/8 * prod(NAXISn) bytes
    and is returned padded to whole 2880-byte records: with the file's own
    padding bytes when the file holds them, else with zero bytes."""
    end = None
    for rec in range(0, len(fits) // FITS_RECORD):
        for c in range(FITS_RECORD // FITS_CARD):
            off = rec * FITS_RECORD + c * FITS_CARD
            if fits[off: off + 8] == b"END     ":
                end = (rec + 1) * FITS_RECORD
                break
        if end is not None:
            break
    if end is None:
        raise ValueError("no END card")
    header = fits[:end]
    keys = {}
    for c in range(0, end, FITS_CARD):
        card = header[c: c + FITS_CARD]
        name = card[:8].decode("ascii").strip()
        val = _card_value(card)
        if val is not None and name not in keys:
            keys[name] = val
    bitpix = int(keys["BITPIX"])
    naxis = int(keys["NAXIS"])
    nbytes = abs(bitpix) // 8 if naxis > 0 else 0
    for i in range(1, naxis + 1):
        nbytes *= int(keys["NAXIS%d" % i])
    full = nbytes + (-nbytes) % FITS_RECORD
    if len(fits) >= end + full:
        # the file carries the whole record-padded data unit (zero fill for a
        # plain FITS file, ciphertext for an encrypted one)
        return header, fits[end: end + full], nbytes
    data = fits[end: end + nbytes]
    if len(data) != nbytes:
        raise ValueError("truncated data unit")
    return header, data + bytes(full - nbytes), nbytes


def fits_encrypt(key: bytes, iv: bytes, fits: bytes) -> Tuple[bytes, bytes]:
    """Encrypt a FITS file the way the data path does: header in clear and
    authenticated as AAD, padded data unit encrypted.  Returns (file, tag)."""
    header, padded, _ = fits_split(fits)
    ct, tag = gcm_encrypt(key, iv, header, padded)
    return header + ct, tag


def fits_decrypt(key: bytes, iv: bytes, enc: bytes, tag: bytes) -> Tuple[bool, bytes]:
    header, padded, _ = fits_split(enc)
    ok, pt = gcm_decrypt(key, iv, header, padded, tag)
    return ok, header + pt


def serialize_int(v: int) -> bytes:
    """Strict ASCII decimal (Sec. 3.2.3: the integer -32 becomes b'-32')."""
    return str(int(v)).encode("ascii")


def paper_aad_data(nonce: bytes, bitpix: int, naxes: Sequence[int]) -> bytes:
    """AAD_Data = NONCE_D || Serialize(ORIG_BITPIX) || Serialize(ORIG_NAXIS)
    || Serialize(ORIG_NAXIS1) || ... (Sec. 3.2.3), concatenated with no
    separators, exactly as printed."""
    out = bytes(nonce) + serialize_int(bitpix) + serialize_int(len(naxes))
    for n in naxes:
        out += serialize_int(n)
    return out
