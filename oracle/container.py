"""The paper's dual-key authenticated FITS container (Sec. 3.2.2, Fig.
"Structure of the Authenticated FITS Format"; access behaviour Sec. 4.2,
Table "Role-based and temporal access control policies") -- test
infrastructure only, like the rest of this package.

Layout (the paper fixes the contents; the encodings below are this library's
readings where the paper is silent):

* HDU 0, metadata only (NAXIS = 0): NONCE_H, NONCE_D (12-byte nonces, as
  24 lowercase hex characters), AUTHTAG_H and AUTHTAG_D stored as AUTHTG_H
  and AUTHTG_D (16-byte tags, 32 hex characters; the paper's names have nine
  characters, one more than a FITS keyword holds), ORIG_BPX, ORIG_NAX, ORIG_NA1, ORIG_NA2, ... (the original
  BITPIX, NAXIS, NAXISn under the abbreviated names of the paper's footnote)
  and ENCHDR: the original header records (through the END record) encrypted
  with the header key under NONCE_H and no AAD, as lowercase hex in a long
  string of 64 characters per card (FITS CONTINUE convention).
* HDU 1, a one-row binary table with one column of N bytes (TFORM1 = 'NB',
  TTYPE1 = 'ENCDATA'): the original pixel bytes (the data unit without its
  record padding, N = |BITPIX|/8 * prod NAXISn) encrypted with the data key
  under NONCE_D with AAD_D = NONCE_D || Serialize(ORIG_BITPIX) ||
  Serialize(ORIG_NAXIS) || Serialize(ORIG_NAXIS1) || ... (Sec. 3.2.3).
* Both HDUs end with DATASUM and CHECKSUM cards (Sec. 3.2.2: the container
  carries the FITS-standard CHECKSUM/DATASUM keywords in both HDUs): DATASUM
  is the 32-bit ones' complement sum of the data unit ('0' for the primary,
  which has none) and CHECKSUM the 16-character encoding, defined by the FITS
  checksum convention the paper cites, of the complement of the HDU's sum,
  so that the whole HDU then sums to -0 (0xFFFFFFFF).

Decryption (the paper's gfc_decrypt_frame): the header is the authenticated
ENCHDR when the header key is given and its tag verifies, else a minimal
header rebuilt from the ORIG_* keywords (header fallback, warning 1); the
pixels are decrypted when the data key is given and AUTHTAG_D verifies,
else zero-filled (payload suppression, warning 2, which takes precedence).
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence, Tuple

from . import datasum, fits_split, gcm_decrypt, gcm_encrypt, paper_aad_data

RECORD = 2880
CARD = 80
HEX_PER_CARD = 64


def _pad_card(text: str) -> bytes:
    if len(text) > CARD:
        raise ValueError("card longer than 80 characters: %r" % text)
    return text.ljust(CARD).encode("ascii")


def card_int(key: str, v: int) -> bytes:
    """Fixed-format integer: keyword, '= ', value right-justified to column 30."""
    return _pad_card("%-8s= %20d" % (key, v))


def card_logical(key: str, v: bool) -> bytes:
    return _pad_card("%-8s= %20s" % (key, "T" if v else "F"))


def card_str(key: str, s: str) -> bytes:
    """Fixed-format string: opening quote in column 11, at least 8 characters
    between the quotes (blank-padded)."""
    return _pad_card("%-8s= '%s'" % (key, s.ljust(8)))


def cards_long_str(key: str, s: str) -> List[bytes]:
    """A long string value over CONTINUE cards, 64 characters per card, each
    card but the last ending its part with '&'."""
    parts = [s[i: i + HEX_PER_CARD] for i in range(0, len(s), HEX_PER_CARD)] or [""]
    out = []
    for i, p in enumerate(parts):
        amp = "&" if i + 1 < len(parts) else ""
        if i == 0:
            out.append(_pad_card("%-8s= '%s%s'" % (key, p, amp)))
        else:
            out.append(_pad_card("CONTINUE  '%s%s'" % (p, amp)))
    return out


def header_block(cards: Sequence[bytes]) -> bytes:
    """Cards, the END card, blank fill to whole 2880-byte records."""
    h = b"".join(cards) + _pad_card("END")
    return h + b" " * ((-len(h)) % RECORD)


def ones_add(a: int, b: int) -> int:
    """Ones' complement sum of two 32-bit ones' complement sums."""
    s = a + b
    while s >> 32:
        s = (s & 0xFFFFFFFF) + (s >> 32)
    return s


_PUNCT = set(range(0x3A, 0x41)) | set(range(0x5B, 0x61))


def checksum_chars(value: int) -> str:
    """The 16 ASCII characters that stand for a 32-bit value in a CHECKSUM
    card.  Byte i of the value (i = 0 most significant) becomes four
    characters whose codes add up to the byte plus 4 * 0x30: all equal to
    0x30 + byte // 4, the first raised by byte % 4.  Characters that would be
    punctuation (0x3A..0x40, 0x5B..0x60) are avoided by moving one unit from
    the second to the first character of a pair ((0,1) and (2,3)), which
    keeps the pair's sum, until neither is punctuation.  The four characters
    of byte i go to positions i, i+4, i+8, i+12, so in 4-byte words each
    byte lane adds up to the value's byte plus 4 * 0x30; the string is then
    rotated right by one, because a card value starts at column 12, one byte
    before a word boundary of the header."""
    out = [0] * 16
    for i in range(4):
        byte = (value >> (24 - 8 * i)) & 0xFF
        c = [0x30 + byte // 4] * 4
        c[0] += byte % 4
        for j in (0, 2):
            while c[j] in _PUNCT or c[j + 1] in _PUNCT:
                c[j] += 1
                c[j + 1] -= 1
        for j in range(4):
            out[4 * j + i] = c[j]
    rotated = out[15:] + out[:15]
    return bytes(rotated).decode("ascii")


def header_with_checksum(cards: Sequence[bytes], data_sum: int, data_sum_text: str) -> bytes:
    """The header block of cards + DATASUM + CHECKSUM, the CHECKSUM value
    chosen so that header and data together sum to -0."""
    zero = "0" * 16
    h = header_block(list(cards) + [card_str("DATASUM", data_sum_text), card_str("CHECKSUM", zero)])
    total = ones_add(datasum(h), data_sum)
    at = h.index(("CHECKSUM= '%s'" % zero).encode("ascii")) + 11
    enc = checksum_chars(~total & 0xFFFFFFFF).encode("ascii")
    return h[:at] + enc + h[at + 16:]


def parse_header(buf: bytes, off: int = 0) -> Tuple[Dict[str, str], int]:
    """Keyword -> raw value text (strings without quotes; long strings joined
    over CONTINUE cards), and the offset just past the header's last record."""
    keys: Dict[str, str] = {}
    last = None
    pos = off
    while True:
        if pos + CARD > len(buf):
            raise ValueError("no END card")
        card = buf[pos: pos + CARD].decode("ascii")
        pos += CARD
        name = card[:8].strip()
        if name == "END":
            break
        if name == "CONTINUE" and last is not None:
            v = card[10:].strip()
            assert v.startswith("'") and v.endswith("'")
            keys[last] = keys[last][:-1] + v[1:-1] if keys[last].endswith("&") else keys[last]
            continue
        if card[8:10] != "= ":
            last = None
            continue
        v = card[10:].strip()
        if v.startswith("'"):
            v = v[1: v.rindex("'")].rstrip()
        else:
            v = v.split("/", 1)[0].strip()  # drop the comment
        keys[name] = v
        last = name
    pos = off + ((pos - off + RECORD - 1) // RECORD) * RECORD
    return keys, pos


def _structure(header: bytes) -> Tuple[int, List[int]]:
    keys, _ = parse_header(header)
    bitpix = int(keys["BITPIX"])
    naxis = int(keys["NAXIS"])
    return bitpix, [int(keys["NAXIS%d" % i]) for i in range(1, naxis + 1)]


def container_encrypt(key_h: bytes, key_d: bytes, nonce_h: bytes, nonce_d: bytes, fits: bytes) -> bytes:
    """The two-HDU container of a single-HDU FITS image."""
    header, padded, nbytes = fits_split(fits)
    pixels = padded[:nbytes]
    bitpix, naxes = _structure(header)
    enchdr, tag_h = gcm_encrypt(key_h, nonce_h, b"", header)
    blob, tag_d = gcm_encrypt(key_d, nonce_d, paper_aad_data(nonce_d, bitpix, naxes), pixels)
    cards = [card_logical("SIMPLE", True), card_int("BITPIX", 8), card_int("NAXIS", 0),
             card_logical("EXTEND", True),
             card_str("NONCE_H", nonce_h.hex()), card_str("NONCE_D", nonce_d.hex()),
             card_str("AUTHTG_H", tag_h.hex()), card_str("AUTHTG_D", tag_d.hex()),
             card_int("ORIG_BPX", bitpix), card_int("ORIG_NAX", len(naxes))]
    cards += [card_int("ORIG_NA%d" % (i + 1), n) for i, n in enumerate(naxes)]
    cards += cards_long_str("ENCHDR", enchdr.hex())
    primary = header_with_checksum(cards, 0, "0")
    dsum = datasum(blob)
    ext = header_with_checksum([card_str("XTENSION", "BINTABLE"), card_int("BITPIX", 8), card_int("NAXIS", 2),
                                card_int("NAXIS1", len(blob)), card_int("NAXIS2", 1), card_int("PCOUNT", 0),
                                card_int("GCOUNT", 1), card_int("TFIELDS", 1), card_str("TTYPE1", "ENCDATA"),
                                card_str("TFORM1", "%dB" % len(blob))], dsum, str(dsum))
    return primary + ext + blob + bytes((-len(blob)) % RECORD)


def minimal_header(bitpix: int, naxes: Sequence[int]) -> bytes:
    """The header fallback: a structurally valid header from ORIG_* alone."""
    cards = [card_logical("SIMPLE", True), card_int("BITPIX", bitpix), card_int("NAXIS", len(naxes))]
    cards += [card_int("NAXIS%d" % (i + 1), n) for i, n in enumerate(naxes)]
    return header_block(cards)


def decrypt_frame(container: bytes, key_h: Optional[bytes], key_d: Optional[bytes]) -> Tuple[bytes, int]:
    """(FITS file, warning_code): 0 full access, 1 header fallback, 2 payload
    suppressed."""
    p, off = parse_header(container, 0)
    x, data_off = parse_header(container, off)
    n = int(x["NAXIS1"])
    blob = container[data_off: data_off + n]
    nonce_h, nonce_d = bytes.fromhex(p["NONCE_H"]), bytes.fromhex(p["NONCE_D"])
    tag_h, tag_d = bytes.fromhex(p["AUTHTG_H"]), bytes.fromhex(p["AUTHTG_D"])
    bitpix, naxis = int(p["ORIG_BPX"]), int(p["ORIG_NAX"])
    naxes = [int(p["ORIG_NA%d" % i]) for i in range(1, naxis + 1)]
    header = None
    if key_h is not None:
        ok, h = gcm_decrypt(key_h, nonce_h, b"", bytes.fromhex(p["ENCHDR"]), tag_h)
        header = h if ok else None
    warning = 0
    if header is None:
        header = minimal_header(bitpix, naxes)
        warning = 1
    pixels = bytes(n)
    data_ok = False
    if key_d is not None:
        data_ok, pixels = gcm_decrypt(key_d, nonce_d, paper_aad_data(nonce_d, bitpix, naxes), blob, tag_d)
    if not data_ok:
        pixels = bytes(n)
        warning = 2
    return header + pixels + bytes((-n) % RECORD), warning
