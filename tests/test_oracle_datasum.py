"""Pins of the oracle's FITS DATASUM (32-bit ones' complement sum with
end-around carry, the FITS checksum convention the paper's container uses
through cfitsio, Sec. 3.2.2)."""
import random

import oracle


def words(*ws):
    return b"".join(w.to_bytes(4, "big") for w in ws)


def test_special_values():
    assert oracle.datasum(b"") == 0
    assert oracle.datasum(bytes(2880)) == 0  # all-zero data: +0
    assert oracle.datasum(words(0x12345678)) == 0x12345678
    assert oracle.datasum(words(0xFFFFFFFF, 1)) == 1  # carry out of bit 31 wraps to bit 0
    assert oracle.datasum(words(0x80000000, 0x80000000)) == 1
    assert oracle.datasum(words(0xFFFFFFFF)) == 0xFFFFFFFF
    assert oracle.datasum(words(0xFFFFFFFE, 1)) == 0xFFFFFFFF  # -0: a nonzero multiple of 2^32 - 1
    assert oracle.datasum(b"\x01") == 0x01000000  # partial word zero-padded on the right


def test_closed_form_and_byte_order():
    # a nonzero total is congruent to the sum mod 2^32 - 1, with 2^32 - 1
    # standing for 0; the words are big-endian
    r = random.Random(31)
    for n in (4, 8, 64, 2880, 11520, 4 * 1000 + 3):
        data = bytes(r.getrandbits(8) for _ in range(n))
        padded = data + bytes(-len(data) % 4)
        total = sum(int.from_bytes(padded[i:i + 4], "big") for i in range(0, len(padded), 4))
        expect = 0 if total == 0 else (total - 1) % 0xFFFFFFFF + 1
        assert oracle.datasum(data) == expect
    assert oracle.datasum(words(0x01020304)) != oracle.datasum(bytes([4, 3, 2, 1]))


def test_complement_closes_the_sum():
    # the FITS CHECKSUM principle: adding the complement of the sum gives -0
    r = random.Random(32)
    for _ in range(20):
        data = bytes(r.getrandbits(8) for _ in range(4 * r.randrange(1, 500)))
        s = oracle.datasum(data)
        assert oracle.datasum(data + words(~s & 0xFFFFFFFF)) == 0xFFFFFFFF


def test_split_invariance():
    # ones' complement addition is associative: sums of word-aligned parts add up
    r = random.Random(33)
    data = bytes(r.getrandbits(8) for _ in range(4 * 3000))
    for cut in (4, 400, 4 * 1234, 4 * 2999):
        a, b = oracle.datasum(data[:cut]), oracle.datasum(data[cut:])
        assert oracle.datasum(words(a, b)) == oracle.datasum(data)
