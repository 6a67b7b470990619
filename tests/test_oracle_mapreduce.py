"""Pins for the chunked oracle (``oracle/mapreduce.py``), no GPU.

The chunked form is what the full-size GPU parity tests compare against, so
it is pinned here to the serial definition (``oracle.gcm_encrypt``, itself
pinned to pyca/cryptography and to the field identities in
``test_oracle_pins.py``): for every cut of small messages into chunks, the
per-chunk ciphertext digests and the tag must equal those of the serial
encryption.  A wrong chunk counter (inc32^b instead of inc32^(b+1)), a
dropped AAD or length block, a combine with the wrong power of H or a
partial block hashed without its zero pad each fail one of these cases.
"""
import ctypes
import hashlib
import random

import numpy as np
import pytest

import oracle
from oracle import mapreduce


def rnd(r, n):
    return bytes(r.getrandbits(8) for _ in range(n))


def serial_digests(ct, chunk):
    return [hashlib.sha256(ct[a:b]).digest() for a, b in mapreduce.chunk_bounds(len(ct), chunk)]


def run(msgs, chunk, workers=1):
    total = sum(len(m["pt"]) for m in msgs)
    with mapreduce.HostInput(total) as src:
        off = 0
        spec = []
        for m in msgs:
            n = len(m["pt"])
            src.array[off:off + n] = np.frombuffer(m["pt"], dtype=np.uint8)
            spec.append({"key": m["key"], "iv": m["iv"], "aad": m["aad"], "off": off, "len": n})
            off += n
        return mapreduce.gcm_encrypt_digests(spec, src, chunk_bytes=chunk, workers=workers)


def test_counter_block_is_repeated_inc32_across_a_wrap():
    r = random.Random(41)
    for low in (0, 1, 0xFFFFFFF0, 0xFFFFFFFF):
        j0 = rnd(r, 12) + low.to_bytes(4, "big")
        cb = j0
        for i in range(40):
            assert oracle.counter_block(j0, i) == cb
            cb = oracle.inc32(cb)


def test_chunked_equals_serial_for_every_cut():
    r = random.Random(42)
    cases = []
    for n in (0, 1, 15, 16, 17, 100, 1000, 4097):
        for kl, ivl, al in ((16, 12, 0), (24, 1, 20), (32, 60, 33)):
            cases.append({"key": rnd(r, kl), "iv": rnd(r, ivl), "aad": rnd(r, al), "pt": rnd(r, n)})
    for chunk in (16, 32, 48, 160, 4096, 1 << 20):
        got = run(cases, chunk)
        for m, (dg, tag) in zip(cases, got):
            ct, ref_tag = oracle.gcm_encrypt(m["key"], m["iv"], m["aad"], m["pt"])
            assert tag == ref_tag, (len(m["pt"]), chunk)
            assert dg == serial_digests(ct, chunk), (len(m["pt"]), chunk)


def test_chunked_equals_serial_across_a_counter_wrap_in_worker_processes():
    # A non-96-bit IV whose J0 low word lies within 2^14 of 2^32, so the
    # 32-bit counter wraps inside a message of 2^14 + 50 blocks, at a chunk
    # boundary or inside a chunk depending on the cut.
    r = random.Random(43)
    key = rnd(r, 16)
    h, _, _ = oracle.h_j0(key, bytes(12))
    hb = ctypes.create_string_buffer(h, 16)
    out = ctypes.create_string_buffer(16)
    for _ in range(1 << 22):
        iv = rnd(r, 16)
        ivb = ctypes.create_string_buffer(iv, 16)
        oracle.lib().oracle_j0(ctypes.addressof(hb), ctypes.addressof(ivb), 16, ctypes.addressof(out))
        if int.from_bytes(out.raw[12:16], "big") >= (1 << 32) - (1 << 14):
            break
    else:
        pytest.fail("no IV found")
    m = {"key": key, "iv": iv, "aad": b"hdr", "pt": rnd(r, 16 * ((1 << 14) + 50) - 3)}
    ct, ref_tag = oracle.gcm_encrypt(m["key"], m["iv"], m["aad"], m["pt"])
    for chunk in (4096, 16 * 997):
        (dg, tag), = run([m], chunk, workers=3)
        assert tag == ref_tag
        assert dg == serial_digests(ct, chunk)


def test_digests_helper_cuts_like_the_oracle():
    data = bytes(range(256)) * 3 + b"x"
    assert mapreduce.digests(data, 160) == serial_digests(data, 160)
    with pytest.raises(ValueError):
        mapreduce.chunk_bounds(100, 24)


def test_planted_mistakes_are_detected(monkeypatch):
    # The comparison above would catch a chunk counter that is one block off
    # and a combine that skips one power of H.
    r = random.Random(44)
    m = {"key": rnd(r, 16), "iv": rnd(r, 12), "aad": rnd(r, 5), "pt": rnd(r, 200)}
    ct, ref_tag = oracle.gcm_encrypt(m["key"], m["iv"], m["aad"], m["pt"])
    good = oracle.counter_block
    monkeypatch.setattr(oracle, "counter_block", lambda j0, i: good(j0, i - 1))
    (dg, tag), = run([m], 64)
    assert dg[1:] != serial_digests(ct, 64)[1:]
    monkeypatch.setattr(oracle, "counter_block", good)
    comb = oracle.combine
    monkeypatch.setattr(oracle, "combine", lambda h, a, b, n: comb(h, a, b, max(0, n - 1)))
    (dg, tag), = run([m], 64)
    assert dg == serial_digests(ct, 64) and tag != ref_tag


def test_ciphertext_written_to_an_output_file():
    r = random.Random(45)
    msgs = [{"key": rnd(r, 32), "iv": rnd(r, 12), "aad": rnd(r, 9), "pt": rnd(r, n)} for n in (0, 33, 5000, 160)]
    total = sum(len(m["pt"]) for m in msgs)
    with mapreduce.HostInput(total) as src, mapreduce.HostInput(total) as dst:
        spec, off = [], 0
        for m in msgs:
            src.array[off:off + len(m["pt"])] = np.frombuffer(m["pt"], dtype=np.uint8)
            spec.append({"key": m["key"], "iv": m["iv"], "aad": m["aad"], "off": off, "len": len(m["pt"])})
            off += len(m["pt"])
        got = mapreduce.gcm_encrypt_digests(spec, src, chunk_bytes=64, workers=2, dest=dst)
        for m, s_, (dg, tag) in zip(msgs, spec, got):
            ct, ref_tag = oracle.gcm_encrypt(m["key"], m["iv"], m["aad"], m["pt"])
            assert tag == ref_tag
            assert bytes(dst.array[s_["off"]: s_["off"] + s_["len"]]) == ct
