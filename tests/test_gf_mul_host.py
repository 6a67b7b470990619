"""The library's general GF(2^128) multiplier (carry-less integer products,
two Karatsuba levels, reduction by x^128 + x^7 + x^2 + x + 1), compiled for
the host from the same header the kernels use, against the oracle's
shift-and-add multiply (SP 800-38D Algorithm 1) on special and random
operands.  No GPU needed."""
import os
import random
import shutil
import subprocess

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2602_23067_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("gf") / "gf_mul_host")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "gf_mul_host.cu"), "-o", exe],
                   check=True, capture_output=True)
    return exe


def run(exe, pairs):
    inp = "".join("%s %s\n" % (a.hex(), b.hex()) for a, b in pairs)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
    return [bytes.fromhex(x) for x in out]


def test_special_operands(harness):
    one = bytes([0x80]) + bytes(15)  # x^0
    top = bytes(15) + bytes([0x01])  # x^127
    ones = bytes([0xFF]) * 16
    zero = bytes(16)
    vals = [zero, one, top, ones, bytes([0x40]) + bytes(15), bytes(15) + bytes([0x02]),
            bytes([0xE1]) + bytes(15), bytes(8) + bytes([0x80]) + bytes(7)]
    pairs = [(a, b) for a in vals for b in vals]
    got = run(harness, pairs)
    for (a, b), g in zip(pairs, got):
        assert g == oracle.gf_mul(a, b), (a.hex(), b.hex())


def test_random_operands(harness):
    r = random.Random(77)
    pairs = []
    for _ in range(3000):
        a = bytes(r.getrandbits(8) for _ in range(16))
        b = bytes(r.getrandbits(8) for _ in range(16))
        # sparse and dense bit patterns exercise the per-class counts
        if r.random() < 0.2:
            a = bytes(x | 0xEE for x in a)
        if r.random() < 0.2:
            b = bytes(x & 0x11 for x in b)
        pairs.append((a, b))
    got = run(harness, pairs)
    bad = [(a.hex(), b.hex()) for (a, b), g in zip(pairs, got) if g != oracle.gf_mul(a, b)]
    assert not bad, bad[:3]
