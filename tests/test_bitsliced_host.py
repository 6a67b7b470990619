"""The bitsliced AES of the GPU path (the generated S-box circuit, bitsliced
ShiftRows / MixColumns / AddRoundKey and the 32 x 32 bit transposes that
load counters and unload keystream), compiled for the host from the same
headers the kernel uses, against the oracle's FIPS-197 cipher on counter
blocks.  No GPU needed."""
import os
import random
import shutil
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2602_23067_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("bs") / "aes_bitsliced_host")
    subprocess.run([nvcc, "-O1", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "aes_bitsliced_host.cu"),
                    "-o", exe], check=True, capture_output=True)
    return exe


def run(exe, cases):
    lines = []
    for key, j0, ctrs in cases:
        w, nr = oracle.key_expansion(key)
        lines.append("%d %s %s %s" % (nr, w.hex(), j0.hex(), " ".join(str(c) for c in ctrs)))
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.split()
    return [bytes.fromhex(x) for x in out]


def expected(key, j0, ctrs):
    return [oracle.aes_encrypt_block(key, j0 + c.to_bytes(4, "big")) for c in ctrs]


@pytest.mark.parametrize("key_len", [16, 24, 32])
def test_counter_blocks_match_the_cipher(harness, key_len):
    r = random.Random(key_len)
    cases = []
    for n in range(6):
        key = bytes(r.getrandbits(8) for _ in range(key_len))
        j0 = bytes(r.getrandbits(8) for _ in range(12))
        base = r.getrandbits(32)
        if n == 0:
            ctrs = [(base + k) & 0xFFFFFFFF for k in range(32)]  # consecutive
        elif n == 1:
            ctrs = [(0xFFFFFFF0 + k) & 0xFFFFFFFF for k in range(32)]  # inc32 wrap inside the group
        elif n == 2:
            ctrs = [(base + 5 + 32 * k) & 0xFFFFFFFF for k in range(32)]  # one lane's stride-32 chain
        else:
            ctrs = [r.getrandbits(32) for _ in range(32)]
        cases.append((key, j0, ctrs))
    got = run(harness, cases)
    want = [b for key, j0, ctrs in cases for b in expected(key, j0, ctrs)]
    assert len(got) == len(want)
    bad = [i for i, (g, w) in enumerate(zip(got, want)) if g != w]
    assert not bad, (bad[:4], got[bad[0]].hex(), want[bad[0]].hex())


def test_generated_circuit_is_current(tmp_path):
    """The committed header is what the generator writes (and the generator
    checks its circuit against the S-box on all 256 inputs)."""
    out = tmp_path / "sbox.cuh"
    subprocess.run([sys.executable, os.path.join(CSRC, "gen_bitsliced_sbox.py"), str(out)], check=True,
                   capture_output=True)
    with open(os.path.join(CSRC, "bitsliced_sbox.cuh")) as f:
        assert f.read() == out.read_text()
