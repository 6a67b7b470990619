"""The library used from C alone: tests/abi_consumer.c (built against
include/gcmgpu.h and linked to libgcmgpu.so) encrypts a deterministic
message in host memory, decrypt-verifies it, checks that a tampered tag is
refused with the output zero-filled, and writes its ciphertext and tag;
both must equal the oracle's for the same inputs."""
import os
import subprocess

import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [0, 5, 4096, 1000003])
def test_c_program_matches_the_oracle(tmp_path, n):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_23067_gb300 import build

    build.build()
    from test_abi import build_c_consumer

    exe = build_c_consumer(str(tmp_path))
    out = os.path.join(str(tmp_path), "ct.bin")
    r = subprocess.run([exe, str(n), out], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    key = bytes((11 * i + 1) & 0xFF for i in range(32))
    iv = bytes(0xA0 + i for i in range(12))
    aad = bytes(3 * i for i in range(20))
    pt = bytes((7 * i + 3) & 0xFF for i in range(n))
    ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, aad, pt)
    with open(out, "rb") as f:
        assert f.read() == ref_ct
    assert r.stdout.strip() == ref_tag.hex()
