"""Tile size and the autotuner: every tile size 2^9..2^16 blocks gives the
oracle's ciphertext and tag (the tree combine is an exact regrouping, so the
split must not matter), and the autotuned table keeps results exact."""
import random

import pytest

import oracle
from paper_2602_23067_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def dev(torch, b):
    t = torch.empty(max(1, len(b)), dtype=torch.uint8, device="cuda")
    if b:
        t[: len(b)].copy_(torch.frombuffer(bytearray(b), dtype=torch.uint8))
    return t[: len(b)]


@pytest.mark.parametrize("tile_log2", list(range(9, 17)))
def test_every_tile_size_is_exact(torch_cuda, tile_log2):
    from paper_2602_23067_gb300 import Context

    torch = torch_cuda
    r = random.Random(9400 + tile_log2)
    with Context(0) as ctx:
        ctx.set_tile_log2(tile_log2)
        for n, a in ((3 * (1 << 20) + 7, 2880), (16 * 1000 + 3, 17), (1 << 16, 0)):
            key, iv, aad = bytes(r.getrandbits(8) for _ in range(32)), bytes(r.getrandbits(8) for _ in range(12)), \
                bytes(r.getrandbits(8) for _ in range(a))
            pt = workloads.random_bytes(9400 + n, n).tobytes()
            ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, aad, pt)
            ct, tag = ctx.encrypt_device(key, iv, dev(torch, aad) if aad else None, dev(torch, pt))
            torch.cuda.synchronize()
            assert bytes(tag.cpu().numpy()) == ref_tag and bytes(ct.cpu().numpy()) == ref_ct
            back = ctx.decrypt_verify_device(key, iv, dev(torch, aad) if aad else None, ct, tag)
            assert bytes(back.cpu().numpy()) == pt


def test_autotune_table_and_parity(torch_cuda):
    from paper_2602_23067_gb300 import Context

    torch = torch_cuda
    with Context(0) as ctx:
        table = ctx.autotune(key_len=16, max_bytes=4 << 20)
        assert len(table) == 64
        assert all(t == 0 or 9 <= t <= 16 for t in table)
        assert table[((16 << 10) // 16).bit_length() - 1] != 0  # the smallest measured size's class is tuned
        r = random.Random(9500)
        for n in (1000, 300000, 5 << 20):
            key, iv = bytes(r.getrandbits(8) for _ in range(16)), bytes(r.getrandbits(8) for _ in range(12))
            pt = workloads.random_bytes(9500 + n, n).tobytes()
            ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, b"", pt)
            ct, tag = ctx.encrypt_device(key, iv, None, dev(torch, pt))
            torch.cuda.synchronize()
            assert bytes(tag.cpu().numpy()) == ref_tag and bytes(ct.cpu().numpy()) == ref_ct
        ctx.set_tuning(table)
        ctx.set_tuning(None)
