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


@pytest.mark.parametrize("tile_log2", [10, 12])
def test_segment_start_offsets(torch_cuda, tile_log2):
    # Whole-payload segments are walked in 32-block windows from the segment
    # start; a lane takes the AES round-1/2 constants of its own 256-counter
    # group and refreshes them when its counter enters a new group, so a
    # window that straddles a group boundary refreshes only some lanes.
    # AAD of 0..31 blocks moves every segment's first counter through all
    # residues mod 32, and non-96-bit IVs (J0 from GHASH(IV)) start the
    # counter word anywhere mod 256 (and let it wrap mod 2^32).
    from paper_2602_23067_gb300 import Context

    torch = torch_cuda
    r = random.Random(9600 + tile_log2)
    n = 3 * (16 << tile_log2) + 37
    with Context(0) as ctx:
        ctx.set_tile_log2(tile_log2)
        for k in range(32):
            a = 0 if k == 0 else 16 * k - (k % 7)
            key = bytes(r.getrandbits(8) for _ in range(16 if k % 2 else 32))
            iv = bytes(r.getrandbits(8) for _ in range(12 if k % 4 < 2 else 8 + 13 * (k % 5)))
            aad = bytes(r.getrandbits(8) for _ in range(a))
            pt = workloads.random_bytes(9600 + 64 * tile_log2 + k, n).tobytes()
            ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, aad, pt)
            d_aad = dev(torch, aad) if aad else None
            ct, tag = ctx.encrypt_device(key, iv, d_aad, dev(torch, pt))
            torch.cuda.synchronize()
            assert bytes(tag.cpu().numpy()) == ref_tag, (k, len(iv))
            assert bytes(ct.cpu().numpy()) == ref_ct, (k, len(iv))
            back = ctx.decrypt_verify_device(key, iv, d_aad, ct, tag)
            assert bytes(back.cpu().numpy()) == pt, (k, len(iv))
