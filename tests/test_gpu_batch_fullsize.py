"""Parity of the batched form at its full size, in the launch configuration
the benchmark times: one gcm_batch call over the 10,000-message mix
(lognormal lengths, median 2 MiB, sigma 1.0, 16 B..64 MiB, ~30% not
multiples of 16, AES-128/AES-256 with distinct keys, 5% IVs of 8..128
bytes, AAD 0..4 KiB; 33.8 GB of payload in device memory).

The oracle cannot encrypt all 33.8 GB in test time, so it checks whole
messages chosen across the length range, and single blocks:
  * the first 120 messages of at most 256 KiB: ciphertext and tag equal the
    oracle's, byte for byte;
  * the 12 longest messages (up to 64 MiB, many tiles each) and 36 random
    messages above 256 KiB, whole: ciphertext (SHA-256 of 8 MiB chunks) and
    tag equal those of the oracle run chunk by chunk on all host cores
    (``oracle.mapreduce``);
  * sampled blocks of the 12 longest (both ends, tile edges, random) equal
    P_j xor E_K(inc32^(j+1)(J0)) from single oracle keystream blocks;
  * decrypt-verify of the whole batch, in place, accepts every message and
    gives back every plaintext.
"""
import ctypes
import random

import numpy as np
import pytest

import oracle
from oracle import mapreduce
from paper_2602_23067_gb300 import workloads

pytestmark = pytest.mark.gpu

COUNT = 10000


def test_ten_thousand_messages_in_one_launch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_23067_gb300 import Context, _native

    descs = workloads.message_mix(3, COUNT, median=2 << 20, sigma=1.0, lo=16, hi=64 << 20, frac_unaligned=0.3,
                                  frac_long_iv=0.05, aad_max=4096, key_sizes=(16, 32))
    lens = [d["len"] for d in descs]
    slot = [(n + 255) // 256 * 256 for n in lens]
    offs = np.concatenate([[0], np.cumsum(slot)]).astype(np.int64)
    total = int(offs[-1])
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < 2 * total + (8 << 30):
        pytest.skip("needs %.0f GB of free device memory" % ((2 * total + (8 << 30)) / 1e9))
    assert sum(lens) > 33e9

    g = torch.Generator(device="cuda")
    g.manual_seed(33)
    arena_in = torch.empty(total, dtype=torch.uint8, device="cuda")
    for o in range(0, total, 1 << 30):
        n = min(1 << 30, total - o)
        arena_in[o:o + n].copy_(torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda", generator=g))
    for i in range(COUNT):  # slot gaps hold zeros on both sides
        if slot[i] > lens[i]:
            arena_in[int(offs[i]) + lens[i]: int(offs[i]) + slot[i]].zero_()
    arena_out = torch.zeros_like(arena_in)
    aad_sizes = [d["aad_len"] for d in descs]
    aoffs = np.concatenate([[0], np.cumsum(aad_sizes)]).astype(np.int64)
    aad_arena = torch.randint(0, 256, (max(1, int(aoffs[-1])),), dtype=torch.uint8, device="cuda", generator=g)
    tags = torch.zeros(COUNT * 16, dtype=torch.uint8, device="cuda")
    keep = []

    def msgs(src, dst):
        arr = (_native.GcmMsg * COUNT)()
        for i, d in enumerate(descs):
            kb = ctypes.create_string_buffer(d["key"], len(d["key"]))
            ib = ctypes.create_string_buffer(d["iv"], len(d["iv"]))
            keep.extend([kb, ib])
            arr[i] = _native.GcmMsg(ctypes.addressof(kb), len(d["key"]), ctypes.addressof(ib), len(d["iv"]),
                                    aad_arena.data_ptr() + int(aoffs[i]) if aad_sizes[i] else None, aad_sizes[i],
                                    src.data_ptr() + int(offs[i]), dst.data_ptr() + int(offs[i]), lens[i],
                                    tags.data_ptr() + 16 * i)
        return arr

    status = (ctypes.c_int32 * COUNT)()
    with Context(0) as ctx:
        stream = torch.cuda.current_stream()
        rc = _native.lib.gcm_batch(ctx.handle, msgs(arena_in, arena_out), COUNT, 0, status, 0, stream.cuda_stream)
        assert rc == 0, _native.last_error()
        torch.cuda.synchronize()
        host_tags = tags.cpu().numpy().reshape(COUNT, 16)

        def host(t, i, n):
            return bytes(t[int(offs[i]): int(offs[i]) + n].cpu().numpy())

        def aad_of(i):
            return bytes(aad_arena[int(aoffs[i]): int(aoffs[i]) + aad_sizes[i]].cpu().numpy()) if aad_sizes[i] else b""

        # short messages against the oracle, whole
        short = [i for i in range(COUNT) if lens[i] <= (256 << 10)][:120]
        assert len(short) == 120 and any(len(descs[i]["iv"]) != 12 for i in short)
        for i in short:
            d = descs[i]
            ref_ct, ref_tag = oracle.gcm_encrypt(d["key"], d["iv"], aad_of(i), host(arena_in, i, lens[i]))
            assert host(arena_out, i, lens[i]) == ref_ct, i
            assert bytes(host_tags[i]) == ref_tag, i

        # the 12 longest messages and 36 random ones of 256 KiB..64 MiB, whole:
        # ciphertext digests and tags against the chunked oracle on all host
        # cores (GCTR from each chunk's counter, serial GHASH per chunk,
        # partials joined by Combine, length block, E_K(J0))
        longest = sorted(range(COUNT), key=lambda i: -lens[i])[:12]
        r = random.Random(34)
        mid = [i for i in range(COUNT) if (256 << 10) < lens[i] and i not in longest]
        whole = longest + r.sample(mid, 36)
        total_whole = sum(lens[i] for i in whole)
        chunk = 8 << 20
        with mapreduce.HostInput(total_whole) as src:
            spec, o = [], 0
            for i in whole:
                torch.from_numpy(src.array[o:o + lens[i]]).copy_(arena_in[int(offs[i]): int(offs[i]) + lens[i]])
                spec.append({"key": descs[i]["key"], "iv": descs[i]["iv"], "aad": aad_of(i), "off": o,
                             "len": lens[i]})
                o += lens[i]
            ref = mapreduce.gcm_encrypt_digests(spec, src, chunk_bytes=chunk)
        for i, (ref_dg, ref_tag) in zip(whole, ref):
            assert bytes(host_tags[i]) == ref_tag, i
            got = arena_out[int(offs[i]): int(offs[i]) + lens[i]].cpu().numpy()
            assert mapreduce.digests(got, chunk) == ref_dg, i

        # sampled blocks of the longest messages against single oracle
        # keystream blocks (both ends, tile edges, random)
        for i in longest:
            d = descs[i]
            n = lens[i]
            nb = (n + 15) // 16
            a_blocks = (aad_sizes[i] + 15) // 16
            m = a_blocks + nb
            idx = {0, 1, nb - 2, nb - 1}
            for k in range(1, 6):
                for e in (-1, 0, 1):
                    j = m - k * (1 << 16) + e - a_blocks
                    if 0 <= j < nb:
                        idx.add(j)
            while len(idx) < 60:
                idx.add(r.randrange(nb))
            _, j0, _ = oracle.h_j0(d["key"], d["iv"])
            base = int(offs[i])
            for j in sorted(idx):
                w = min(16, n - 16 * j)
                p = bytes(arena_in[base + 16 * j: base + 16 * j + w].cpu().numpy())
                c = bytes(arena_out[base + 16 * j: base + 16 * j + w].cpu().numpy())
                ks = oracle.keystream_block(d["key"], j0, j + 1)[:w]
                assert c == bytes(x ^ y for x, y in zip(p, ks)), (i, j)

        # the whole batch back, in place
        rc = _native.lib.gcm_batch(ctx.handle, msgs(arena_out, arena_out), COUNT, 1, status, 0, stream.cuda_stream)
        assert rc == 0, _native.last_error()
        torch.cuda.synchronize()
        assert not any(status[i] for i in range(COUNT))
        assert torch.equal(arena_out, arena_in)
    del arena_in, arena_out, aad_arena, tags
    torch.cuda.empty_cache()
