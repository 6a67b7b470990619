"""Messages finished inside the fused launch (the last CTA runs the reduce
of the tile partials, the length block, the tag and the verify gate)
against the oracle, and the boundary to the separate combine kernel.

A message of 1..1024 tiles and at most 2^22 blocks is finished by the last
CTA to take a ticket; the ticket word (one per stream) wraps back to zero
on the last ticket, so consecutive launches of any grid size on one stream
must all finish correctly.  Every result here is compared with the oracle.
"""
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


def rnd(r, n):
    return bytes(r.getrandbits(8) for _ in range(n))


def dev(torch, b):
    t = torch.empty(len(b), dtype=torch.uint8, device="cuda")
    if b:
        t.copy_(torch.frombuffer(bytearray(b), dtype=torch.uint8))
    return t


def host(t):
    return bytes(t.cpu().numpy().tobytes())


def launches(ctx):
    from paper_2602_23067_gb300 import _native

    return _native.gcm_profile_read(ctx.handle, reset=True)["launches"]


def test_one_launch_per_call_with_a_cached_key(torch_cuda):
    torch = torch_cuda
    from paper_2602_23067_gb300 import Context, _native

    r = random.Random(61)
    key, iv, aad = rnd(r, 16), rnd(r, 12), rnd(r, 20)
    pt = workloads.random_bytes(61, 1 << 20).tobytes()
    ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, aad, pt)
    with Context(0) as ctx:
        a, p = dev(torch, aad), dev(torch, pt)
        ctx.encrypt_device(key, iv, a, p)  # sets the key up (cached afterwards)
        torch.cuda.synchronize()
        _native.gcm_profile_enable(ctx.handle, True)
        launches(ctx)
        ct, tag = ctx.encrypt_device(key, iv, a, p)
        torch.cuda.synchronize()
        assert launches(ctx) == 1  # the fused launch alone
        assert host(tag) == ref_tag and host(ct) == ref_ct
        back = ctx.decrypt_verify_device(key, iv, a, ct, tag)
        torch.cuda.synchronize()
        assert launches(ctx) == 1
        assert host(back) == pt


def test_grid_sizes_in_a_row_on_one_stream_and_two_streams(torch_cuda):
    # Grids of 1, 2, 17, 65, 152 CTAs (tiles of 2^9..2^16 blocks, K up to
    # 1024), alternating, on the current stream and on a second stream.
    torch = torch_cuda
    from paper_2602_23067_gb300 import Context

    r = random.Random(62)
    sizes = [16, 4000, 17 * 8192 - 5, 65 * 16384, (1 << 20) + 48, 1024 * 512 * 16 - 2880, 33, 152 * 8192 * 16]
    cases = []
    for k, n in enumerate(sizes):
        kl = (16, 24, 32)[k % 3]
        cases.append((rnd(r, kl), rnd(r, 12 if k % 2 == 0 else 40), rnd(r, 2880 if k == 5 else 13), rnd(r, n)))
    refs = [oracle.gcm_encrypt(*c) for c in cases]
    with Context(0) as ctx:
        side = torch.cuda.Stream()
        for rep in range(3):
            outs = []
            for k, (key, iv, aad, pt) in enumerate(cases):
                st = side if (rep == 2 and k % 2) else torch.cuda.current_stream()
                with torch.cuda.stream(st):
                    a, p = dev(torch, aad), dev(torch, pt)
                    ct, tag = ctx.encrypt_device(key, iv, a, p, stream=st)
                    outs.append((st, ct, tag))
            torch.cuda.synchronize()
            for (st, ct, tag), (ref_ct, ref_tag) in zip(outs, refs):
                assert host(tag) == ref_tag
                assert host(ct) == ref_ct


def test_tamper_on_the_finish_path_zero_fills_a_ragged_payload(torch_cuda):
    torch = torch_cuda
    from paper_2602_23067_gb300 import Context, GcmError

    r = random.Random(63)
    key, iv, aad = rnd(r, 32), rnd(r, 12), rnd(r, 5)
    pt = rnd(r, 300001)  # 18751 blocks, the last one partial: several tiles
    ct, tag = oracle.gcm_encrypt(key, iv, aad, pt)
    with Context(0) as ctx:
        for flip in ("tag", "ct", "aad"):
            t, c, a = bytearray(tag), bytearray(ct), bytearray(aad)
            {"tag": t, "ct": c, "aad": a}[flip][3] ^= 0x10
            out = torch.full((len(ct),), 0xA5, dtype=torch.uint8, device="cuda")
            with pytest.raises(GcmError):
                ctx.decrypt_verify_device(key, iv, dev(torch, bytes(a)), dev(torch, bytes(c)), dev(torch, bytes(t)),
                                          pt=out)
            torch.cuda.synchronize()
            assert int(out.to(torch.int32).sum().item()) == 0, flip
        back = ctx.decrypt_verify_device(key, iv, dev(torch, aad), dev(torch, ct), dev(torch, tag))
        torch.cuda.synchronize()
        assert host(back) == pt


def test_both_sides_of_the_finish_boundary(torch_cuda):
    # Tiles forced to 2^9 blocks: 1024 tiles are finished in the fused
    # launch, 1025 go through the combine kernel; also GHASH alone on both
    # sides, and one non-96-bit IV (E_K(J0) read from the per-message setup).
    torch = torch_cuda
    from paper_2602_23067_gb300 import Context, _native

    r = random.Random(64)
    with Context(0) as ctx:
        ctx.set_tile_log2(9)
        _native.gcm_profile_enable(ctx.handle, True)
        for tiles, ivl in ((1024, 12), (1025, 12), (1024, 16), (1025, 16)):
            key, iv, aad = rnd(r, 16), rnd(r, ivl), rnd(r, 32)
            n = 16 * (tiles * 512 - 2) - 7  # AAD: 2 blocks; last payload block partial
            pt = rnd(r, n)
            ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, aad, pt)
            a, p = dev(torch, aad), dev(torch, pt)
            ctx.encrypt_device(key, iv, a, p)
            torch.cuda.synchronize()
            launches(ctx)
            ct, tag = ctx.encrypt_device(key, iv, a, p)
            torch.cuda.synchronize()
            got = launches(ctx)
            assert host(tag) == ref_tag and host(ct) == ref_ct, (tiles, ivl)
            fused_only = 1 if tiles <= 1024 else 2
            assert got == fused_only + (0 if ivl == 12 else 1), (tiles, ivl, got)
            h, _, _ = oracle.h_j0(key, iv)
            blob = aad + bytes((-len(aad)) % 16) + ref_ct + bytes((-len(ref_ct)) % 16)
            blob += (8 * len(aad)).to_bytes(8, "big") + (8 * len(ref_ct)).to_bytes(8, "big")
            gh = ctx.ghash_device(key, a, ct)
            torch.cuda.synchronize()
            assert host(gh) == oracle.ghash(h, blob), tiles


def test_streams_destroyed_with_work_in_flight_and_per_thread_streams(torch_cuda):
    # Stream handles can be reused once a stream is destroyed, even while its
    # work still runs; the per-thread default stream is one handle for one
    # stream per thread.  Calls on both kinds must finish correctly.
    import threading

    torch = torch_cuda
    from paper_2602_23067_gb300 import Context

    r = random.Random(65)
    cases = [(rnd(r, 16), rnd(r, 12), rnd(r, 20), rnd(r, 4096 * (3 + k % 5) + k)) for k in range(24)]
    refs = [oracle.gcm_encrypt(*c) for c in cases]
    with Context(0) as ctx:
        outs = []
        for k, (key, iv, aad, pt) in enumerate(cases[:12]):
            st = torch.cuda.Stream()  # released (destroyed) when dropped below
            a, p = dev(torch, aad), dev(torch, pt)
            torch.cuda.synchronize()
            ct, tag = ctx.encrypt_device(key, iv, a, p, stream=st)
            outs.append((ct, tag, a, p))
            del st
        torch.cuda.synchronize()
        for (ct, tag, _, _), (ref_ct, ref_tag) in zip(outs, refs[:12]):
            assert host(tag) == ref_tag and host(ct) == ref_ct

        per_thread = 2  # cudaStreamPerThread
        res = {}

        def worker(tid):
            for k in range(tid, 12, 2):
                key, iv, aad, pt = cases[12 + k]
                a, p = dev(torch, aad), dev(torch, pt)
                torch.cuda.synchronize()
                ct, tag = ctx.encrypt_device(key, iv, a, p, stream=per_thread)
                res[12 + k] = (ct, tag)

        th = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        torch.cuda.synchronize()
        for k in range(12, 24):
            ct, tag = res[k]
            assert host(tag) == refs[k][1] and host(ct) == refs[k][0], k


def test_block_limit_of_the_finish_and_a_64_mib_zero_fill(torch_cuda):
    # Tiles forced to 2^13 blocks: a sequence of exactly 2^22 blocks (512
    # tiles, 64 MiB) is finished inside the fused launch -- including, for a
    # tampered tag, the zero-fill of the whole payload by the finishing CTA --
    # while 2^22 + 16 blocks go through the combine and zero-fill kernels.
    # The oracle runs chunk by chunk on the host cores.
    torch = torch_cuda
    from oracle import mapreduce
    from paper_2602_23067_gb300 import Context, GcmError, _native

    r = random.Random(66)
    with Context(0) as ctx:
        ctx.set_tile_log2(13)
        _native.gcm_profile_enable(ctx.handle, True)
        for extra, enc_launches, dec_launches in ((0, 1, 1), (16, 2, 3)):
            key, iv, aad = rnd(r, 32), rnd(r, 12), rnd(r, 32)
            n = 16 * ((1 << 22) - 2 + extra) - 3  # AAD: 2 blocks; last payload block partial
            g = torch.Generator(device="cuda")
            g.manual_seed(66 + extra)
            pt = torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda", generator=g)
            with mapreduce.HostInput(n) as src, mapreduce.HostInput(n) as dst:
                torch.from_numpy(src.array).copy_(pt)
                (ref_dg, ref_tag), = mapreduce.gcm_encrypt_digests(
                    [{"key": key, "iv": iv, "aad": aad, "off": 0, "len": n}], src, chunk_bytes=4 << 20, dest=dst)
                ref_ct = torch.from_numpy(dst.array.copy()).cuda()
            a = dev(torch, aad)
            ctx.encrypt_device(key, iv, a, pt)  # key setup (cached afterwards)
            torch.cuda.synchronize()
            launches(ctx)
            ct, tag = ctx.encrypt_device(key, iv, a, pt)
            torch.cuda.synchronize()
            assert launches(ctx) == enc_launches, extra
            assert host(tag) == ref_tag, extra
            assert torch.equal(ct, ref_ct), extra
            bad = bytearray(ref_tag)
            bad[0] ^= 0x01
            out = torch.full((n,), 0x5A, dtype=torch.uint8, device="cuda")
            with pytest.raises(GcmError):
                ctx.decrypt_verify_device(key, iv, a, ref_ct, dev(torch, bytes(bad)), pt=out)
            torch.cuda.synchronize()
            assert launches(ctx) == dec_launches, extra
            assert int(torch.count_nonzero(out).item()) == 0, extra
            back = ctx.decrypt_verify_device(key, iv, a, ref_ct, dev(torch, ref_tag), pt=out)
            torch.cuda.synchronize()
            assert torch.equal(back, pt), extra
            del pt, ct, ref_ct, out
