"""gcm_batch: many independent messages in one persistent launch (device
memory) or streamed through device chunk buffers (host memory).  Every
message is checked byte for byte against the oracle, and each result must
be the same alone and in the mix (tolerance: exact)."""
import random

import numpy as np
import pytest

import oracle
from paper_2602_23067_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_23067_gb300 import Context

    ctx = Context(0)
    yield torch, ctx
    ctx.close()


def make_mix(seed, count, median, sigma, hi, long_iv=0.2):
    """Message descriptors from the seeded mix generator, payloads materialised."""
    descs = workloads.message_mix(seed, count, median=median, sigma=sigma, lo=1, hi=hi, frac_unaligned=0.4,
                                  frac_long_iv=long_iv, aad_max=300, key_sizes=(16, 24, 32))
    r = random.Random(seed)
    out = []
    for d in descs:
        n = d["len"] if r.random() > 0.05 else 0  # a few empty payloads
        out.append({
            "key": d["key"], "iv": d["iv"],
            "aad": workloads.random_bytes(d["seed"] + 1, d["aad_len"]).tobytes(),
            "pt": workloads.random_bytes(d["seed"], n).tobytes(),
        })
    return out


def dev(torch, b):
    t = torch.empty(max(1, len(b)), dtype=torch.uint8, device="cuda")
    if b:
        t[: len(b)].copy_(torch.frombuffer(bytearray(b), dtype=torch.uint8))
    return t


def test_batch_device_matches_oracle_and_single_calls(env):
    torch, ctx = env
    msgs = make_mix(31, 60, median=20000, sigma=1.5, hi=3 << 20)
    # include a message that spans many 2^16-block tiles
    msgs.append({"key": bytes(range(32)), "iv": bytes(range(12)), "aad": b"hdr" * 7,
                 "pt": workloads.random_bytes(77, (1 << 20) * 5 + 3).tobytes()})
    dm = []
    for m in msgs:
        dm.append({"key": m["key"], "iv": m["iv"], "aad": dev(torch, m["aad"]) if m["aad"] else None,
                   "inp": dev(torch, m["pt"]), "out": torch.empty(max(1, len(m["pt"])), dtype=torch.uint8,
                                                                  device="cuda"),
                   "tag": torch.empty(16, dtype=torch.uint8, device="cuda"), "len": len(m["pt"])})
    for d, m in zip(dm, msgs):
        if d["aad"] is not None:
            d["aad"] = d["aad"][: len(m["aad"])]
    st = ctx.batch(dm)
    torch.cuda.synchronize()
    assert st == [0] * len(msgs)
    for d, m in zip(dm, msgs):
        ref_ct, ref_tag = oracle.gcm_encrypt(m["key"], m["iv"], m["aad"], m["pt"])
        assert bytes(d["tag"].cpu().numpy()) == ref_tag
        assert bytes(d["out"][: len(m["pt"])].cpu().numpy()) == ref_ct
    # alone (single-message entry point) == in the mix
    for d, m in list(zip(dm, msgs))[:8]:
        ct, tag = ctx.encrypt_device(m["key"], m["iv"], d["aad"], d["inp"][: len(m["pt"])] if m["pt"] else
                                     d["inp"][:0])
        torch.cuda.synchronize()
        assert bytes(tag.cpu().numpy()) == bytes(d["tag"].cpu().numpy())


def test_batch_device_decrypt_rejects_only_the_tampered(env):
    torch, ctx = env
    msgs = make_mix(32, 40, median=8000, sigma=1.0, hi=1 << 20, long_iv=0.1)
    enc = [oracle.gcm_encrypt(m["key"], m["iv"], m["aad"], m["pt"]) for m in msgs]
    bad = {3, 17, 29}
    dm = []
    for i, (m, (ct, tag)) in enumerate(zip(msgs, enc)):
        t = bytearray(tag)
        if i in bad:
            t[i % 16] ^= 1 << (i % 8)
        dm.append({"key": m["key"], "iv": m["iv"],
                   "aad": dev(torch, m["aad"])[: len(m["aad"])] if m["aad"] else None,
                   "inp": dev(torch, ct), "out": torch.full((max(1, len(ct)),), 0x5A, dtype=torch.uint8,
                                                            device="cuda"),
                   "tag": dev(torch, bytes(t)), "len": len(ct)})
    st = ctx.batch(dm, decrypt=True)
    torch.cuda.synchronize()
    for i, (d, m) in enumerate(zip(dm, msgs)):
        got = bytes(d["out"][: len(m["pt"])].cpu().numpy())
        if i in bad:
            assert st[i] == -3
            assert got == bytes(len(m["pt"]))
        else:
            assert st[i] == 0
            assert got == m["pt"]


@pytest.mark.parametrize("host_access", [2, 0])
def test_batch_host_streaming_small_chunks(env, host_access):
    """host_access 2: staged through a ring of 3 device chunk buffers of
    64 KiB (many chunks per message); 0: the kernels work on the host
    buffers directly when the device can reach host memory."""
    torch, ctx = env
    from paper_2602_23067_gb300 import Context

    c2 = Context(0)
    try:
        c2.set_host_access(host_access)
        c2.set_streaming(64 * 1024, 3)
        msgs = make_mix(33, 25, median=150000, sigma=1.0, hi=2 << 20)
        hm = []
        for m in msgs:
            hm.append({"key": m["key"], "iv": m["iv"], "aad": m["aad"],
                       "inp": np.frombuffer(m["pt"], dtype=np.uint8).copy(),
                       "out": np.empty(max(1, len(m["pt"])), dtype=np.uint8),
                       "tag": np.empty(16, dtype=np.uint8), "len": len(m["pt"])})
        st = c2.batch(hm)
        assert st == [0] * len(msgs)
        for h, m in zip(hm, msgs):
            ref_ct, ref_tag = oracle.gcm_encrypt(m["key"], m["iv"], m["aad"], m["pt"])
            assert h["tag"].tobytes() == ref_tag
            assert h["out"][: len(m["pt"])].tobytes() == ref_ct
        # decrypt back, with one tampered tag
        for i, (h, m) in enumerate(zip(hm, msgs)):
            h["inp"], h["out"] = h["out"][: max(1, len(m["pt"]))].copy(), np.zeros(max(1, len(m["pt"])), np.uint8)
            if i == 5:
                h["tag"] = h["tag"].copy()
                h["tag"][0] ^= 1
        st = c2.batch(hm, decrypt=True)
        for i, (h, m) in enumerate(zip(hm, msgs)):
            if i == 5:
                assert st[i] == -3 and h["out"][: len(m["pt"])].tobytes() == bytes(len(m["pt"]))
            else:
                assert st[i] == 0 and h["out"][: len(m["pt"])].tobytes() == m["pt"]
    finally:
        c2.close()


@pytest.mark.parametrize("host_access", [2, 0])
def test_host_mode_single_message_many_chunks(env, host_access):
    torch, ctx = env
    from paper_2602_23067_gb300 import Context

    c2 = Context(0)
    try:
        c2.set_host_access(host_access)
        c2.set_streaming(128 * 1024, 2)
        key, iv = bytes(range(16)), bytes(range(12))
        aad = workloads.random_bytes(5, 3000).tobytes()
        pt = workloads.random_bytes(6, 3 * (1 << 20) + 11).tobytes()
        ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, aad, pt)
        ct, tag = c2.encrypt_host(key, iv, aad, np.frombuffer(pt, np.uint8).copy())
        assert tag == ref_tag and ct.tobytes() == ref_ct
        back = c2.decrypt_verify_host(key, iv, aad, ct, tag)
        assert back.tobytes() == pt
    finally:
        c2.close()


@pytest.mark.parametrize("lg", [9, 10, 11, 12, 13, 14, 15, 16])
def test_batch_at_every_tile_size(env, lg):
    """A batch's tiles are 2^lg blocks for all its messages (by default the
    largest size that gives every SM four tiles of the batch; forced here):
    encryption and decrypt-verify (one tampered tag) against the oracle at
    every size, with a message spanning 2..129 tiles."""
    torch, ctx = env
    msgs = make_mix(33 + lg, 12, median=30000, sigma=1.5, hi=600000)
    msgs.append({"key": bytes(range(16)), "iv": bytes(range(12)), "aad": b"a" * 50,
                 "pt": workloads.random_bytes(90 + lg, (1 << 20) + 9).tobytes()})
    enc = [oracle.gcm_encrypt(m["key"], m["iv"], m["aad"], m["pt"]) for m in msgs]
    dm = []
    for m in msgs:
        dm.append({"key": m["key"], "iv": m["iv"], "aad": dev(torch, m["aad"])[: len(m["aad"])] if m["aad"] else None,
                   "inp": dev(torch, m["pt"]), "out": torch.empty(max(1, len(m["pt"])), dtype=torch.uint8,
                                                                  device="cuda"),
                   "tag": torch.empty(16, dtype=torch.uint8, device="cuda"), "len": len(m["pt"])})
    ctx.set_tile_log2(lg)
    try:
        assert ctx.batch(dm) == [0] * len(msgs)
        torch.cuda.synchronize()
        for d, m, (ref_ct, ref_tag) in zip(dm, msgs, enc):
            assert bytes(d["tag"].cpu().numpy()) == ref_tag
            assert bytes(d["out"][: len(m["pt"])].cpu().numpy()) == ref_ct
        bad = len(msgs) - 1
        back = []
        for i, (d, m) in enumerate(zip(dm, msgs)):
            t = bytearray(enc[i][1])
            if i == bad:
                t[3] ^= 4
            back.append({"key": m["key"], "iv": m["iv"], "aad": d["aad"], "inp": d["out"],
                         "out": torch.full((max(1, len(m["pt"])),), 0x5A, dtype=torch.uint8, device="cuda"),
                         "tag": dev(torch, bytes(t)), "len": len(m["pt"])})
        st = ctx.batch(back, decrypt=True)
        torch.cuda.synchronize()
    finally:
        ctx.set_tile_log2(0)
    for i, (b, m) in enumerate(zip(back, msgs)):
        got = bytes(b["out"][: len(m["pt"])].cpu().numpy())
        if i == bad:
            assert st[i] == -3
            assert got == bytes(len(m["pt"]))
        else:
            assert st[i] == 0
            assert got == m["pt"]


def _wrap_iv(key, nblocks, r):
    """A 16-byte IV whose J0 has a low word within nblocks - 100 of 2^32, so
    that inc32 wraps inside a message of nblocks blocks (searched with the
    oracle's J0)."""
    import ctypes

    h, _, _ = oracle.h_j0(key, bytes(12))
    hb = ctypes.create_string_buffer(h, 16)
    out = ctypes.create_string_buffer(16)
    for _ in range(1 << 24):
        iv = bytes(r.randrange(256) for _ in range(16))
        ivb = ctypes.create_string_buffer(iv, 16)
        oracle.lib().oracle_j0(ctypes.addressof(hb), ctypes.addressof(ivb), 16, ctypes.addressof(out))
        if int.from_bytes(out.raw[12:16], "big") >= (1 << 32) - nblocks + 100:
            return iv
    raise AssertionError("no wrapping IV found")


@pytest.mark.parametrize("lg", [0, 16])
def test_batch_with_one_byte_iv_and_counter_wrap(env, lg):
    """Batch members on the GHASH(IV) path: a 1-byte IV (outside what other
    libraries accept) and a 16-byte IV whose counter wraps mod 2^32 inside
    the message, among ordinary ones; encrypt (gcm_batch and a batch plan)
    and decrypt-verify against the oracle, at the batch's own tile size and
    at 2^16-block tiles."""
    torch, ctx = env
    r = random.Random(6000 + lg)
    wrap_key = bytes(r.randrange(256) for _ in range(32))
    nwrap = 1 << 16
    msgs = [
        {"key": bytes(r.randrange(256) for _ in range(16)), "iv": bytes([r.randrange(256)]), "aad": b"x" * 21,
         "pt": workloads.random_bytes(6001, 50007).tobytes()},
        {"key": wrap_key, "iv": _wrap_iv(wrap_key, nwrap, r), "aad": b"", "pt": workloads.random_bytes(
            6002, 16 * nwrap - 3).tobytes()},
    ] + make_mix(6003, 4, median=20000, sigma=1.0, hi=200000)
    enc = [oracle.gcm_encrypt(m["key"], m["iv"], m["aad"], m["pt"]) for m in msgs]

    def dmsgs(src, dst, tags):
        return [{"key": m["key"], "iv": m["iv"], "aad": dev(torch, m["aad"])[: len(m["aad"])] if m["aad"] else None,
                 "inp": s, "out": d, "tag": t, "len": len(m["pt"])} for m, s, d, t in zip(msgs, src, dst, tags)]

    src = [dev(torch, m["pt"]) for m in msgs]
    outs = [torch.empty(max(1, len(m["pt"])), dtype=torch.uint8, device="cuda") for m in msgs]
    tags = [torch.empty(16, dtype=torch.uint8, device="cuda") for _ in msgs]
    ctx.set_tile_log2(lg)
    try:
        assert ctx.batch(dmsgs(src, outs, tags)) == [0] * len(msgs)
        torch.cuda.synchronize()
        for m, o, t, (ref_ct, ref_tag) in zip(msgs, outs, tags, enc):
            assert bytes(t.cpu().numpy()) == ref_tag
            assert bytes(o[: len(m["pt"])].cpu().numpy()) == ref_ct
        outs2 = [torch.zeros_like(o) for o in outs]
        tags2 = [torch.zeros_like(t) for t in tags]
        with ctx.batch_plan(dmsgs(src, outs2, tags2)) as plan:
            assert plan.run() == [0] * len(msgs)
        for m, o, t, (ref_ct, ref_tag) in zip(msgs, outs2, tags2, enc):
            assert bytes(t.cpu().numpy()) == ref_tag
            assert bytes(o[: len(m["pt"])].cpu().numpy()) == ref_ct
        back = [torch.zeros_like(o) for o in outs]
        assert ctx.batch(dmsgs(outs, back, tags), decrypt=True) == [0] * len(msgs)
        torch.cuda.synchronize()
    finally:
        ctx.set_tile_log2(0)
    for m, b in zip(msgs, back):
        assert bytes(b[: len(m["pt"])].cpu().numpy()) == m["pt"]
