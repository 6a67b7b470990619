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
