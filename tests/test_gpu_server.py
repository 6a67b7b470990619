"""The continuous-batching server: mixed encrypt / decrypt-verify requests on
several cached keys, some arriving while others are on the GPU; each result
must equal the oracle's (i.e. be the same alone and in the mix), and
tampered tags must be rejected with zero-filled output."""
import random
import time

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


def _requests(seed, count, keys):
    r = random.Random(seed)
    reqs = []
    for i in range(count):
        kidx = r.randrange(len(keys))
        key = keys[kidx]
        iv = bytes(r.getrandbits(8) for _ in range(12 if r.random() < 0.8 else r.randrange(8, 70)))
        aad = bytes(r.getrandbits(8) for _ in range(r.choice((0, 20, 2880))))
        n = r.choice((0, 1, 15, 16, 2880, 5000, 70000, 200003))
        pt = workloads.random_bytes(seed * 1000 + i, n).tobytes()
        op = r.randrange(2)
        ct, tag = oracle.gcm_encrypt(key, iv, aad, pt)
        bad = op == 1 and r.random() < 0.15
        if bad:
            tag = bytes([tag[0] ^ 0x01]) + tag[1:]
        reqs.append({"k": kidx, "key": key, "iv": iv, "aad": aad, "pt": pt, "ct": ct, "tag": tag, "op": op, "bad": bad})
    return reqs


def _run(ctx, reqs, handles, max_wave, max_inflight, spread_s=0.0):
    srv = ctx.server(hbm_budget_bytes=1 << 30, max_wave_msgs=max_wave, max_inflight=max_inflight)
    outs = {}
    try:
        pending = {}
        for i, q in enumerate(reqs):
            src = q["pt"] if q["op"] == 0 else q["ct"]
            inp = np.frombuffer(src, dtype=np.uint8).copy() if src else np.zeros(1, np.uint8)
            out = np.full(max(1, len(src)), 0xA5, dtype=np.uint8)
            tag = np.frombuffer(q["tag"], dtype=np.uint8).copy() if q["op"] == 1 else np.zeros(16, np.uint8)
            t = srv.submit(q["op"], handles[q["k"]], q["iv"], q["aad"] or None, inp[: len(src)] if src else inp[:0],
                           out, tag, user=i)
            pending[t] = (i, out, tag)
            if spread_s:
                time.sleep(spread_s)
        deadline = time.time() + 120
        while pending and time.time() < deadline:
            for ticket, status, arr, done, user in srv.poll():
                i, out, tag = pending.pop(ticket)
                outs[i] = (status, out, tag)
            time.sleep(0.001)
        assert not pending, "requests did not complete"
        return outs, srv.stats()
    finally:
        srv.close()


@pytest.mark.parametrize("max_wave,max_inflight,spread,host_access",
                         [(64, 3, 0.0, 0), (8, 2, 0.0005, 0), (1, 1, 0.0, 0), (64, 3, 0.0, 2), (8, 2, 0.0005, 2)])
def test_server_results_match_the_oracle(env, max_wave, max_inflight, spread, host_access):
    torch, ctx = env
    ctx.set_host_access(host_access)
    keys = [bytes(range(16)), bytes(range(32)), bytes(range(50, 82)), bytes(range(7, 23))]
    handles = [ctx.key_register(k) for k in keys]
    reqs = _requests(41, 48, keys)
    outs, stats = _run(ctx, reqs, handles, max_wave, max_inflight, spread)
    assert stats["error"] == 0
    for i, q in enumerate(reqs):
        status, out, tag = outs[i]
        if q["op"] == 0:
            assert status == 0
            assert out[: len(q["pt"])].tobytes() == q["ct"]
            assert tag.tobytes() == q["tag"]
        elif q["bad"]:
            assert status == -3
            assert out[: len(q["ct"])].tobytes() == bytes(len(q["ct"]))
        else:
            assert status == 0
            assert out[: len(q["ct"])].tobytes() == q["pt"]
    if max_wave > 1 and spread == 0.0:
        assert stats["waves"] < len(reqs)  # requests were batched
    ctx.set_host_access(0)


def test_server_rejects_bad_requests(env):
    torch, ctx = env
    from paper_2602_23067_gb300 import GcmError

    h = ctx.key_register(bytes(16))
    big = np.zeros(2 << 20, np.uint8)
    out = np.zeros(2 << 20, np.uint8)
    ctx.set_host_access(2)  # staged: the payload must fit the device budget
    try:
        with ctx.server(hbm_budget_bytes=1 << 20) as srv:
            with pytest.raises(GcmError):
                srv.submit(0, h + 100, bytes(12), None, np.zeros(16, np.uint8), np.zeros(16, np.uint8),
                           np.zeros(16, np.uint8))
            with pytest.raises(GcmError) as e:
                srv.submit(0, h, bytes(12), None, big, out, np.zeros(16, np.uint8))
            assert e.value.code == -4
    finally:
        ctx.set_host_access(0)
    # direct host access keeps the payload in host memory, so it fits
    with ctx.server(hbm_budget_bytes=1 << 20) as srv:
        tag = np.zeros(16, np.uint8)
        srv.submit(0, h, bytes(12), None, big, out, tag)
        deadline = time.time() + 30
        done = []
        while not done and time.time() < deadline:
            done = srv.poll()
            time.sleep(0.001)
        assert done and done[0][1] == 0
        ref_ct, ref_tag = oracle.gcm_encrypt(bytes(16), bytes(12), b"", big.tobytes())
        assert tag.tobytes() == ref_tag and out.tobytes() == ref_ct


def test_admission_under_a_binding_budget_with_mib_requests(env):
    # Staged host access, so that every payload occupies device memory, and a
    # 48 MiB budget for about 150 MiB of requests queued at once (4..32 MiB
    # and small ones, encrypt and decrypt-verify, one tampered tag): the
    # server must hold requests back until waves in flight release memory,
    # never hold more than the budget, and still give every request the
    # oracle's result.  The oracle runs chunk by chunk on the host cores.
    torch, ctx = env
    from oracle import mapreduce

    keys = [bytes(range(32)), bytes(range(16)), bytes(range(100, 124))]
    handles = [ctx.key_register(k) for k in keys]
    r = random.Random(71)
    sizes = [32 << 20, 4 << 20, 2880, 16 << 20, (8 << 20) + 5, 70000, (32 << 20) - 2880, (4 << 20) + 7, 5000,
             16 << 20, (24 << 20) + 3, 0, 200003]
    reqs = []
    for i, n in enumerate(sizes):
        k = r.randrange(len(keys))
        iv = bytes(r.getrandbits(8) for _ in range(12 if i % 4 else 40))
        aad = bytes(r.getrandbits(8) for _ in range(r.choice((0, 20, 2880))))
        reqs.append({"k": k, "key": keys[k], "iv": iv, "aad": aad, "n": n, "op": i % 2,
                     "bad": i == 9})
    total = sum(q["n"] for q in reqs)
    with mapreduce.HostInput(total) as src, mapreduce.HostInput(total) as dst:
        spec, off = [], 0
        for i, q in enumerate(reqs):
            src.array[off:off + q["n"]] = workloads.random_bytes(7100 + i, q["n"])
            spec.append({"key": q["key"], "iv": q["iv"], "aad": q["aad"], "off": off, "len": q["n"]})
            q["off"] = off
            off += q["n"]
        ref = mapreduce.gcm_encrypt_digests(spec, src, chunk_bytes=4 << 20, dest=dst)
        pts = np.array(src.array[:max(1, total)])
        cts = np.array(dst.array[:max(1, total)])
    budget = 48 << 20
    ctx.set_host_access(2)
    try:
        # every buffer is ready before the first submission, so the requests
        # reach the server's queue within a fraction of the first wave's time
        bufs = []
        for i, q in enumerate(reqs):
            o, n = q["off"], q["n"]
            if q["op"] == 0:
                inp, tag = pts[o:o + n].copy(), np.zeros(16, np.uint8)
            else:
                inp = cts[o:o + n].copy()
                tb = bytearray(ref[i][1])
                if q["bad"]:
                    tb[7] ^= 0x40
                tag = np.frombuffer(bytes(tb), dtype=np.uint8).copy()
            bufs.append((inp, np.full(max(1, n), 0xA5, dtype=np.uint8), tag))
        srv = ctx.server(hbm_budget_bytes=budget, max_wave_msgs=64, max_inflight=3)
        try:
            pending = {}
            for i, q in enumerate(reqs):
                n = q["n"]
                inp, out, tag = bufs[i]
                t = srv.submit(q["op"], handles[q["k"]], q["iv"], q["aad"] or None,
                               inp if n else np.zeros(0, np.uint8), out[:n] if n else out[:0], tag, user=i)
                pending[t] = (i, inp, out, tag)
            done = {}
            deadline = time.time() + 300
            while pending and time.time() < deadline:
                for ticket, status, arr, fin, user in srv.poll():
                    i, inp, out, tag = pending.pop(ticket)
                    done[i] = (status, out, tag)
                time.sleep(0.001)
            assert not pending, "requests did not complete"
            stats = srv.stats()
        finally:
            srv.close()
    finally:
        ctx.set_host_access(0)
    assert stats["error"] == 0
    assert stats["budget"] == budget
    assert 0 < stats["peak_bytes_in_flight"] <= budget
    assert stats["budget_waits"] > 0  # admission was deferred on memory
    assert total > 2 * budget
    for i, q in enumerate(reqs):
        status, out, tag = done[i]
        o, n = q["off"], q["n"]
        if q["op"] == 0:
            assert status == 0, i
            assert tag.tobytes() == ref[i][1], i
            assert np.array_equal(out[:n], cts[o:o + n]), i
        elif q["bad"]:
            assert status == -3, i
            assert not out[:n].any(), i
        else:
            assert status == 0, i
            assert np.array_equal(out[:n], pts[o:o + n]), i
