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
