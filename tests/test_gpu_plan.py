"""gcm_batch_plan: a device batch captured once into a CUDA graph and
replayed with new keys, IVs, buffers and data (runs whose keys changed set
up the key material again; the others reuse it).  Every run's ciphertexts
and tags are checked byte for byte against the oracle (tolerance: exact);
the plan's results also equal gcm_batch's on the same messages."""
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


def dev(torch, b, n=None):
    n = len(b) if n is None else n
    t = torch.empty(max(16, n), dtype=torch.uint8, device="cuda")
    if b:
        t[: len(b)].copy_(torch.frombuffer(bytearray(b), dtype=torch.uint8))
    return t


def shapes(seed, count):
    """Lengths, key and IV sizes of a mixed batch: AES-128/192/256, 96-bit
    and 8..128-byte IVs, AAD 0..300 bytes, ragged and empty payloads, and one
    message spanning several tiles of the batched kernel (2^16 blocks)."""
    descs = workloads.message_mix(seed, count, median=6000, sigma=1.5, lo=1, hi=300000, frac_unaligned=0.4,
                                  frac_long_iv=0.25, aad_max=300, key_sizes=(16, 24, 32))
    r = random.Random(seed)
    out = [{"len": d["len"] if r.random() > 0.08 else 0, "key_len": len(d["key"]), "iv_len": len(d["iv"]),
            "aad_len": d["aad_len"]} for d in descs]
    out.append({"len": 3 * (1 << 20) + 7, "key_len": 32, "iv_len": 12, "aad_len": 2880})
    out.append({"len": 0, "key_len": 16, "iv_len": 1, "aad_len": 0})
    return out


def contents(seed, shp, keys=None):
    """Fresh key (unless given), IV, AAD and plaintext bytes of the given sizes."""
    r = workloads.rng(seed)

    def b(n):
        return r.integers(0, 256, n, dtype=np.uint8).tobytes()

    out = [{"key": b(s["key_len"]), "iv": b(s["iv_len"]), "aad": b(s["aad_len"]), "pt": b(s["len"])} for s in shp]
    if keys is not None:
        for d, k in zip(out, keys):
            d["key"] = k
    return out


def device_msgs(torch, shp):
    """Device buffers of each message's shape (AAD, input, output, tag)."""
    return [{"aad": dev(torch, b"", s["aad_len"]), "inp": dev(torch, b"", s["len"]), "out": dev(torch, b"", s["len"]),
             "tag": torch.empty(16, dtype=torch.uint8, device="cuda")} for s in shp]


def load(torch, bufs, data, key="pt", into="inp"):
    for b, d in zip(bufs, data):
        if d["aad"]:
            b["aad"][: len(d["aad"])].copy_(torch.frombuffer(bytearray(d["aad"]), dtype=torch.uint8))
        if d[key]:
            b[into][: len(d[key])].copy_(torch.frombuffer(bytearray(d[key]), dtype=torch.uint8))


def as_msg(b, d, key="pt", tag=None):
    return {"key": d["key"], "iv": d["iv"], "aad": b["aad"][: len(d["aad"])] if d["aad"] else None,
            "inp": b["inp"], "out": b["out"], "tag": b["tag"] if tag is None else tag, "len": len(d[key])}


def check_against_oracle(bufs, data):
    for i, (b, d) in enumerate(zip(bufs, data)):
        ref_ct, ref_tag = oracle.gcm_encrypt(d["key"], d["iv"], d["aad"], d["pt"])
        assert bytes(b["tag"].cpu().numpy()) == ref_tag, i
        assert bytes(b["out"][: len(d["pt"])].cpu().numpy()) == ref_ct, i


def test_plan_runs_match_the_oracle_across_replays(env):
    torch, ctx = env
    shp = shapes(41, 46)
    bufs = device_msgs(torch, shp)
    data = contents(1, shp)
    load(torch, bufs, data)
    torch.cuda.synchronize()
    with ctx.batch_plan([as_msg(b, d) for b, d in zip(bufs, data)]) as plan:
        assert plan.run() == [0] * len(shp)
        check_against_oracle(bufs, data)
        spare = device_msgs(torch, shp)
        for run in range(2, 5):
            # new keys, IVs, AAD and plaintexts (same lengths) in the same
            # buffers; every third message moved to other buffers
            data = contents(run, shp)
            if run == 3:
                bufs = [s if i % 3 == 0 else b for i, (b, s) in enumerate(zip(bufs, spare))]
            load(torch, bufs, data)
            torch.cuda.synchronize()
            for i, (b, d) in enumerate(zip(bufs, data)):
                plan.set(i, as_msg(b, d))
            assert plan.run() == [0] * len(shp)
            check_against_oracle(bufs, data)
        # Runs that keep every key (new IVs, AAD and data) reuse the key
        # material of the last run that set it up; then one key changes,
        # which sets up all keys again, and the next run reuses those.
        keys = [d["key"] for d in data]
        for run in range(5, 9):
            if run == 7:
                keys = list(keys)
                keys[5] = bytes(len(keys[5]))
            data = contents(run, shp, keys=keys)
            load(torch, bufs, data)
            torch.cuda.synchronize()
            plan.set_many(0, [as_msg(b, d) for b, d in zip(bufs, data)])
            assert plan.run() == [0] * len(shp)
            check_against_oracle(bufs, data)
        # the same messages through gcm_batch: identical results
        out_plan = [bytes(b["out"][: len(d["pt"])].cpu().numpy()) + bytes(b["tag"].cpu().numpy())
                    for b, d in zip(bufs, data)]
        assert ctx.batch([as_msg(b, d) for b, d in zip(bufs, data)]) == [0] * len(shp)
        torch.cuda.synchronize()
        assert out_plan == [bytes(b["out"][: len(d["pt"])].cpu().numpy()) + bytes(b["tag"].cpu().numpy())
                            for b, d in zip(bufs, data)]


def test_plan_decrypt_gate_then_replay_with_the_right_tags(env):
    torch, ctx = env
    shp = shapes(42, 30)
    data = contents(7, shp)
    for d in data:
        d["ct"], d["tag"] = oracle.gcm_encrypt(d["key"], d["iv"], d["aad"], d["pt"])
    bufs = device_msgs(torch, shp)
    load(torch, bufs, data, key="ct")
    bad = {2, 11, len(shp) - 2}
    for i, (b, d) in enumerate(zip(bufs, data)):
        t = bytearray(d["tag"])
        if i in bad:
            t[i % 16] ^= 0x80
        b["tag"].copy_(torch.frombuffer(t, dtype=torch.uint8))
        b["out"].fill_(0x5A)
    torch.cuda.synchronize()
    with ctx.batch_plan([as_msg(b, d, key="ct") for b, d in zip(bufs, data)], decrypt=True) as plan:
        st = plan.run()
        for i, (b, d) in enumerate(zip(bufs, data)):
            got = bytes(b["out"][: len(d["pt"])].cpu().numpy())
            if i in bad:
                assert st[i] == -3, i
                assert got == bytes(len(d["pt"])), i
            else:
                assert st[i] == 0, i
                assert got == d["pt"], i
        # the expected tags are read at run time: fix them in place and run again
        for i in bad:
            bufs[i]["tag"].copy_(torch.frombuffer(bytearray(data[i]["tag"]), dtype=torch.uint8))
        torch.cuda.synchronize()
        assert plan.run() == [0] * len(shp)
        for b, d in zip(bufs, data):
            assert bytes(b["out"][: len(d["pt"])].cpu().numpy()) == d["pt"]


def test_plan_contract(env):
    torch, ctx = env
    from paper_2602_23067_gb300 import GcmError
    from paper_2602_23067_gb300 import _native as nat

    shp = [{"len": 1000, "key_len": 16, "iv_len": 12, "aad_len": 20}, {"len": 70000, "key_len": 32, "iv_len": 60,
                                                                      "aad_len": 0}]
    bufs = device_msgs(torch, shp)
    data = contents(9, shp)
    load(torch, bufs, data)
    torch.cuda.synchronize()
    with pytest.raises(GcmError) as e:
        ctx.batch_plan([])
    assert e.value.code == nat.GCM_ERR_INVALID_ARG
    with ctx.batch_plan([as_msg(b, d) for b, d in zip(bufs, data)]) as plan:
        free0 = None
        for run in range(6):
            plan.launch()
            if run == 0:
                with pytest.raises(GcmError) as e:  # one run in flight at a time
                    plan.launch()
                assert e.value.code == nat.GCM_ERR_BUSY
            assert plan.wait() == [0, 0]
            if run == 1:
                free0 = torch.cuda.mem_get_info()[0]
        assert torch.cuda.mem_get_info()[0] == free0  # runs allocate nothing
        check_against_oracle(bufs, data)
        with pytest.raises(GcmError) as e:
            plan.wait()
        assert e.value.code == nat.GCM_ERR_INVALID_ARG
        longer = dict(as_msg(bufs[0], data[0]), len=999)
        with pytest.raises(GcmError) as e:  # lengths are fixed at creation
            plan.set(0, longer)
        assert e.value.code == nat.GCM_ERR_INVALID_ARG
        other_key = dict(as_msg(bufs[1], data[1]), key=bytes(16))
        with pytest.raises(GcmError) as e:  # so is the key size
            plan.set(1, other_key)
        assert e.value.code == nat.GCM_ERR_INVALID_ARG
        with pytest.raises(GcmError) as e:
            plan.set(2, as_msg(bufs[1], data[1]))
        assert e.value.code == nat.GCM_ERR_INVALID_ARG
        # the rejected updates changed nothing
        assert plan.run() == [0, 0]
        check_against_oracle(bufs, data)


def test_plan_scratch_counts_against_the_budget(env):
    """A plan holds its scratch (one message: ~70 KB, mostly the key
    material) until it is destroyed, counted in the context's HBM budget: with
    a 120 KB budget a second plan is refused until the first is gone."""
    torch, _ = env
    from paper_2602_23067_gb300 import Context, GcmError
    from paper_2602_23067_gb300 import _native as nat

    shp = [{"len": 4000, "key_len": 32, "iv_len": 12, "aad_len": 16}]
    bufs = device_msgs(torch, shp)
    data = contents(11, shp)
    load(torch, bufs, data)
    torch.cuda.synchronize()
    msgs = [as_msg(b, d) for b, d in zip(bufs, data)]
    with Context(0, hbm_budget_bytes=120_000) as ctx:
        first = ctx.batch_plan(msgs)
        with pytest.raises(GcmError) as e:
            ctx.batch_plan(msgs)
        assert e.value.code == nat.GCM_ERR_NO_MEMORY
        assert first.run() == [0]
        first.close()
        with ctx.batch_plan(msgs) as second:
            assert second.run() == [0]
    check_against_oracle(bufs, data)
