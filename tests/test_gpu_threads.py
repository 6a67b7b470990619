"""One context driven by several host threads at once, each on its own CUDA
stream: the calls' key-cache lookups and replacements, stream-ordered
scratch and launches interleave (ctypes releases the GIL for the library's
calls).  Every ciphertext and tag must still be the oracle's, round trips
must hold, and a tampered tag must be refused with the output zero-filled.
The oracle's results are computed on the main thread before the threads
start."""
import random
import threading

import pytest

import oracle
from paper_2602_23067_gb300 import workloads

pytestmark = pytest.mark.gpu

THREADS = 4
CALLS = 12


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_concurrent_calls_on_one_context(torch_cuda):
    from paper_2602_23067_gb300 import Context, GcmError

    torch = torch_cuda
    r = random.Random(8800)
    keys = [bytes(r.getrandbits(8) for _ in range(r.choice((16, 24, 32)))) for _ in range(5)]
    cases = []
    for t in range(THREADS):
        mine = []
        for k in range(CALLS):
            key = keys[r.randrange(len(keys))]
            iv = bytes(r.getrandbits(8) for _ in range(12 if r.random() < 0.7 else r.randrange(1, 100)))
            aad = bytes(r.getrandbits(8) for _ in range(r.randrange(0, 3000)))
            n = r.choice((0, r.randrange(1, 5000), r.randrange(5000, 300000)))
            pt = workloads.random_bytes(8800 + 100 * t + k, n).tobytes()
            ct, tag = oracle.gcm_encrypt(key, iv, aad, pt)
            mine.append((key, iv, aad, pt, ct, tag, k % 5 == 4))
        cases.append(mine)

    def dev(b):
        x = torch.empty(max(1, len(b)), dtype=torch.uint8, device="cuda")
        if b:
            x[: len(b)].copy_(torch.frombuffer(bytearray(b), dtype=torch.uint8))
        return x[: len(b)]

    inputs = [[(dev(c[2]) if c[2] else None, dev(c[3])) for c in mine] for mine in cases]
    torch.cuda.synchronize()
    errors = []
    with Context(0) as ctx:
        ctx.set_key_cache(3)  # fewer entries than keys: hits, misses and replacements race
        barrier = threading.Barrier(THREADS, timeout=120)

        def worker(t):
            try:
                s = torch.cuda.Stream()
                barrier.wait()
                with torch.cuda.stream(s):
                    for (key, iv, aad, pt, ref_ct, ref_tag, tamper), (d_aad, d_pt) in zip(cases[t], inputs[t]):
                        ct, tag = ctx.encrypt_device(key, iv, d_aad, d_pt, stream=s)
                        s.synchronize()
                        got_tag = bytes(tag.cpu().numpy())
                        got_ct = bytes(ct.cpu().numpy()) if len(pt) else b""
                        if got_tag != ref_tag or got_ct != ref_ct:
                            errors.append((t, len(pt), len(iv), "encrypt"))
                            continue
                        if tamper:
                            bad = tag.clone()
                            bad[3] ^= 0x10
                            out = torch.full_like(d_pt, 7)
                            try:
                                ctx.decrypt_verify_device(key, iv, d_aad, ct, bad, pt=out, stream=s)
                                errors.append((t, len(pt), "tamper accepted"))
                            except GcmError:
                                s.synchronize()
                                if len(pt) and int(out.count_nonzero().item()) != 0:
                                    errors.append((t, len(pt), "output not zeroed"))
                        else:
                            back = ctx.decrypt_verify_device(key, iv, d_aad, ct, tag, stream=s)
                            s.synchronize()
                            if len(pt) and bytes(back.cpu().numpy()) != pt:
                                errors.append((t, len(pt), "round trip"))
            except Exception as e:  # reported below with the thread's index
                errors.append((t, repr(e)))

        threads = [threading.Thread(target=worker, args=(t,)) for t in range(THREADS)]
        for th in threads:
            th.start()
        for th in threads:
            th.join(timeout=600)
        assert not any(th.is_alive() for th in threads), "a worker did not finish"
        torch.cuda.synchronize()
    assert not errors, errors[:5]
