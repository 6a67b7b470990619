"""The secondary benchmark workloads (``bench.py --workload ...``): the
10,000-message batch, the Poisson serving stream, the 64 GiB catalog in host
memory, the single 1 MiB message and small batches replayed as CUDA graphs.

Each runner times the library's calls and prints one JSON line.  The CPU
baselines (and the 1 MiB workload's check of message 0) are callables that
``bench.py`` passes in; they run outside every timed region.
"""
from __future__ import annotations

import json
import math
import statistics
import time

from .harness import (ClockSampler, ctypes_buf, dist_setup, load_peaks, mem_available, percentile)


def run_batched(args, cpu_baseline=None):
    """10,000 independent messages (lognormal lengths, median 2 MiB, clipped
    to 16 B..64 MiB, ~30% not multiples of 16, AES-128/256 mixed, 5% non-96-bit
    IVs, AAD 0..4 KiB; payloads are float32 and int16 sky-image bytes):
    one persistent gcm_batch launch versus one gcm_encrypt/gcm_decrypt_verify
    call per message on the same GPU."""
    import ctypes

    import numpy as np
    import torch

    from paper_2602_23067_gb300 import Context, _native, workloads

    rank, local, world = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    n = args.messages
    descs = workloads.message_mix(3 + rank, n, median=2 << 20, sigma=1.0, lo=16, hi=64 << 20, frac_unaligned=0.3,
                                  frac_long_iv=0.05, aad_max=4096, key_sizes=(16, 32))
    lens = [d["len"] for d in descs]
    slot = [(l + 255) // 256 * 256 for l in lens]
    offs = np.concatenate([[0], np.cumsum(slot)]).astype(np.int64)
    total_slots = int(offs[-1])
    payload = sum(lens)
    arena_in = torch.empty(total_slots, dtype=torch.uint8, device="cuda")
    half = total_slots // 2 // 16 * 16
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    step_b = 1 << 28
    for i in range(0, half, step_b):  # float32 sky-like bytes
        arena_in[i: min(half, i + step_b)].view(torch.float32).normal_(1000.0, 50.0, generator=g)
    for i in range(half, total_slots, step_b):  # int16 sky-like bytes
        seg = arena_in[i: min(total_slots, i + step_b)]
        seg.view(torch.int16).copy_(torch.randint(800, 1400, (seg.numel() // 2,), generator=g, device="cuda",
                                                  dtype=torch.int16))
    for i in range(n):  # gaps between 256-byte aligned slots hold zeros
        if slot[i] > lens[i]:
            arena_in[int(offs[i]) + lens[i]: int(offs[i]) + slot[i]].zero_()
    arena_out = torch.empty_like(arena_in)
    arena_back = torch.zeros_like(arena_in)
    aad_sizes = [d["aad_len"] for d in descs]
    aoffs = np.concatenate([[0], np.cumsum(aad_sizes)]).astype(np.int64)
    aad_arena = torch.randint(0, 256, (max(1, int(aoffs[-1])),), dtype=torch.uint8, device="cuda", generator=g)
    tags = torch.empty(n * 16, dtype=torch.uint8, device="cuda")
    ctx = Context(local)
    stream = torch.cuda.current_stream()
    keep = []

    def msg_array(decrypt):
        arr = (_native.GcmMsg * n)()
        for i, d in enumerate(descs):
            kb = ctypes.create_string_buffer(d["key"], len(d["key"]))
            ib = ctypes.create_string_buffer(d["iv"], len(d["iv"]))
            keep.extend([kb, ib])
            src = arena_out if decrypt else arena_in
            dst = arena_back if decrypt else arena_out
            arr[i] = _native.GcmMsg(ctypes.addressof(kb), len(d["key"]), ctypes.addressof(ib), len(d["iv"]),
                                    aad_arena.data_ptr() + int(aoffs[i]) if aad_sizes[i] else None, aad_sizes[i],
                                    src.data_ptr() + int(offs[i]), dst.data_ptr() + int(offs[i]), lens[i],
                                    tags.data_ptr() + 16 * i)
        return arr

    enc_arr, dec_arr = msg_array(False), msg_array(True)
    status = (ctypes.c_int32 * n)()
    done = (ctypes.c_uint64 * n)()

    def batch(arr, decrypt):
        rc = _native.lib.gcm_batch_timed(ctx.handle, arr, n, 1 if decrypt else 0, status, done, stream.cuda_stream)
        if rc != 0:
            raise SystemExit("gcm_batch failed: %s" % _native.last_error())

    # warm-up and correctness of the round trip
    for _ in range(max(1, args.warmup)):
        batch(enc_arr, False)
        batch(dec_arr, True)
    torch.cuda.synchronize()
    if any(status[i] for i in range(n)) or not torch.equal(arena_back, arena_in):
        raise SystemExit("batched round trip failed")

    def timed(fn, reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, (time.perf_counter() - t0) * 1e3 / reps

    reps = max(1, args.steps)
    _native.gcm_profile_enable(ctx.handle, True)
    _native.gcm_profile_read(ctx.handle, reset=True)
    ms_b_enc, wall_b_enc = timed(lambda: batch(enc_arr, False), reps)
    lat_b_enc = [done[i] / 1e6 for i in range(n)]
    ms_b_dec, wall_b_dec = timed(lambda: batch(dec_arr, True), reps)
    lat_b_dec = [done[i] / 1e6 for i in range(n)]
    prof = _native.gcm_profile_read(ctx.handle, reset=True)
    _native.gcm_profile_enable(ctx.handle, False)

    # plain path: one call per message (device memory), same messages
    kbufs = [(ctypes.create_string_buffer(d["key"], len(d["key"])), ctypes.create_string_buffer(d["iv"], len(d["iv"])))
             for d in descs]
    enc_fn, dec_fn = _native.lib.gcm_encrypt, _native.lib.gcm_decrypt_verify
    st_handle = stream.cuda_stream

    def per_message(decrypt, events):
        src = arena_out if decrypt else arena_in
        dst = arena_back if decrypt else arena_out
        sp, dp, ap, tp = src.data_ptr(), dst.data_ptr(), aad_arena.data_ptr(), tags.data_ptr()
        for i in range(n):
            kb, ib = kbufs[i]
            a = ap + int(aoffs[i]) if aad_sizes[i] else None
            if decrypt:
                rc = dec_fn(ctx.handle, ctypes.addressof(kb), len(kb), ctypes.addressof(ib), len(ib), a,
                            aad_sizes[i], sp + int(offs[i]), lens[i], tp + 16 * i, dp + int(offs[i]), 0, st_handle)
            else:
                rc = enc_fn(ctx.handle, ctypes.addressof(kb), len(kb), ctypes.addressof(ib), len(ib), a,
                            aad_sizes[i], sp + int(offs[i]), lens[i], dp + int(offs[i]), tp + 16 * i, 0, st_handle)
            if rc != 0:
                raise SystemExit("per-message call failed: %s" % _native.last_error())
            if events is not None:
                events[i].record(stream)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    per_message(False, None)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    t0 = time.perf_counter()
    per_message(False, ev)
    torch.cuda.synchronize()
    wall_p_enc = (time.perf_counter() - t0) * 1e3
    lat_p_enc = [e0.elapsed_time(x) for x in ev]
    ms_p_enc = lat_p_enc[-1]
    e0.record(stream)
    t0 = time.perf_counter()
    per_message(True, ev)
    torch.cuda.synchronize()
    wall_p_dec = (time.perf_counter() - t0) * 1e3
    lat_p_dec = [e0.elapsed_time(x) for x in ev]
    ms_p_dec = lat_p_dec[-1]
    if not torch.equal(arena_back, arena_in):
        raise SystemExit("per-message round trip failed")

    gbs = lambda ms: payload / (ms * 1e-3) / 1e9
    value = 2 * payload / ((wall_b_enc + wall_b_dec) * 1e-3) / 1e9
    cpu = cpu_baseline(descs) if cpu_baseline is not None and rank == 0 else None
    peak, peak_kind = load_peaks()
    kern_ms = prof["fused_ms"] / max(1, prof["fused_launches"])
    kern_bytes = prof["fused_bytes"] / max(1, prof["fused_launches"])
    line = {
        "metric": "AES-GCM GB/s, 10,000-message batch in one persistent launch (enc + decrypt-verify), "
                  "p50/p99 per-message latency vs per-message launches",
        "value": value,
        "unit": "GB/s",
        "n_gpus": world,
        "steps": reps,
        "warmup": args.warmup,
        "ms_per_step": wall_b_enc + wall_b_dec,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": "batched_10k_lognormal2MiB", "messages": n, "payload_bytes": payload,
                   "lengths": "lognormal median 2 MiB sigma 1.0 clipped 16 B..64 MiB, 30% not multiples of 16",
                   "keys": "AES-128/AES-256 50/50, distinct", "ivs": "96-bit, 5% 8..128 bytes",
                   "aad": "0..4 KiB", "tile": "2^16 blocks"},
        "batched": {"encrypt_gbs": gbs(wall_b_enc), "decrypt_verify_gbs": gbs(wall_b_dec),
                    "encrypt_device_ms": ms_b_enc, "decrypt_device_ms": ms_b_dec,
                    "latency_ms_encrypt": {"p50": percentile(lat_b_enc, 0.5), "p99": percentile(lat_b_enc, 0.99)},
                    "latency_ms_decrypt": {"p50": percentile(lat_b_dec, 0.5), "p99": percentile(lat_b_dec, 0.99)}},
        "per_message": {"encrypt_gbs": gbs(wall_p_enc), "decrypt_verify_gbs": gbs(wall_p_dec),
                        "latency_ms_encrypt": {"p50": percentile(lat_p_enc, 0.5), "p99": percentile(lat_p_enc, 0.99)},
                        "latency_ms_decrypt": {"p50": percentile(lat_p_dec, 0.5), "p99": percentile(lat_p_dec, 0.99)}},
        "speedup_batched_vs_per_message": {"encrypt": wall_p_enc / wall_b_enc, "decrypt_verify": wall_p_dec / wall_b_dec},
        "roofline": {"bound": "hbm", "achieved": kern_bytes / (kern_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": kern_bytes / (kern_ms * 1e-3) / 1e9 / peak, "traffic": None,
                     "kernel": "batch_kernel (persistent, all messages)"},
        "gpu_launches": prof["launches"],
        "e2e": None,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_serving(args):
    """Poisson arrivals of encrypt / decrypt-verify requests (50/50) on pinned
    host buffers, sizes lognormal (median 1 MiB, sigma 1.5) clipped to
    2880 B..256 MiB and rounded up to whole 2880-byte records, 256 cached keys
    (AES-128/AES-256), 1% of decryptions with one flipped tag bit; the
    continuous-batching server against a one-request-per-launch server, per
    arrival rate: p50/p99 latency (arrival to outputs in host memory) and
    GB/s."""
    import ctypes
    import math

    import numpy as np
    import torch

    from paper_2602_23067_gb300 import Context, workloads

    rank, local, world = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    rng = np.random.default_rng(4)
    ctx = Context(local)
    n_keys, n_prep = 256, args.prepared
    keys = [rng.integers(0, 256, 16 if i % 2 else 32, dtype=np.uint8).tobytes() for i in range(n_keys)]
    handles = [ctx.key_register(k) for k in keys]
    sizes = np.clip(rng.lognormal(math.log(1 << 20), 1.5, n_prep), 2880, 256 << 20)
    sizes = (np.ceil(sizes / 2880) * 2880).astype(np.int64)
    prep = []
    total = int(sizes.sum())
    pt_all = torch.empty(total, dtype=torch.uint8, pin_memory=True)
    ct_all = torch.empty(total, dtype=torch.uint8, pin_memory=True)
    out_all = torch.empty(total, dtype=torch.uint8, pin_memory=True)
    pt_all.copy_(torch.randint(0, 256, (total,), dtype=torch.uint8, device="cuda"))
    off = 0
    batch = []
    for i in range(n_prep):
        n = int(sizes[i])
        k = int(rng.integers(0, n_keys))
        iv = rng.integers(0, 256, 12, dtype=np.uint8).tobytes()
        aad = workloads.fits_header(int(rng.integers(0, 1 << 30)), -32, [n // 4, 1], ncards=36)
        tag = np.zeros(16, np.uint8)
        prep.append({"n": n, "k": k, "iv": iv, "aad": np.frombuffer(aad, np.uint8).copy(),
                     "pt": pt_all[off: off + n], "ct": ct_all[off: off + n], "out": out_all[off: off + n],
                     "tag": tag})
        batch.append({"key": keys[k], "iv": iv, "aad": prep[-1]["aad"], "inp": pt_all[off: off + n],
                      "out": ct_all[off: off + n], "tag": tag})
        off += n
    ctx.batch(batch)  # pre-encrypt: ciphertexts and tags for the decrypt requests
    for p in prep:
        bad = p["tag"].copy()
        bad[int(rng.integers(0, 16))] ^= np.uint8(1 << int(rng.integers(0, 8)))
        p["bad"] = bad
    rates = [int(r) for r in args.rates.split(",")]

    def run_rate(rate, server_kind):
        if server_kind == "continuous":
            srv = ctx.server(hbm_budget_bytes=40 * 10 ** 9, max_wave_msgs=4096, max_inflight=3)
        else:
            srv = ctx.server(hbm_budget_bytes=40 * 10 ** 9, max_wave_msgs=1, max_inflight=1)
        count = int(min(args.max_requests, max(2000, rate * args.seconds)))
        r = np.random.default_rng(rate)
        gaps = r.exponential(1.0 / rate, count)
        picks = r.integers(0, n_prep, count)
        ops = r.integers(0, 2, count)
        flips = r.random(count) < 0.01
        from paper_2602_23067_gb300 import _native

        now = _native.lib.gcm_now_ns
        rel = np.cumsum(gaps * 1e9).astype(np.int64)
        lat, done_bytes, auth_ok, auth_bad = [], 0, 0, 0
        # All requests are built up front; the loop hands every request whose
        # arrival time has passed to the server in one call.
        from paper_2602_23067_gb300.api import _host_buf

        reqs = (_native.GcmRequest * count)()
        tags = np.zeros((count, 16), np.uint8)
        keep = []
        expect_bad = set()
        for j in range(count):
            p = prep[picks[j]]
            ivp, ivl, ivk = _host_buf(p["iv"])
            keep.append(ivk)
            if ops[j] == 0:
                src, tg = p["pt"], tags[j]
            else:
                src = p["ct"]
                tg = p["bad"] if flips[j] else p["tag"]
                if flips[j]:
                    expect_bad.add(j)
            reqs[j] = _native.GcmRequest(int(ops[j]), handles[p["k"]], ivp, ivl, p["aad"].ctypes.data, p["aad"].size,
                                         src.data_ptr(), p["out"].data_ptr(), p["n"],
                                         tg.ctypes.data if isinstance(tg, np.ndarray) else tg, 0, j)
        t0 = now() + 50_000_000
        arrivals = t0 + rel
        for j in range(count):
            reqs[j].arrival_ns = int(arrivals[j])
        req_size = ctypes.sizeof(_native.GcmRequest)
        base = ctypes.addressof(reqs)
        comp = (_native.GcmCompletion * 8192)()
        outstanding = 0
        i = 0
        while i < count or outstanding:
            tnow = now()
            j = int(np.searchsorted(arrivals, tnow, side="right"))
            if j > i:
                rc = _native.lib.gcm_server_submit_batch(srv.handle, base + i * req_size, j - i, None)
                if rc != 0:
                    raise SystemExit("submit failed: %s" % _native.last_error())
                outstanding += j - i
                i = j
            m = _native.lib.gcm_server_poll(srv.handle, comp, 8192)
            for q in range(m):
                c = comp[q]
                outstanding -= 1
                user = c.user
                lat.append((c.complete_ns - c.arrival_ns) / 1e6)
                done_bytes += prep[picks[user]]["n"]
                if user in expect_bad:
                    auth_bad += 1 if c.status == -3 else 0
                elif c.status == 0:
                    auth_ok += 1
        t_end = now()
        stats = srv.stats()
        tm = (ctypes.c_double * 4)()
        _native.lib.gcm_server_timing(srv.handle, tm)
        srv.close()
        elapsed = (t_end - t0) / 1e9
        return {"rate_req_s": rate, "requests": count, "achieved_req_s": count / elapsed,
                "gbs": done_bytes / elapsed / 1e9, "p50_ms": percentile(lat, 0.5), "p99_ms": percentile(lat, 0.99),
                "waves": stats["waves"], "flipped_tags": len(expect_bad), "flipped_rejected": auth_bad,
                "stage_ms": {"host_issue": tm[0], "copy_in": tm[1], "compute": tm[2], "copy_out": tm[3]},
                "good_ok": auth_ok, "good_total": count - len(expect_bad)}

    results = {"continuous": [], "per_request": []}
    for rate in rates:
        results["continuous"].append(run_rate(rate, "continuous"))
        results["per_request"].append(run_rate(rate, "per_request"))
    best = max(results["continuous"], key=lambda x: x["gbs"])
    line = {
        "metric": "AES-GCM serving: p50/p99 latency and GB/s under Poisson arrivals, continuous batching vs "
                  "per-request launch",
        "value": best["gbs"],
        "unit": "GB/s",
        "n_gpus": world,
        "steps": len(rates),
        "warmup": 0,
        "ms_per_step": None,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": "serving_poisson", "rates_req_s": rates, "prepared_messages": n_prep,
                   "sizes": "lognormal median 1 MiB sigma 1.5, 2880 B..256 MiB, whole 2880-B records",
                   "keys": "256 cached (AES-128/AES-256)", "ops": "50/50 encrypt / decrypt-verify",
                   "tamper": "1% of decryptions with one flipped tag bit", "hbm_budget_bytes": 40 * 10 ** 9,
                   "host_buffers": "pinned"},
        "serving": results,
        "e2e": None,
        "cpu_baseline": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_catalog(args, cpu_baseline=None):
    """A catalog of FITS files in host memory: alternating 4096 x 4096 float32
    (67,109,760-byte data unit) and int16 (33,554,880-byte) images with random
    2880-byte headers as AAD, AES-256-GCM encrypt then decrypt-verify of every
    file through gcm_batch with host buffers -- once with the kernels working
    on host memory directly over the CPU-GPU link, once staged through a ring
    of 3 x 256 MiB device chunk buffers with copies overlapped on streams."""
    import ctypes

    import numpy as np
    import torch

    from paper_2602_23067_gb300 import Context, _native, workloads

    rank, local, world = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    n_pairs = args.catalog_pairs
    sizes = []
    for i in range(2 * n_pairs):
        sizes.append(workloads.padded_len(4096 * 4096 * (4 if i % 2 == 0 else 2)))
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    total = int(offs[-1])
    # The catalog lives in host memory, filled from the GPU: page-locked
    # (gcm_host_alloc, exact size) by default, or ordinary pageable memory.
    # Page-locked memory is taken only when the host has room for it.
    hostbuf = None
    memory = args.catalog_memory
    if memory == "pinned":
        avail = mem_available()
        if avail >= total + (16 << 30):
            from paper_2602_23067_gb300 import HostBuffer

            hostbuf = HostBuffer(total, local)
            cat = hostbuf.tensor
        else:
            memory = "pageable (page-locked requested; %.0f GB available)" % (avail / 1e9)
    if hostbuf is None:
        cat = torch.empty(total, dtype=torch.uint8)
    ref_sample = []
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    chunk = 1 << 30
    for o in range(0, total, chunk):
        n = min(chunk, total - o)
        cat[o: o + n].copy_(torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda", generator=g))
    headers = [np.frombuffer(workloads.fits_header(5000 + i, -32 if i % 2 == 0 else 16, [4096, 4096]), np.uint8)
               for i in range(2 * n_pairs)]
    r = np.random.default_rng(5)
    keys = [r.integers(0, 256, 32, dtype=np.uint8).tobytes() for _ in range(2 * n_pairs)]
    ivs = [r.integers(0, 256, 12, dtype=np.uint8).tobytes() for _ in range(2 * n_pairs)]
    tags = np.zeros((2 * n_pairs, 16), np.uint8)
    check_idx = [0, 1, 2 * n_pairs - 1]
    for i in check_idx:
        ref_sample.append(cat[int(offs[i]): int(offs[i]) + sizes[i]].clone())
    keep = []
    arr = (_native.GcmMsg * (2 * n_pairs))()
    base = cat.data_ptr()
    for i in range(2 * n_pairs):
        kb = ctypes.create_string_buffer(keys[i], 32)
        ib = ctypes.create_string_buffer(ivs[i], 12)
        keep += [kb, ib]
        arr[i] = _native.GcmMsg(ctypes.addressof(kb), 32, ctypes.addressof(ib), 12, headers[i].ctypes.data, 2880,
                                base + int(offs[i]), base + int(offs[i]), sizes[i], tags[i].ctypes.data)
    status = (ctypes.c_int32 * (2 * n_pairs))()
    results = {}
    for mode, name in ((0, "direct"), (2, "staged_256MiB_x3")):
        ctx = Context(local)
        ctx.set_host_access(mode)
        ctx.set_streaming(256 << 20, 3)
        times = []
        for direction in (0, 1):  # encrypt in place, then decrypt-verify in place
            t0 = time.perf_counter()
            rc = _native.lib.gcm_batch(ctx.handle, arr, 2 * n_pairs, direction, status, 1, None)
            times.append(time.perf_counter() - t0)
            if rc != 0 or any(status[i] for i in range(2 * n_pairs)):
                raise SystemExit("catalog %s failed: %s" % (name, _native.last_error()))
        for k, i in enumerate(check_idx):
            if not torch.equal(cat[int(offs[i]): int(offs[i]) + sizes[i]], ref_sample[k]):
                raise SystemExit("catalog round trip mismatch")
        results[name] = {"encrypt_gbs": total / times[0] / 1e9, "decrypt_verify_gbs": total / times[1] / 1e9,
                         "encrypt_s": times[0], "decrypt_s": times[1]}
        ctx.close()
    best = max(results.values(), key=lambda x: x["encrypt_gbs"] + x["decrypt_verify_gbs"])
    cpu = cpu_baseline(keys, ivs) if cpu_baseline is not None and rank == 0 else None
    line = {
        "metric": "AES-256-GCM catalog stream GB/s: 64 GiB of FITS files in host memory, encrypt + decrypt-verify",
        "value": 2 * total / (best["encrypt_s"] + best["decrypt_s"]) / 1e9,
        "unit": "GB/s",
        "n_gpus": world,
        "steps": 1,
        "warmup": 0,
        "ms_per_step": 1e3 * (best["encrypt_s"] + best["decrypt_s"]),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": "catalog_64GiB", "files": 2 * n_pairs, "bytes": total,
                   "files_kind": "alternating 4096x4096 float32 / int16 data units, random headers as AAD",
                   "host_memory": "page-locked (gcm_host_alloc)" if hostbuf is not None else memory,
                   "in_place": True},
        "catalog": results,
        "e2e": {"value": 2 * total / (best["encrypt_s"] + best["decrypt_s"]) / 1e9, "unit": "GB/s",
                "h2d_bytes_per_step": 2 * total, "d2h_bytes_per_step": 2 * total},
        "cpu_baseline": cpu,
    }
    del cat
    if hostbuf is not None:
        hostbuf.free()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_small(args, cpu_baseline=None, check=None):
    """The plain single-message workload: one 1 MiB AES-128-GCM message
    (uniform random bytes, 96-bit IV, 20-byte AAD), encrypt then
    decrypt-verify through gcm_encrypt / gcm_decrypt_verify on device
    buffers.  The timed steps rotate over 256 distinct messages (256 MiB of
    inputs, above the 129 MB L2), so no step reads a warm input; message 0 is
    the seeded message the parity tests use and is handed to ``check`` (if
    given) before any timing."""
    import numpy as np
    import torch

    from paper_2602_23067_gb300 import Context, _native, workloads

    rank, local, world = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    n_msgs, size = 256, 1 << 20
    r = workloads.rng(1)
    key = r.integers(0, 256, 16, dtype=np.uint8).tobytes()
    iv = r.integers(0, 256, 12, dtype=np.uint8).tobytes()
    aad = r.integers(0, 256, 20, dtype=np.uint8).tobytes()
    pt0 = workloads.random_bytes(11, size).tobytes()
    ctx = Context(local)
    stream = torch.cuda.current_stream()
    pts = torch.empty((n_msgs, size), dtype=torch.uint8, device="cuda")
    pts[0].copy_(torch.frombuffer(bytearray(pt0), dtype=torch.uint8))
    g = torch.Generator(device="cuda")
    g.manual_seed(1 + rank)
    pts[1:].random_(0, 256, generator=g)
    cts = torch.empty_like(pts)
    backs = torch.empty_like(pts)
    tags = torch.empty((n_msgs, 16), dtype=torch.uint8, device="cuda")
    d_aad = torch.frombuffer(bytearray(aad), dtype=torch.uint8).cuda()

    # Per-message views made once, so that the timed calls measure the
    # library calls rather than tensor indexing.
    pv, cv, tv, bv = ([x[i] for i in range(n_msgs)] for x in (pts, cts, tags, backs))

    def step(i):
        ctx.encrypt_device(key, iv, d_aad, pv[i], ct=cv[i], tag=tv[i], stream=stream)
        ctx.decrypt_verify_device(key, iv, d_aad, cv[i], tv[i], pt=bv[i], stream=stream)

    step(0)
    torch.cuda.synchronize()
    if check is not None:  # before any timing
        check(key, iv, aad, pt0, bytes(cts[0].cpu().numpy()), bytes(tags[0].cpu().numpy()))
    if not torch.equal(backs[0], pts[0]):
        raise SystemExit("1 MiB round trip mismatch")
    for i in range(max(args.warmup, 3)):
        step(i % n_msgs)
    steps = max(args.steps, 200)
    _native.gcm_profile_enable(ctx.handle, True)
    _native.gcm_profile_read(ctx.handle, reset=True)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.25)
    torch.cuda.synchronize()
    lat = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        t0 = time.perf_counter()
        step(k % n_msgs)  # decrypt-verify returns after the verdict is on the host
        lat.append(time.perf_counter() - t0)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    prof = _native.gcm_profile_read(ctx.handle, reset=True)
    _native.gcm_profile_enable(ctx.handle, False)

    # the allocation-free entry point, encryption only, same rotation
    tagbuf = torch.empty(16, dtype=torch.uint8, device="cuda")
    kb, ib = (ctypes_buf(key), ctypes_buf(iv))
    na_lat = []
    for k in range(steps + 3):
        i = k % n_msgs
        t0 = time.perf_counter()
        rc = _native.gcm_encrypt_noalloc(kb[0], len(key), ib[0], len(iv), d_aad.data_ptr(), len(aad),
                                         pts[i].data_ptr(), size, cts[i].data_ptr(), tagbuf.data_ptr(),
                                         stream.cuda_stream)
        if rc:
            raise SystemExit("gcm_encrypt_noalloc failed: %s" % _native.noalloc_last_error())
        stream.synchronize()
        if k >= 3:
            na_lat.append(time.perf_counter() - t0)
    if rank != 0:
        return 0
    peak, peak_kind = load_peaks()
    kern_ms = prof["fused_ms"] / max(1, prof["fused_launches"])
    kern_bytes = prof["fused_bytes"] / max(1, prof["fused_launches"])
    achieved = kern_bytes / (kern_ms * 1e-3) / 1e9
    cpu = cpu_baseline(key, iv, aad, pt0) if cpu_baseline is not None else None
    us = [x * 1e6 for x in lat]
    line = {
        "metric": "AES-128-GCM GB/s, one 1 MiB message per call (encrypt + decrypt-verify), latency p50/p99",
        "value": world * 2 * size * steps / (ms * 1e-3) / 1e9,
        "unit": "GB/s",
        "n_gpus": world,
        "steps": steps,
        "warmup": max(args.warmup, 3),
        "ms_per_step": ms / steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": "plain_1MiB_aes128gcm_enc+dec", "cipher": "AES-128-GCM", "iv_bits": 96,
                   "aad_bytes": 20, "payload_bytes": size,
                   "l2": "steps rotate over 256 distinct 1 MiB messages (256 MiB > 129 MB L2)"},
        "latency_us": {"p50": percentile(us, 0.5), "p99": percentile(us, 0.99), "mean": statistics.mean(us),
                       "what": "host wall time of gcm_encrypt + gcm_decrypt_verify (the verdict read back)"},
        "noalloc_encrypt_latency_us": {"p50": percentile([x * 1e6 for x in na_lat], 0.5),
                                       "p99": percentile([x * 1e6 for x in na_lat], 0.99),
                                       "what": "gcm_encrypt_noalloc + stream synchronize"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "fused_kernel<10> (AES-128 CTR + GHASH map)",
                     "algorithmic_bytes_per_launch": kern_bytes, "avg_launch_ms": kern_ms,
                     "peak_source": "%s hbm_gbs" % peak_kind},
        "cpu_baseline": cpu,
        "e2e": None,
        "gpu_launches": prof["launches"],
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_plan(args):
    """Small batches, where the host's work per batch is comparable to the
    device's: for batches of B messages (lognormal lengths, median 16 KiB,
    clipped 16 B..256 KiB, ~30% not multiples of 16, AES-128/256 mixed, 5%
    non-96-bit IVs, AAD 0..4 KiB), the host latency from the first call to
    the verdicts being on the host, of

      * one gcm_encrypt call per message, then a stream synchronisation
        (the key cache holds every key of the batch);
      * one gcm_batch call (the persistent launch; returns with the verdicts);
      * a batch plan: one gcm_batch_plan_set replacing all B messages (the
        next window's buffers and IVs, the same keys: the key material is
        kept), one graph launch, the wait;
      * the same plan replayed without changes (the floor of a replay);
      * the plan with other keys in every window (key setup in every run).

    Every repetition takes the next of 8 windows of the input arena (other
    buffers, other IVs), and L2 is flushed (a 256 MiB write) before each
    repetition, outside the timed interval.  Calls go through the ctypes
    binding with their argument arrays built beforehand."""
    import ctypes

    import numpy as np
    import torch

    from paper_2602_23067_gb300 import Context, _native, workloads

    rank, local, world = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    ctx = Context(local)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    lib = _native.lib
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    sizes = [int(x) for x in args.batch_sizes.split(",")]
    reps = max(20, args.steps)
    W = 8
    results = {}
    launches = 0
    _native.gcm_profile_read(ctx.handle, reset=True)
    for B in sizes:
        descs = workloads.message_mix(40 + B, B, median=16 << 10, sigma=1.0, lo=16, hi=256 << 10,
                                      frac_unaligned=0.3, frac_long_iv=0.05, aad_max=4096, key_sizes=(16, 32))
        lens = [d["len"] for d in descs]
        aads = [d["aad_len"] for d in descs]
        slot = [(n + 255) // 256 * 256 for n in lens]
        offs = np.concatenate([[0], np.cumsum(slot)]).astype(np.int64)
        aoffs = np.concatenate([[0], np.cumsum(aads)]).astype(np.int64)
        win = int(offs[-1])
        g = torch.Generator(device="cuda")
        g.manual_seed(B)
        arena_in = torch.randint(0, 256, (W * win,), dtype=torch.uint8, device="cuda", generator=g)
        arena_out = torch.empty_like(arena_in)
        aad_arena = torch.randint(0, 256, (max(1, W * int(aoffs[-1])),), dtype=torch.uint8, device="cuda",
                                  generator=g)
        tags = torch.empty(W * B * 16, dtype=torch.uint8, device="cuda")
        r = workloads.rng(7 + B)
        keep = []

        def window_arrays(new_keys):
            return [window_array(w, new_keys) for w in range(W)]

        def window_array(w, new_keys):
            arr = (_native.GcmMsg * B)()
            for i, d in enumerate(descs):
                key = r.integers(0, 256, len(d["key"]), dtype=np.uint8).tobytes() if new_keys else d["key"]
                kb = ctypes.create_string_buffer(key, len(d["key"]))
                ib = ctypes.create_string_buffer(r.integers(0, 256, len(d["iv"]), dtype=np.uint8).tobytes(),
                                                 len(d["iv"]))
                keep.extend([kb, ib])
                a = aad_arena.data_ptr() + w * int(aoffs[-1]) + int(aoffs[i]) if aads[i] else None
                arr[i] = _native.GcmMsg(ctypes.addressof(kb), len(d["key"]), ctypes.addressof(ib), len(d["iv"]),
                                        a, aads[i], arena_in.data_ptr() + w * win + int(offs[i]),
                                        arena_out.data_ptr() + w * win + int(offs[i]), lens[i],
                                        tags.data_ptr() + 16 * (w * B + i))
            return arr

        arrays = window_arrays(False)  # the same keys in every window, other IVs
        arrays_new_keys = window_arrays(True)  # other keys and IVs in every window
        status = (ctypes.c_int32 * B)()

        ctx.set_key_cache(max(64, B))  # every key of the batch stays set up for the per-message calls

        def per_message(w):
            for m in arrays[w]:
                rc = lib.gcm_encrypt(ctx.handle, m.key, m.key_len, m.iv, m.iv_len, m.aad, m.aad_len, m.in_,
                                     m.len, m.out, m.tag, 0, sh)
                if rc:
                    raise SystemExit("gcm_encrypt failed: %s" % _native.last_error())
            stream.synchronize()

        def batch(w):
            if lib.gcm_batch(ctx.handle, arrays[w], B, 0, status, 0, sh):
                raise SystemExit("gcm_batch failed: %s" % _native.last_error())

        plan = ctypes.c_void_p()
        if lib.gcm_batch_plan_create(ctx.handle, arrays[0], B, 0, ctypes.byref(plan)):
            raise SystemExit("gcm_batch_plan_create failed: %s" % _native.last_error())

        def plan_run(w, source=arrays):
            if w is not None and lib.gcm_batch_plan_set(plan, 0, source[w], B):
                raise SystemExit("gcm_batch_plan_set failed: %s" % _native.last_error())
            if lib.gcm_batch_plan_launch(plan, sh) or lib.gcm_batch_plan_wait(plan, status):
                raise SystemExit("batch plan run failed: %s" % _native.last_error())

        # the three paths agree on every window (parity against the oracle is
        # in the tests)
        outs = []
        for fn in (per_message, batch, plan_run):
            arena_out.zero_()
            tags.zero_()
            for w in range(W):
                fn(w)
            torch.cuda.synchronize()
            outs.append(torch.cat([arena_out, tags]).clone())
        if not (torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])):
            raise SystemExit("the batch paths disagree")
        del outs

        def timed(fn, replay=False):
            lat = []
            for k in range(reps + 3):
                flush.fill_(k & 255)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                fn(None if replay else k % W)
                dt = (time.perf_counter() - t0) * 1e3
                if k >= 3:
                    lat.append(dt)
            return {"p50_ms": percentile(lat, 0.5), "p99_ms": percentile(lat, 0.99), "mean_ms": statistics.mean(lat)}

        res = {"per_message": timed(per_message), "gcm_batch": timed(batch), "plan": timed(plan_run),
               "plan_replay_unchanged": timed(plan_run, replay=True),
               "plan_new_keys_every_run": timed(lambda w: plan_run(w, arrays_new_keys))}
        lib.gcm_batch_plan_destroy(plan)
        payload = sum(lens)
        for v in res.values():
            v["gbs_at_p50"] = payload / (v["p50_ms"] * 1e-3) / 1e9
        res["payload_bytes"] = payload
        res["plan_speedup_p50"] = {"vs_gcm_batch": res["gcm_batch"]["p50_ms"] / res["plan"]["p50_ms"],
                                   "vs_per_message": res["per_message"]["p50_ms"] / res["plan"]["p50_ms"]}
        results[str(B)] = res
        del arena_in, arena_out, aad_arena, tags
        torch.cuda.empty_cache()
    launches = _native.gcm_profile_read(ctx.handle, reset=True)["launches"]
    ref_b = "128" if "128" in results else str(sizes[-1])
    line = {
        "metric": "small batches: host latency per batch (p50/p99), batch plan replayed as a CUDA graph vs "
                  "gcm_batch vs one call per message",
        "value": results[ref_b]["plan"]["p50_ms"],
        "unit": "ms (p50, batch of %s messages, plan)" % ref_b,
        "n_gpus": world,
        "steps": reps,
        "warmup": 3,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": "small_batches_lognormal16KiB", "batch_sizes": sizes,
                   "lengths": "lognormal median 16 KiB sigma 1.0 clipped 16 B..256 KiB, 30% not multiples of 16",
                   "keys": "AES-128/AES-256 50/50", "ivs": "96-bit, 5% 8..128 bytes", "aad": "0..4 KiB",
                   "l2": "256 MiB write before every repetition, outside the timed interval",
                   "host": "ctypes binding, argument arrays built beforehand; encrypt direction"},
        "batches": results,
        "gpu_launches": launches,
        "e2e": None,
        "cpu_baseline": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_plan_tiles(args):
    """The tile size of a device-memory batch, swept: for batches of B small
    messages (the mix of ``run_plan``), plan replays with the same keys at
    every forced tile size 2^9..2^16 (``gcm_ctx_set_tile_log2``), host
    latency p50 / p99 per run (L2 flushed before each, outside the timed
    interval), beside the size the library's own rule picks."""
    import ctypes

    import numpy as np
    import torch

    from paper_2602_23067_gb300 import Context, _native, workloads

    rank, local, world = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    ctx = Context(local)
    lib = _native.lib
    sh = torch.cuda.current_stream().cuda_stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    sizes = [int(x) for x in args.batch_sizes.split(",")]
    reps = max(20, args.steps)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    results = {}
    for B in sizes:
        descs = workloads.message_mix(40 + B, B, median=16 << 10, sigma=1.0, lo=16, hi=256 << 10,
                                      frac_unaligned=0.3, frac_long_iv=0.05, aad_max=4096, key_sizes=(16, 32))
        lens = [d["len"] for d in descs]
        aads = [d["aad_len"] for d in descs]
        offs = np.concatenate([[0], np.cumsum([(n + 255) // 256 * 256 for n in lens])]).astype(np.int64)
        aoffs = np.concatenate([[0], np.cumsum(aads)]).astype(np.int64)
        arena_in = torch.randint(0, 256, (int(offs[-1]),), dtype=torch.uint8, device="cuda")
        arena_out = torch.empty_like(arena_in)
        aad_arena = torch.randint(0, 256, (max(1, int(aoffs[-1])),), dtype=torch.uint8, device="cuda")
        tags = torch.empty(B * 16, dtype=torch.uint8, device="cuda")
        keep = []
        arr = (_native.GcmMsg * B)()
        for i, d in enumerate(descs):
            kb = ctypes.create_string_buffer(d["key"], len(d["key"]))
            ib = ctypes.create_string_buffer(d["iv"], len(d["iv"]))
            keep.extend([kb, ib])
            a = aad_arena.data_ptr() + int(aoffs[i]) if aads[i] else None
            arr[i] = _native.GcmMsg(ctypes.addressof(kb), len(d["key"]), ctypes.addressof(ib), len(d["iv"]), a,
                                    aads[i], arena_in.data_ptr() + int(offs[i]), arena_out.data_ptr() + int(offs[i]),
                                    lens[i], tags.data_ptr() + 16 * i)
        status = (ctypes.c_int32 * B)()
        blocks = sum((n + 15) // 16 + (a + 15) // 16 for n, a in zip(lens, aads))
        ref, sweep = None, {}
        for lg in range(9, 17):
            ctx.set_tile_log2(lg)
            plan = ctypes.c_void_p()
            rc = lib.gcm_batch_plan_create(ctx.handle, arr, B, 0, ctypes.byref(plan))
            ctx.set_tile_log2(0)
            if rc:
                raise SystemExit("gcm_batch_plan_create failed: %s" % _native.last_error())
            lat = []
            for k in range(reps + 3):
                flush.fill_(k & 255)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if (lib.gcm_batch_plan_set(plan, 0, arr, B) or lib.gcm_batch_plan_launch(plan, sh)
                        or lib.gcm_batch_plan_wait(plan, status)):
                    raise SystemExit("batch plan run failed: %s" % _native.last_error())
                if k >= 3:
                    lat.append((time.perf_counter() - t0) * 1e6)
            torch.cuda.synchronize()
            lib.gcm_batch_plan_destroy(plan)
            out = torch.cat([arena_out, tags]).clone()
            if ref is None:
                ref = out
            elif not torch.equal(ref, out):  # every tile size gives the same bytes
                raise SystemExit("tile size %d changed the result" % lg)
            sweep[str(lg)] = {"p50_us": percentile(lat, 0.5), "p99_us": percentile(lat, 0.99)}
        rule = min(16, max(9, round(0.5 * math.log2(max(1.0, blocks / sms) * 2400.0))))
        results[str(B)] = {"blocks_per_sm": blocks / sms, "rule_tile_log2": rule, "sweep": sweep}
        del arena_in, arena_out, aad_arena, tags
        torch.cuda.empty_cache()
    line = {
        "metric": "batch tile size sweep: host latency per plan run (p50/p99) at every forced tile size",
        "value": None,
        "unit": "us",
        "n_gpus": world,
        "steps": reps,
        "warmup": 3,
        "higher_is_better": False,
        "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": "small_batches_lognormal16KiB_tile_sweep", "batch_sizes": sizes,
                   "l2": "256 MiB write before every repetition, outside the timed interval"},
        "batches": results,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0
