#!/usr/bin/env python3
"""Benchmark: AES-256-GCM on a 4 GiB FITS data unit on GB300.

Workload: one synthetic FITS file, a 2880-byte header (36 cards, used as
AAD) and the data unit of a 32768 x 32768 float32 image (N(1000, 50^2) sky
plus Poisson point sources), zero-padded to whole 2880-byte records:
4,294,969,920 bytes, generated on the device.  One step is the whole data
path in both directions: GCM encryption of the data unit (key setup, fused
CTR + GHASH map, tree combine and tag) followed by decrypt-verify (the same
pass over the ciphertext, the tag check and the validation gate).

    value = payload bytes processed (2 x data unit per step) / device time

measured with CUDA events on the launching stream between a synchronised
start and end; the inputs (4.3 GB) are far larger than the 129 MB L2, so no
flush is needed between steps.  ``e2e`` is the same metric through the C ABI
with pinned host buffers, host<->device copies inside the timed region.

``--impl reference`` times the CPU oracle (plain byte-at-a-time AES-GCM) on a
bounded prefix of the same data unit, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2602_23067_gb300.harness import (ClockSampler, dist_setup, load_peaks,  # noqa: E402
                                            load_pipe_counters, load_traffic, max_over_ranks, mem_available,
                                            whole_job_gbs)

N1 = N2 = 32768  # default image side (the 4 GiB workload); --side changes it
DATA_BYTES = N1 * N2 * 4
METRIC = "AES-GCM GB/s @4GiB on 1 GB300; batched p50/p99 latency vs per-msg launch"
WORKLOAD = "fits_4gib_aes256gcm_enc+dec"
AES_IMPLS = {"tables": 0, "bitsliced": 1}  # GCM_AES_TABLES, GCM_AES_BITSLICED


def workload_config(n_gpus):
    from paper_2602_23067_gb300 import workloads

    padded = workloads.padded_len(DATA_BYTES)
    name = WORKLOAD if N1 == 32768 else "fits_%dx%d_aes256gcm_enc+dec" % (N1, N2)
    return {
        "workload": name,
        "cipher": "AES-256-GCM",
        "iv_bits": 96,
        "aad_bytes": 2880,
        "payload_bytes": padded,
        "image": "%dx%d float32 BITPIX=-32, N(1000,50^2) + 10^4 Poisson point sources" % (N1, N2),
        "step": "gfc_fits_encrypt + gfc_fits_decrypt_verify of the whole file (device memory)",
        "l2": "inputs (4.3 GB) exceed L2 (129 MB); no flush",
        "per_gpu": "one 4 GiB message per GPU" if n_gpus > 1 else "one 4 GiB message",
    }


def cpu_oracle_sample(sample_bytes: int, seed: int = 2):
    """Times the oracle (as it stands) on the first sample_bytes of the
    workload's data unit, encrypt + decrypt-verify, one host thread."""
    import numpy as np

    import oracle
    from paper_2602_23067_gb300 import workloads

    r = workloads.rng(seed)
    key = r.integers(0, 256, 32, dtype=np.uint8).tobytes()
    iv = r.integers(0, 256, 12, dtype=np.uint8).tobytes()
    header = workloads.fits_header(seed, -32, [N1, N2], ncards=36)
    rows = max(1, sample_bytes // (N1 * 4))
    pt = workloads.sky_image_host(seed, N1, rows, n_sources=5).tobytes()[:sample_bytes]
    t0 = time.perf_counter()
    ct, tag = oracle.gcm_encrypt(key, iv, header, pt)
    ok, back = oracle.gcm_decrypt(key, iv, header, ct, tag)
    dt = time.perf_counter() - t0
    assert ok and back == pt
    return 2 * len(pt), dt


def _oracle_message(job):
    """One message through the oracle (encrypt + decrypt-verify) in a pool
    worker; returns (payload bytes processed, seconds)."""
    import oracle
    from paper_2602_23067_gb300 import workloads

    key, iv, aad_len, n, seed = job
    pt = workloads.random_bytes(seed, n).tobytes()
    aad = workloads.random_bytes(seed + 1, aad_len).tobytes()
    t0 = time.perf_counter()
    ct, tag = oracle.gcm_encrypt(key, iv, aad, pt)
    ok, back = oracle.gcm_decrypt(key, iv, aad, ct, tag)
    dt = time.perf_counter() - t0
    assert ok and back == pt
    return 2 * n, dt


def cpu_oracle_pool(jobs, what):
    """Times the oracle, one message per process over all host cores
    (processes started with spawn, so no CUDA state is inherited)."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_message, jobs[:cores])  # warm-up: imports, oracle build check
        t0 = time.perf_counter()
        res = pool.map(_oracle_message, jobs)
        wall = time.perf_counter() - t0
    nbytes = sum(r[0] for r in res)
    return {"value": nbytes / wall / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": "%s: %d messages, %d payload bytes, one message per process on %d host cores (%.1f s)"
                      % (what, len(jobs), nbytes // 2, cores, wall)}


def cpu_batched(descs):
    """Oracle baseline of the batched workload: the first messages of the mix
    no longer than 4 MiB, one message per process."""
    sample = [(d["key"], d["iv"], d["aad_len"], d["len"], d["seed"]) for d in descs if d["len"] <= (4 << 20)]
    return cpu_oracle_pool(sample[: 2 * (os.cpu_count() or 1)],
                           "the first messages of the same mix no longer than 4 MiB (seeded bytes)")


def cpu_catalog(keys, ivs):
    """Oracle baseline of the catalog workload: 4 MiB prefixes of the first
    files, one file per process."""
    cores = os.cpu_count() or 1
    jobs = [(keys[i], ivs[i], 2880, 4 << 20, 5000 + i) for i in range(min(len(keys), 2 * cores))]
    return cpu_oracle_pool(jobs, "4 MiB prefixes of the first catalog files (seeded bytes), AES-256")


def cpu_small(key, iv, aad, pt0):
    """Oracle baseline of the 1 MiB workload: message 0, one host thread."""
    import oracle

    t0 = time.perf_counter()
    c, t = oracle.gcm_encrypt(key, iv, aad, pt0)
    ok, _ = oracle.gcm_decrypt(key, iv, aad, c, t)
    dt = time.perf_counter() - t0
    assert ok
    return {"value": 2 * len(pt0) / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "the whole 1 MiB message 0, encrypt + decrypt-verify, one host thread (%.2f s)" % dt}


def check_small(key, iv, aad, pt0, ct, tag):
    """Message 0 of the 1 MiB workload against the oracle (before timing)."""
    import oracle

    ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, aad, pt0)
    if tag != ref_tag or ct != ref_ct:
        raise SystemExit("1 MiB message differs from the oracle")


def run_reference(args):
    rank, local, world = dist_setup(args.gpus)
    if rank != 0:
        return 0
    # Bound the run to about a minute of host work in total.
    per_step = max(64 * 1024, min(4 << 20, int(60.0 / max(1, args.steps + args.warmup) * 1.5e6)))
    per_step -= per_step % 16
    for _ in range(args.warmup):
        cpu_oracle_sample(per_step)
    total_b, total_t = 0, 0.0
    for _ in range(args.steps):
        b, t = cpu_oracle_sample(per_step)
        total_b += b
        total_t += t
    gbs = total_b / total_t / 1e9
    sample = "first %d bytes of the 4 GiB data unit per step, header as AAD, encrypt + decrypt-verify" % per_step
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": gbs,
        "unit": "GB/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": workload_config(args.gpus),
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    rank, local, world = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import numpy as np

    from paper_2602_23067_gb300 import Context, _native, workloads

    padded = workloads.padded_len(DATA_BYTES)
    seed = 2 + rank
    r = workloads.rng(2)
    key = r.integers(0, 256, 32, dtype=np.uint8).tobytes()
    iv = r.integers(0, 256, 12, dtype=np.uint8).tobytes()
    header = workloads.fits_header(2, -32, [N1, N2], ncards=36)
    hl = len(header)
    ctx = Context(local)
    ctx.set_aes_impl(AES_IMPLS[args.aes_impl])
    # The FITS file on the device: header records, then the padded data unit.
    fits = torch.empty(hl + padded, dtype=torch.uint8, device="cuda")
    fits[:hl].copy_(torch.frombuffer(bytearray(header), dtype=torch.uint8))
    workloads.sky_image_device(seed, N1, N2, out=fits[hl:])
    stream = torch.cuda.current_stream()
    state = {}

    def step(check=False):
        # gfc_fits_encrypt + gfc_fits_decrypt_verify: header parse, header as
        # AAD, fused CTR+GHASH over the data unit, tree combine, tag, and the
        # verify gate on the way back.
        enc, tag = ctx.fits_encrypt_raw(key, fits, iv, stream=stream)
        dec = ctx.fits_decrypt_verify_raw(key, enc.data_buffer, enc.buffer_size, iv, tag, stream=stream)
        if dec.error_code != 0:
            raise SystemExit("tag rejected: %s" % dec.error_message)
        if check:
            torch.cuda.synchronize()
            ok = torch.equal(Context.result_view(dec), fits) and not torch.equal(Context.result_view(enc), fits)
            if not ok:
                raise SystemExit("round trip mismatch")
        state["tag"] = tag
        ctx.release(enc)
        ctx.release(dec)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for i in range(args.warmup):
        step(check=(i == 0))
    torch.cuda.synchronize()

    # ---- device-resident timed region ----
    _native.gcm_profile_enable(ctx.handle, True)
    _native.gcm_profile_read(ctx.handle, reset=True)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.25)
    barrier()
    # One event between consecutive steps (no extra device work), so that
    # the per-step distribution (median, spread; the paper's protocol,
    # Sec. 5.3.1) comes with the total.
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for i in range(args.steps):
        step()
        evs[i + 1].record(stream)
    barrier()
    clocks = sampler.stop() if sampler else None
    e0, e1 = evs[0], evs[-1]
    ms = e0.elapsed_time(e1)
    step_ms = np.array([evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)])
    prof = _native.gcm_profile_read(ctx.handle, reset=True)
    _native.gcm_profile_enable(ctx.handle, False)
    ms = max_over_ranks(ms, dist)
    bytes_per_step = 2 * padded
    value = whole_job_gbs(world, bytes_per_step, args.steps, ms * 1e-3)

    # ---- per-direction device throughput (secondary) ----
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        enc, tag = ctx.fits_encrypt_raw(key, fits, iv, stream=stream)
        ctx.release(enc)
    e1.record(stream)
    barrier()
    enc_gbs = padded * args.steps / (e0.elapsed_time(e1) * 1e-3) / 1e9
    enc, tag = ctx.fits_encrypt_raw(key, fits, iv, stream=stream)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        dec = ctx.fits_decrypt_verify_raw(key, enc.data_buffer, enc.buffer_size, iv, tag, stream=stream)
        ctx.release(dec)
    e1.record(stream)
    barrier()
    dec_gbs = padded * args.steps / (e0.elapsed_time(e1) * 1e-3) / 1e9
    ctx.release(enc)
    pt = fits[hl:]

    # ---- the two halves alone: CTR keystream XOR, GHASH (no AES) ----
    ctr_out = torch.empty_like(pt)
    d_aad = fits[:hl]
    ctx.ctr_xor_device(key, iv, pt, out=ctr_out, stream=stream)
    ctx.ghash_device(key, d_aad, pt, stream=stream)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        ctx.ctr_xor_device(key, iv, pt, out=ctr_out, stream=stream)
    e1.record(stream)
    barrier()
    ctr_ms = e0.elapsed_time(e1) / args.steps
    e0.record(stream)
    for _ in range(args.steps):
        ctx.ghash_device(key, d_aad, pt, stream=stream)
    e1.record(stream)
    barrier()
    ghash_ms = e0.elapsed_time(e1) / args.steps
    tag_buf = torch.empty(16, dtype=torch.uint8, device="cuda")
    e0.record(stream)
    for _ in range(args.steps):
        ctx.encrypt_device(key, iv, d_aad, pt, ct=ctr_out, tag=tag_buf, stream=stream)
    e1.record(stream)
    barrier()
    plain_ms = e0.elapsed_time(e1) / args.steps
    other = None
    if args.aes_impl == "tables":
        # The same two passes with the bitsliced AES engine (same results,
        # checked by the parity tests; timed here for the comparison).
        ctx.set_aes_impl(AES_IMPLS["bitsliced"])
        ctx.ctr_xor_device(key, iv, pt, out=ctr_out, stream=stream)
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            ctx.ctr_xor_device(key, iv, pt, out=ctr_out, stream=stream)
        e1.record(stream)
        barrier()
        bs_ctr_ms = e0.elapsed_time(e1) / args.steps
        e0.record(stream)
        for _ in range(args.steps):
            ctx.encrypt_device(key, iv, d_aad, pt, ct=ctr_out, tag=tag_buf, stream=stream)
        e1.record(stream)
        barrier()
        bs_gcm_ms = e0.elapsed_time(e1) / args.steps
        ctx.set_aes_impl(AES_IMPLS["tables"])
        other = {"engine": "bitsliced (gcm_ctx_set_aes_impl = GCM_AES_BITSLICED)",
                 "ctr_only_gbs": padded / (bs_ctr_ms * 1e-3) / 1e9,
                 "gcm_encrypt_gbs": padded / (bs_gcm_ms * 1e-3) / 1e9}
    del ctr_out
    modes = {
        "ctr_only_gbs": padded / (ctr_ms * 1e-3) / 1e9,
        "ghash_only_gbs": (hl + padded) / (ghash_ms * 1e-3) / 1e9,
        "gcm_encrypt_over_ctr_time": (plain_ms * 1e-3) / (ctr_ms * 1e-3),
        "gcm_encrypt_without_datasum_gbs": padded / (plain_ms * 1e-3) / 1e9,
        "api": "gcm_ctr_xor, gcm_ghash and gcm_encrypt over the same data unit (device memory); the FITS calls of "
               "the step also compute the DATASUM of the encrypted data unit in the same pass",
        "aes_engine": args.aes_impl,
    }
    if other is not None:
        modes["bitsliced"] = other

    # ---- end to end through the C ABI with pinned host buffers ----
    e2e = None
    # Three exact-size page-locked buffers per rank (gcm_host_alloc), when
    # the host has room for them next to the other ranks' (MemAvailable is
    # shared by all ranks of the node).
    local_world = int(os.environ.get("LOCAL_WORLD_SIZE", str(world)))
    barrier()
    short = 0.0 if mem_available() >= 3 * padded * local_world + (16 << 30) else 1.0
    host_room = max_over_ranks(short, dist) == 0.0  # every rank takes the same decision
    if not args.no_e2e and not host_room:
        e2e = {"value": None, "unit": "GB/s", "skipped": "not enough free host memory for 3 page-locked "
                                                         "4.3 GB buffers per rank"}
    if not args.no_e2e and host_room:
        from paper_2602_23067_gb300 import HostBuffer

        torch.cuda.empty_cache()
        bufs = [HostBuffer(padded, local) for _ in range(3)]
        h_pt, h_ct, h_back = (b.tensor for b in bufs)
        h_pt.copy_(pt)
        h_aad = np.frombuffer(header, dtype=np.uint8).copy()
        ksteps = max(2, min(args.steps, 8))

        def host_step():
            _, t = ctx.encrypt_host(key, iv, h_aad, h_pt, ct=h_ct)
            ctx.decrypt_verify_host(key, iv, h_aad, h_ct, t, pt=h_back)

        host_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(ksteps):
            host_step()
        barrier()
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, dist)
        if not torch.equal(h_back, h_pt):
            raise SystemExit("host round trip mismatch")
        del h_pt, h_ct, h_back
        for b in bufs:
            b.free()
        e2e = {
            "value": whole_job_gbs(world, bytes_per_step, ksteps, dt),
            "unit": "GB/s",
            "h2d_bytes_per_step": (2880 + padded) + (2880 + padded + 16),
            "d2h_bytes_per_step": (padded + 16) + (padded + 4),
            "steps": ksteps,
            "api": "gcm_encrypt + gcm_decrypt_verify of the data unit with the header as AAD, GCM_MEM_HOST, "
                   "page-locked host buffers (gcm_host_alloc)",
        }

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel (the fused CTR+GHASH map) ----
    # Achieved = the kernel's algorithmic HBM bytes per launch (2 x payload +
    # AAD) / its average CUDA-event launch time, against the measured HBM copy
    # peak.  The pipe that actually binds the table engine (the shared-memory
    # data pipe: one 128-byte wavefront per clock per SM) is reported beside
    # it, from the ncu wavefront count of the committed capture and the SM
    # clock sampled during the timed region.
    peak, peak_kind = load_peaks()
    kern_ms = prof["fused_ms"] / max(1, prof["fused_launches"])
    kern_bytes = prof["fused_bytes"] / max(1, prof["fused_launches"])
    achieved = kern_bytes / (kern_ms * 1e-3) / 1e9
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roofline = {
        "bound": "hbm",
        "achieved": achieved,
        "peak": peak,
        "unit": "GB/s",
        "frac": achieved / peak,
        "traffic": load_traffic(),
        "peak_source": "%s hbm_gbs (MEASURED_PEAKS.json, copy bandwidth)" % peak_kind
        if peak_kind == "measured" else "fallback 6.8 TB/s",
        "kernel": "fused_kernel<14> (AES-256 CTR + GHASH map)" if args.aes_impl == "tables"
        else "fused_bs_kernel<14> (bitsliced AES-256 CTR + GHASH map)",
        "algorithmic_bytes_per_launch": kern_bytes,
        "avg_launch_ms": kern_ms,
    }
    if args.aes_impl == "tables":
        counters = load_pipe_counters()
        mhz = clocks["sm_mhz"] if clocks and clocks.get("sm_mhz") else None
        pipe = {"what": "shared-memory (LSU) data pipe: 1 wavefront of 128 B per clock per SM; the table engine's "
                        "binding pipe (AES round-table and GHASH-table lookups)",
                "sms": sms, "sm_mhz": mhz, "sm_mhz_source": "median sampled during the timed region"}
        if counters is not None and mhz:
            wpb = counters["wavefronts"]
            payload_peak = sms * mhz * 1e6 / wpb * 16.0 / 1e9
            pipe_peak = payload_peak * kern_bytes / padded  # in algorithmic bytes, like `achieved`
            pipe.update({"wavefronts_per_block": wpb,
                         "wavefronts_source": "ncu, profiles/fused_traffic.json: " + counters["command"],
                         "peak_payload_gbs": payload_peak, "peak_gbs_algorithmic": pipe_peak,
                         "frac": achieved / pipe_peak})
            if counters["warp_instructions"]:
                # The issue bound beside it: 4 warp instructions per clock per
                # SM over the measured warp instructions per block.
                wi = counters["warp_instructions"]
                issue_payload = sms * 4 * mhz * 1e6 / wi * 16.0 / 1e9
                pipe["issue_bound"] = {"warp_instructions_per_block": wi, "peak_payload_gbs": issue_payload,
                                       "frac": achieved / (issue_payload * kern_bytes / padded)}
        else:
            pipe.update({"wavefronts_per_block": None, "frac": None,
                         "note": "no ncu wavefront count for the current kernel source" if counters is None
                         else "no clock samples"})
        roofline["binding_pipe"] = pipe

    cpu = None
    if not args.no_cpu_baseline:
        nb, dt = cpu_oracle_sample(args.cpu_sample_bytes)
        cpu = {"value": nb / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "first %d bytes of the data unit, header as AAD, AES-256-GCM encrypt + decrypt-verify, "
                         "single host thread (%.1f s)" % (args.cpu_sample_bytes, dt)}

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": workload_config(world),
        "step_ms": {"median": float(np.median(step_ms)), "std": float(np.std(step_ms)),
                    "min": float(step_ms.min()), "max": float(step_ms.max()),
                    "what": "device time of each timed step (rank 0), CUDA events between steps"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": prof["launches"],
        "clocks": clocks,
        "directions": {"encrypt_gbs": enc_gbs, "decrypt_verify_gbs": dec_gbs},
        "modes": modes,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--aes-impl", choices=sorted(AES_IMPLS), default="tables",
                    help="AES engine of the 4 GiB workload's context (gcm_ctx_set_aes_impl)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-bytes", type=int, default=8 << 20)
    ap.add_argument("--catalog-pairs", type=int, default=683, help="catalog: float32/int16 file pairs (683 = 64 GiB)")
    ap.add_argument("--catalog-memory", choices=["pinned", "pageable"], default="pinned",
                    help="catalog: page-locked host memory (default) or ordinary pageable memory")
    ap.add_argument("--workload", choices=["fits4g", "small", "batched", "serving", "catalog", "plan", "plan-tiles"],
                    default="fits4g",
                    help="fits4g (default): one 4 GiB FITS file; batched: 10,000 independent messages; "
                         "serving: Poisson request stream; plan: small batches, CUDA-graph plan vs gcm_batch vs "
                         "one call per message; plan-tiles: the same at every forced batch tile size")
    ap.add_argument("--batch-sizes", default="1,16,128,1024", help="plan: messages per batch")
    ap.add_argument("--rates", default="1000,2000,5000,10000,20000,50000", help="serving arrival rates (req/s)")
    ap.add_argument("--seconds", type=float, default=3.0, help="serving: seconds of arrivals per rate")
    ap.add_argument("--max-requests", type=int, default=20000, help="serving: cap on requests per rate")
    ap.add_argument("--prepared", type=int, default=384, help="serving: distinct prepared messages")
    ap.add_argument("--messages", type=int, default=10000, help="messages of the batched workload")
    ap.add_argument("--side", type=int, default=32768,
                    help="image side in pixels (default 32768: the 4 GiB workload; smaller sides are for profiling)")
    args = ap.parse_args()
    global N1, N2, DATA_BYTES
    N1 = N2 = args.side
    DATA_BYTES = N1 * N2 * 4
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    from paper_2602_23067_gb300 import bench_workloads as bw

    cpu = not args.no_cpu_baseline
    if args.workload == "small":
        return bw.run_small(args, cpu_baseline=cpu_small if cpu else None, check=check_small)
    if args.workload == "batched":
        return bw.run_batched(args, cpu_baseline=cpu_batched if cpu else None)
    if args.workload == "serving":
        return bw.run_serving(args)
    if args.workload == "catalog":
        return bw.run_catalog(args, cpu_baseline=cpu_catalog if cpu else None)
    if args.workload == "plan":
        return bw.run_plan(args)
    if args.workload == "plan-tiles":
        return bw.run_plan_tiles(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
