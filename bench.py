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
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N1 = N2 = 32768  # default image side (the 4 GiB workload); --side changes it
DATA_BYTES = N1 * N2 * 4
METRIC = "AES-GCM GB/s @4GiB on 1 GB300; batched p50/p99 latency vs per-msg launch"
WORKLOAD = "fits_4gib_aes256gcm_enc+dec"
FALLBACK_HBM_GBS = 6800.0
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


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def pipe_bound(nr: int, sms: int, sm_mhz: float):
    """Payload bytes/s at which the shared-memory data pipe (128 bytes per
    clock per SM: 32 conflict-free four-byte lookups) is saturated by the
    table work of AES-GCM counter mode: 16 (Nr - 2) + 5 round-table lookups
    of 4 bytes per block (rounds 1-2 of a counter block depend on the
    counter's low byte through 5 lookups only, the other 27 are per-group
    constants) plus one GHASH multiply by H^32 as 16 lookups of 16 bytes."""
    lookups = 16 * (nr - 2) + 5
    smem_bytes = 4 * lookups + 16 * 16
    blocks_per_s = sms * sm_mhz * 1e6 * 128.0 / smem_bytes
    return blocks_per_s * 16.0, {"round_table_lookups_per_block": lookups, "ghash_lookups_per_block": 16,
                                 "shared_bytes_per_block": smem_bytes,
                                 "wavefronts_per_block": smem_bytes / 128.0, "sms": sms, "sm_mhz": sm_mhz}


def sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    except Exception:
        return 2070.0, "nominal GB300 maximum SM clock"


def strip_c_comments(src):
    """C/C++ source with comments removed and whitespace runs collapsed, so
    that a comment-only edit leaves the code identity unchanged."""
    out = []
    i, n = 0, len(src)
    while i < n:
        c = src[i]
        if c == '"' or c == "'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash():
    """Identity of the fused kernel's code (comments excluded): the files the
    kernel is compiled from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2602_23067_gb300", "csrc")
    for name in ("gcm_kernels.cu", "gcm_device.cuh", "gcm_internal.h"):
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            h.update(strip_c_comments(f.read()).encode())
    return h.hexdigest()


def load_traffic():
    """DRAM bytes per fused-kernel launch from the committed ncu summary, if
    it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "fused_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("source_sha256") == kernel_source_hash():
            return float(d["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


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


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if n_gpus > 1 and world != n_gpus:
        raise SystemExit("--gpus %d needs torchrun with %d processes" % (n_gpus, n_gpus))
    return rank, local, world


def mem_available() -> int:
    """Bytes of host memory available now (/proc/meminfo MemAvailable; 0 if
    unreadable)."""
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return 0


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest of every rank's x (the slowest rank's time); x itself at
    N=1.  `dist` is torch.distributed with an initialised process group."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(world: int, bytes_per_step_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: the bytes all ranks processed / the max-over-ranks
    time (weak scaling: every rank processes the same work)."""
    return world * bytes_per_step_per_rank * steps / seconds / 1e9


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
    peak, peak_kind = load_peaks()
    kern_ms = prof["fused_ms"] / max(1, prof["fused_launches"])
    kern_bytes = prof["fused_bytes"] / max(1, prof["fused_launches"])
    achieved = kern_bytes / (kern_ms * 1e-3) / 1e9
    # Roofline = min(HBM, shared-memory pipe).  Both are expressed in the
    # kernel's algorithmic HBM bytes per second (2 x payload + AAD), so the
    # pipe bound's payload rate is scaled by the same bytes-per-payload ratio.
    mhz, mhz_src = sm_max_mhz()
    pipe_payload, pipe_info = pipe_bound(14, torch.cuda.get_device_properties(local).multi_processor_count, mhz)
    pipe_peak = pipe_payload / 1e9 * kern_bytes / (padded)  # algorithmic bytes per payload byte
    # The pipe bound above is the table engine's; the bitsliced engine is
    # bound by the logic pipe instead and is reported against HBM only.
    bound_is_pipe = pipe_peak < peak and args.aes_impl == "tables"
    rpeak = min(pipe_peak, peak) if bound_is_pipe else peak
    roofline = {
        "bound": "alu" if bound_is_pipe else "hbm",
        "achieved": achieved,
        "peak": rpeak,
        "unit": "GB/s",
        "frac": achieved / rpeak,
        "traffic": load_traffic(),
        "peak_source": ("shared-memory data pipe of the table path (integer S-box and GHASH table lookups), "
                        "derived from %d SMs x %.0f MHz (%s) x 128 B/clk over %.0f shared bytes per block; "
                        "the measured HBM copy peak (%s) is the larger bound"
                        % (pipe_info["sms"], mhz, mhz_src, pipe_info["shared_bytes_per_block"], peak_kind))
        if bound_is_pipe else "%s hbm_gbs (MEASURED_PEAKS.json)" % peak_kind,
        "pipe": dict(pipe_info, peak_gbs_algorithmic=pipe_peak, peak_payload_gbs=pipe_payload / 1e9,
                     frac=achieved / pipe_peak),
        "hbm": {"peak": peak, "frac": achieved / peak,
                "peak_source": "%s hbm_gbs (MEASURED_PEAKS.json)" % peak_kind if peak_kind == "measured"
                else "fallback 6.8 TB/s"},
        "kernel": "fused_kernel<14> (AES-256 CTR + GHASH map)" if args.aes_impl == "tables"
        else "fused_bs_kernel<14> (bitsliced AES-256 CTR + GHASH map)",
        "algorithmic_bytes_per_launch": kern_bytes,
        "avg_launch_ms": kern_ms,
    }

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


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q
    lo = int(k)
    hi = min(lo + 1, len(xs) - 1)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def run_batched(args):
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
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        sample = [(d["key"], d["iv"], d["aad_len"], d["len"], d["seed"]) for d in descs if d["len"] <= (4 << 20)]
        cpu = cpu_oracle_pool(sample[: 2 * (os.cpu_count() or 1)],
                              "the first messages of the same mix no longer than 4 MiB (seeded bytes)")
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


def run_catalog(args):
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
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        # Bounded sample: a 4 MiB prefix of the first files, one file per process.
        cores = os.cpu_count() or 1
        jobs = [(keys[i], ivs[i], 2880, 4 << 20, 5000 + i) for i in range(min(2 * n_pairs, 2 * cores))]
        cpu = cpu_oracle_pool(jobs, "4 MiB prefixes of the first catalog files (seeded bytes), AES-256")
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


def run_small(args):
    """The plain single-message workload: one 1 MiB AES-128-GCM message
    (uniform random bytes, 96-bit IV, 20-byte AAD), encrypt then
    decrypt-verify through gcm_encrypt / gcm_decrypt_verify on device
    buffers.  The timed steps rotate over 256 distinct messages (256 MiB of
    inputs, above the 129 MB L2), so no step reads a warm input; message 0 is
    the seeded message the parity tests use and is checked against the oracle
    first."""
    import numpy as np
    import torch

    import oracle
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

    def step(i):
        ctx.encrypt_device(key, iv, d_aad, pts[i], ct=cts[i], tag=tags[i], stream=stream)
        ctx.decrypt_verify_device(key, iv, d_aad, cts[i], tags[i], pt=backs[i], stream=stream)

    step(0)
    torch.cuda.synchronize()
    ref_ct, ref_tag = oracle.gcm_encrypt(key, iv, aad, pt0)
    if bytes(tags[0].cpu().numpy()) != ref_tag or bytes(cts[0].cpu().numpy()) != ref_ct:
        raise SystemExit("1 MiB message differs from the oracle")
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
    cpu = None
    if not args.no_cpu_baseline:
        t0 = time.perf_counter()
        c, t = oracle.gcm_encrypt(key, iv, aad, pt0)
        ok, _ = oracle.gcm_decrypt(key, iv, aad, c, t)
        dt = time.perf_counter() - t0
        assert ok
        cpu = {"value": 2 * size / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "the whole 1 MiB message 0, encrypt + decrypt-verify, one host thread (%.2f s)" % dt}
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


def ctypes_buf(b: bytes):
    import ctypes

    buf = ctypes.create_string_buffer(b, len(b))
    return ctypes.addressof(buf), buf


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
    ap.add_argument("--workload", choices=["fits4g", "small", "batched", "serving", "catalog"], default="fits4g",
                    help="fits4g (default): one 4 GiB FITS file; batched: 10,000 independent messages; "
                         "serving: Poisson request stream")
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
    if args.workload == "small":
        return run_small(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "catalog":
        return run_catalog(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
