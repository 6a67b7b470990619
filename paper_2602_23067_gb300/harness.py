"""Measurement plumbing shared by the benchmark workloads: peaks, kernel
identity, clock sampling during a timed region, multi-rank timing.

Nothing here computes or checks AES-GCM; the workloads time the library's
own calls and the benchmark adds the CPU baselines.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import threading

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FALLBACK_HBM_GBS = 6800.0


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


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


def load_pipe_counters():
    """Per 16-byte block of the fused kernel, from the committed capture if it
    was taken on the current kernel source (else None): shared-memory (LSU)
    data-pipe wavefronts (ncu l1tex__data_pipe_lsu_wavefronts_mem_shared) and
    warp instructions (smsp__inst_executed), each over the blocks of one
    launch, with the capture's command."""
    p = os.path.join(ROOT, "profiles", "fused_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("source_sha256") == kernel_source_hash() and d.get("lsu_wavefronts_per_block"):
            wi = d.get("warp_instructions_per_block")
            return {"wavefronts": float(d["lsu_wavefronts_per_block"]),
                    "warp_instructions": float(wi) if wi else None, "command": d.get("command", "")}
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


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q
    lo = int(k)
    hi = min(lo + 1, len(xs) - 1)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def ctypes_buf(b: bytes):
    import ctypes

    buf = ctypes.create_string_buffer(b, len(b))
    return ctypes.addressof(buf), buf
