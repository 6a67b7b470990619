"""Rate microbenchmarks behind the design's bounds (``libgcmprobe.so``).

    python -m paper_2602_23067_gb300.probes [--host-bytes N]

prints one JSON object: integer issue rates per clock per SM (lop3, prmt,
shf, mad.lo, add), shared-memory lookups per clock per SM in the fused
kernel's own addressing (4-byte replicated round tables, 4-byte random
addresses, 16-byte GHASH table), random gathers through the texture and
constant caches (alone, and interleaved with shared-memory lookups, to see
whether the paths add up), the 1-bit tensor-core product rate, and
host-memory rates over the CPU-GPU link.  Each kernel runs one CTA per SM
and counts its own clock cycles, so the per-clock rates do not depend on
the clock frequency.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import sys

from . import build as _build


def _lib():
    L = ctypes.CDLL(_build.build_probes())
    d = ctypes.c_double
    L.probe_alu.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(d)]
    L.probe_lds.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(d)]
    L.probe_gather.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(d)]
    L.probe_mma_b1.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(d)]
    L.probe_shfl.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(d)]
    L.probe_host.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(d)]
    return L


def _call(L, fn, *args):
    out = ctypes.c_double()
    rc = fn(*args, ctypes.byref(out))
    if rc != 0:
        raise RuntimeError("%s failed: %d (line %d)" % (fn.__name__, rc, L.probe_last_error_line()))
    return out.value


def run(host_bytes: int = 4 << 30) -> dict:
    L = _lib()
    res = {"per": "per clock per SM (one CTA per SM, cycles counted by the SM clock)"}
    ops = ["lop3", "prmt", "shf", "mad_lo", "add"]
    res["alu_thread_instructions"] = {
        "%s_%dthreads" % (name, t): _call(L, L.probe_alu, i, t, 4096)
        for i, name in enumerate(ops) for t in (512, 1024)}
    kinds = ["aes_rounds_replicated_tables", "aes_rounds_unreplicated_tables", "lds128_ghash_rotated"]
    res["shared_lookups"] = {
        "%s_%dthreads" % (name, t): _call(L, L.probe_lds, k, t, 2048)
        for k, name in enumerate(kinds) for t in (512, 1024)}
    gk = ["tex1Dfetch_4B", "constant_divergent_4B", "tex_plus_8_lds32", "tex_plus_24_lds32"]
    res["other_gather_paths"] = {
        "%s_%dthreads" % (name, t): _call(L, L.probe_gather, k, t, 1024)
        for k, name in enumerate(gk) for t in (512, 1024)}
    sh = {}
    for mix in (0, 4, 8, 16):
        for t in (512, 1024):
            o = (ctypes.c_double * 2)()
            rc = L.probe_shfl(mix, t, 1024, o)
            if rc != 0:
                raise RuntimeError("probe_shfl failed: %d (line %d)" % (rc, L.probe_last_error_line()))
            sh["mix%d_%dthreads" % (mix, t)] = {"shared_lookups": o[0], "shuffle_lookups": o[1]}
    res["shuffle_sbox_lookups"] = sh
    res["mma_b1_m16n8k256"] = {
        "independent4_512threads": _call(L, L.probe_mma_b1, 4, 512, 256),
        "dependent_512threads": _call(L, L.probe_mma_b1, 1, 512, 256),
        "what": "warp-level mma.sync instructions"}
    out = (ctypes.c_double * 7)()
    rc = L.probe_host(host_bytes, 5, out)
    if rc != 0:
        raise RuntimeError("probe_host failed: %d (line %d)" % (rc, L.probe_last_error_line()))
    res["host_link_gbs"] = {
        "bytes_per_transfer": host_bytes,
        "kernel_read_pinned": out[0], "kernel_write_pinned": out[1],
        "copy_h2d": out[2], "copy_d2h": out[3],
        "copy_both_h2d": out[4], "copy_both_d2h": out[5],
        "kernel_read_pageable": out[6] if out[6] >= 0 else None}
    return res


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--host-bytes", type=int, default=4 << 30)
    args = ap.parse_args(argv)
    print(json.dumps(run(args.host_bytes), indent=1))
    return 0


if __name__ == "__main__":
    sys.exit(main())
