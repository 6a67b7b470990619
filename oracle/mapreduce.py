"""GCM of messages too large for one host thread: the oracle's own
definitions applied chunk by chunk on many host cores.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only the test suite
may use this module; the product path never imports it.

A message's payload is cut into chunks of whole 16-byte blocks.  For the
chunk that starts at payload block b:

* its ciphertext is GCTR_K(inc_32^(b+1)(J0), P_chunk) -- Algorithm 3 of
  SP 800-38D started at that block's counter (counter blocks are independent
  of one another, and block j of the payload always uses inc_32^(j+1)(J0));
* its GHASH partial is the serial GHASH_H (Algorithm 2, the paper's Eq. 1)
  over its ciphertext blocks, the last one zero-padded: the sum of
  C_j * H^(m-j+1) over its m blocks, i.e. one partial of the map phase of
  the paper's two-phase GHASH (Sec. 5.2.2);
* the worker returns the SHA-256 digest of the chunk's ciphertext and the
  partial, 48 bytes in all.

The parent joins the partials left to right with
Combine(L, R) = L * H^(#blocks of R) xor R (``oracle.combine``, the paper's
tree step, Fig. 3b), starting from the partial of the zero-padded AAD, then
joins the length block [len(A)]_64 || [len(C)]_64 (one block), and the tag
is E_K(J0) xor that value (Algorithm 4 steps 5-6).  Every bracketing of the
joins gives the same field element; the pins in the test suite check this
module against ``oracle.gcm_encrypt`` (the serial definition) on small
messages cut at many chunk sizes.

Inputs reach the worker processes through a file that they map read-only
(``HostInput``), so a multi-GiB payload is written once and never pickled.
Workers are started with the ``spawn`` method, which is safe after the
parent has initialised CUDA.
"""
from __future__ import annotations

import concurrent.futures
import hashlib
import multiprocessing
import os
import tempfile
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

import oracle


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover - not Linux
        return os.cpu_count() or 1


class HostInput:
    """A byte array in a file (in /dev/shm when it has room, else in the
    temporary directory) that worker processes map read-only.  ``array`` is
    the parent's writable view."""

    def __init__(self, nbytes: int):
        d = None
        for cand in ("/dev/shm", tempfile.gettempdir()):
            try:
                st = os.statvfs(cand)
            except OSError:
                continue
            if os.access(cand, os.W_OK) and st.f_bavail * st.f_frsize >= int(nbytes) + (1 << 30):
                d = cand
                break
        if d is None:
            raise MemoryError("no file system with room for %d bytes of oracle input" % nbytes)
        fd, self.path = tempfile.mkstemp(prefix="gcm_oracle_input_", suffix=".bin", dir=d)
        os.close(fd)
        self.nbytes = int(nbytes)
        with open(self.path, "r+b") as f:
            f.truncate(max(1, self.nbytes))
        self.array = np.memmap(self.path, dtype=np.uint8, mode="r+", shape=(max(1, self.nbytes),))

    def close(self) -> None:
        if self.array is not None:
            self.array.flush()
            del self.array
            self.array = None
        try:
            os.unlink(self.path)
        except FileNotFoundError:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _chunk_job(args) -> Tuple[bytes, bytes]:
    """Worker: ciphertext digest and GHASH partial of one payload chunk (and
    the chunk's ciphertext written to the output file, when one is given)."""
    path, total, off, n, key, icb, h, dest = args
    src = np.memmap(path, dtype=np.uint8, mode="r", shape=(total,))[off: off + n]
    src = np.ascontiguousarray(src)  # one read of the chunk into this process
    ct = np.empty(n + (-n) % 16, dtype=np.uint8)
    ct[n:] = 0  # zero pad of a final partial block (GHASH input only)
    oracle.gctr_ptr(key, icb, src.ctypes.data, n, ct.ctypes.data)
    partial = oracle.ghash_ptr(h, ct.ctypes.data, ct.size // 16)
    if dest is not None:
        out = np.memmap(dest, dtype=np.uint8, mode="r+", shape=(total,))
        out[off: off + n] = ct[:n]
        out.flush()
        del out
    return hashlib.sha256(ct[:n].data).digest(), partial


def chunk_bounds(length: int, chunk_bytes: int) -> List[Tuple[int, int]]:
    """Byte ranges [a, b) of the chunks of a payload of ``length`` bytes;
    every chunk but the last has ``chunk_bytes`` bytes (a multiple of 16)."""
    if chunk_bytes <= 0 or chunk_bytes % 16:
        raise ValueError("chunk_bytes must be a positive multiple of 16")
    return [(a, min(length, a + chunk_bytes)) for a in range(0, length, chunk_bytes)]


def digests(data, chunk_bytes: int) -> List[bytes]:
    """SHA-256 of each chunk of ``data`` (any buffer), cut as ``chunk_bounds``
    cuts: how a ciphertext computed elsewhere is compared with this oracle."""
    mv = memoryview(data).cast("B")
    return [hashlib.sha256(mv[a:b]).digest() for a, b in chunk_bounds(len(mv), chunk_bytes)]


def _finish(key: bytes, iv: bytes, aad: bytes, length: int, parts: Sequence[Tuple[int, bytes]]) -> bytes:
    """Tag from the chunk partials (blocks, partial) in payload order."""
    h, _, ej0 = oracle.h_j0(key, iv)
    g = oracle.ghash(h, aad + bytes((-len(aad)) % 16)) if aad else oracle.ZERO
    for blocks, p in parts:
        g = oracle.combine(h, g, p, blocks)
    lb = (8 * len(aad)).to_bytes(8, "big") + (8 * length).to_bytes(8, "big")
    g = oracle.combine(h, g, oracle.ghash(h, lb), 1)
    return oracle.xor16(ej0, g)


def gcm_encrypt_digests(messages: Sequence[Dict], source: HostInput, chunk_bytes: int = 64 << 20,
                        workers: Optional[int] = None,
                        dest: Optional[HostInput] = None) -> List[Tuple[List[bytes], bytes]]:
    """GCM-AE of each message, computed chunk by chunk on ``workers`` processes.

    Each message is a dict with ``key``, ``iv``, ``aad`` (bytes) and ``off``,
    ``len``: its plaintext is ``source.array[off:off + len]``.  Returns, per
    message, (SHA-256 digests of its ciphertext cut by ``chunk_bounds``, tag).
    With ``dest`` (a HostInput of the same size), the ciphertext itself is
    also written to ``dest.array[off:off + len]``."""
    source.array.flush()
    if dest is not None:
        if dest.nbytes != source.nbytes:
            raise ValueError("dest must have the size of source")
        dest.array.flush()
    jobs: List = []
    owner: List[List[Tuple[int, int]]] = [[] for _ in messages]  # per message: (job index, blocks)
    for mi, m in enumerate(messages):
        h, j0, _ = oracle.h_j0(m["key"], m["iv"])
        for a, b in chunk_bounds(int(m["len"]), chunk_bytes):
            icb = oracle.counter_block(j0, a // 16 + 1)
            jobs.append((source.path, max(1, source.nbytes), int(m["off"]) + a, b - a, m["key"], icb, h,
                         dest.path if dest is not None else None))
            owner[mi].append((len(jobs) - 1, (b - a + 15) // 16))
    results: List = [None] * len(jobs)
    if jobs:
        nproc = max(1, min(workers or host_cores(), len(jobs)))
        if nproc == 1:
            results = [_chunk_job(j) for j in jobs]
        else:
            ctx = multiprocessing.get_context("spawn")
            with concurrent.futures.ProcessPoolExecutor(max_workers=nproc, mp_context=ctx) as ex:
                results = list(ex.map(_chunk_job, jobs, chunksize=1))
    out = []
    for mi, m in enumerate(messages):
        mine = [(nb, results[k]) for k, nb in owner[mi]]
        tag = _finish(m["key"], m["iv"], m["aad"], int(m["len"]), [(nb, r[1]) for nb, r in mine])
        out.append(([r[0] for _, r in mine], tag))
    return out
