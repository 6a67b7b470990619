"""Parity of the catalog form (streaming FITS files from host memory) at the
workload's file sizes and in its launch configuration: one gcm_batch call
over page-locked host memory holding 4096 x 4096 float32 and int16 data
units (67,109,760 and 33,554,880 bytes) with random 2880-byte headers as
AAD, AES-256, encrypted in place, once with the kernels working on the host
buffers directly and once staged through a ring of 3 device chunk buffers of
256 MiB; then decrypt-verify in place.

Every file is compared whole with the oracle run chunk by chunk on the host
cores (``oracle.mapreduce``): SHA-256 of each 8 MiB of ciphertext and the
tag.  A subset of the 1,366-file catalog: each file is at its full size;
only the number of files is reduced to what the oracle finishes in test
time.
"""
import ctypes

import numpy as np
import pytest

from oracle import mapreduce
from paper_2602_23067_gb300 import workloads

pytestmark = pytest.mark.gpu

FILES = 12
CHUNK = 8 << 20


@pytest.mark.parametrize("host_access", [0, 2])
def test_catalog_files_in_host_memory_against_the_oracle(host_access):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_23067_gb300 import Context, HostBuffer, _native

    sizes = [workloads.padded_len(4096 * 4096 * (4 if i % 2 == 0 else 2)) for i in range(FILES)]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    total = int(offs[-1])
    r = np.random.default_rng(55 + host_access)
    keys = [r.integers(0, 256, 32, dtype=np.uint8).tobytes() for _ in range(FILES)]
    ivs = [r.integers(0, 256, 12, dtype=np.uint8).tobytes() for _ in range(FILES)]
    headers = [np.frombuffer(workloads.fits_header(700 + i, -32 if i % 2 == 0 else 16, [4096, 4096]), np.uint8)
               for i in range(FILES)]
    g = torch.Generator(device="cuda")
    g.manual_seed(56 + host_access)
    with HostBuffer(total) as hb, mapreduce.HostInput(total) as src:
        cat = hb.tensor
        for o in range(0, total, 1 << 30):
            n = min(1 << 30, total - o)
            cat[o:o + n].copy_(torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda", generator=g))
        torch.from_numpy(src.array).copy_(cat)
        spec = [{"key": keys[i], "iv": ivs[i], "aad": headers[i].tobytes(), "off": int(offs[i]), "len": sizes[i]}
                for i in range(FILES)]
        ref = mapreduce.gcm_encrypt_digests(spec, src, chunk_bytes=CHUNK)

        tags = np.zeros((FILES, 16), np.uint8)
        keep = []
        arr = (_native.GcmMsg * FILES)()
        for i in range(FILES):
            kb = ctypes.create_string_buffer(keys[i], 32)
            ib = ctypes.create_string_buffer(ivs[i], 12)
            keep += [kb, ib]
            p = hb.ptr + int(offs[i])
            arr[i] = _native.GcmMsg(ctypes.addressof(kb), 32, ctypes.addressof(ib), 12, headers[i].ctypes.data, 2880,
                                    p, p, sizes[i], tags[i].ctypes.data)
        status = (ctypes.c_int32 * FILES)()
        with Context(0) as ctx:
            ctx.set_host_access(host_access)
            ctx.set_streaming(256 << 20, 3)
            rc = _native.lib.gcm_batch(ctx.handle, arr, FILES, 0, status, 1, None)  # encrypt in place
            assert rc == 0, _native.last_error()
            assert not any(status[i] for i in range(FILES))
            host = cat.numpy()
            for i, (dg, tag) in enumerate(ref):
                assert tags[i].tobytes() == tag, i
                assert mapreduce.digests(host[int(offs[i]): int(offs[i]) + sizes[i]], CHUNK) == dg, i
            rc = _native.lib.gcm_batch(ctx.handle, arr, FILES, 1, status, 1, None)  # decrypt-verify in place
            assert rc == 0, _native.last_error()
            assert not any(status[i] for i in range(FILES))
        assert np.array_equal(cat.numpy(), src.array[:total])
