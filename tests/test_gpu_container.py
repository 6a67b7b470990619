"""The dual-key container through the C ABI (gfc_container_encrypt,
gfc_decrypt_frame) against the oracle's container, byte for byte, in the
paper's four access scenarios plus tampering (Sec. 3.2.2, Sec. 4.2)."""
import numpy as np
import pytest

import oracle
from oracle import container as C
from paper_2602_23067_gb300 import workloads

pytestmark = pytest.mark.gpu

KH, KD = bytes(range(16)), bytes(range(100, 132))
NH, ND = bytes(range(12)), bytes(range(50, 62))


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_23067_gb300 import Context

    ctx = Context(0)
    yield torch, ctx
    ctx.close()


def _file(seed, n1, n2, bitpix=-32, pad=True):
    hdr = workloads.fits_header(seed, bitpix, [n1, n2], ncards=36)
    data = workloads.sky_image_host(seed + 1, n1, n2, bitpix, n_sources=5).tobytes()
    if pad:
        data += bytes(workloads.padded_len(len(data)) - len(data))
    return hdr + data


def _as(torch, where, b):
    if where == "device":
        return torch.frombuffer(bytearray(b), dtype=torch.uint8).cuda()
    return np.frombuffer(b, dtype=np.uint8).copy()


def _bytes(where, t):
    return bytes(t.cpu().numpy()) if where == "device" else t.tobytes()


@pytest.mark.parametrize("where", ["device", "host"])
@pytest.mark.parametrize("shape", [(256, 256, -32), (77, 13, 16), (1024, 700, -32)])
def test_container_matches_oracle(env, where, shape):
    torch, ctx = env
    f = _file(20, *shape)
    ref = C.container_encrypt(KH, KD, NH, ND, f)
    r = ctx.container_encrypt(KH, KD, _as(torch, where, f), nonce_h=NH, nonce_d=ND)
    got = _bytes(where, r.data)
    assert got == ref
    _, off = C.parse_header(ref, 0)
    x, doff = C.parse_header(ref, off)
    assert r.datasum == int(x["DATASUM"])


@pytest.mark.parametrize("where", ["device", "host"])
def test_access_scenarios(env, where):
    torch, ctx = env
    f = _file(21, 300, 200)
    cont = C.container_encrypt(KH, KD, NH, ND, f)
    cases = [(KH, KD), (KH, None), (None, KD), (None, None), (bytes(16), KD), (KH, bytes(32))]
    for kh, kd in cases:
        want, wwarn = C.decrypt_frame(cont, kh, kd)
        d = ctx.decrypt_frame(_as(torch, where, cont), kh, kd)
        assert d.error_code == 0 and d.warning_code == wwarn, (kh, kd)
        assert _bytes(where, d.data) == want, (kh, kd)
    assert ctx.decrypt_frame(_as(torch, where, cont), KH, KD).data is not None


def test_tampering(env):
    torch, ctx = env
    f = _file(22, 128, 128)
    cont = C.container_encrypt(KH, KD, NH, ND, f)
    _, off = C.parse_header(cont, 0)
    _, doff = C.parse_header(cont, off)
    variants = []
    t = bytearray(cont)
    t[doff + 5] ^= 1
    variants.append(bytes(t))  # pixel blob
    variants.append(cont.replace(b"ORIG_NA2=                  128", b"ORIG_NA2=                  127"))
    i = cont.index(b"ENCHDR  = '") + 11
    t = bytearray(cont)
    t[i] = ord("0") if t[i] != ord("0") else ord("1")
    variants.append(bytes(t))  # encrypted header
    for v in variants:
        assert v != cont
        want, wwarn = C.decrypt_frame(v, KH, KD)
        d = ctx.decrypt_frame(_as(torch, "device", v), KH, KD)
        assert d.warning_code == wwarn and bytes(d.data.cpu().numpy()) == want
