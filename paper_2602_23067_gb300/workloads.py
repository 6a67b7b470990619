"""Seeded synthetic inputs shaped like the paper's FITS workloads.

The paper benchmarks synthetic float32 FITS images with Gaussian pixel values
and WCS-bearing headers (Appendix, "Synthetic Dataset Generation" and the
dataset table).  These generators make inputs of that shape from a seed.  They
hold none of the AES-GCM arithmetic: both the GPU path and the CPU oracle use
them, so that both see the same bytes.
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np

FITS_RECORD = 2880
FITS_CARD = 80


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def random_bytes(seed: int, n: int) -> np.ndarray:
    return rng(seed).integers(0, 256, size=n, dtype=np.uint8)


def padded_len(n: int) -> int:
    """Length of a data unit zero-padded to whole 2880-byte FITS records."""
    return (n + FITS_RECORD - 1) // FITS_RECORD * FITS_RECORD


# ---------------------------------------------------------------------------
# FITS headers
# ---------------------------------------------------------------------------

def _card(key: str, value, comment: str = "") -> bytes:
    if isinstance(value, bool):
        v = "T" if value else "F"
        v = v.rjust(20)
    elif isinstance(value, int):
        v = str(value).rjust(20)
    elif isinstance(value, float):
        v = ("%.10E" % value).rjust(20)
    else:
        v = ("'%s'" % str(value).ljust(8)).ljust(20)
    s = "%-8s= %s" % (key, v)
    if comment:
        s += " / " + comment
    return s[:FITS_CARD].ljust(FITS_CARD).encode("ascii")


def fits_header(seed: int, bitpix: int, naxes: List[int], ncards: int = 36) -> bytes:
    """A primary-HDU header with structural keywords, a synthetic WCS, some
    observation metadata, END, blank padding to whole 2880-byte records.
    ``ncards`` counts every card including END."""
    r = rng(seed)
    cards = [_card("SIMPLE", True, "conforms to FITS standard"),
             _card("BITPIX", bitpix, "array data type"),
             _card("NAXIS", len(naxes), "number of array dimensions")]
    for i, n in enumerate(naxes):
        cards.append(_card("NAXIS%d" % (i + 1), int(n)))
    ra, dec = float(r.uniform(0, 360)), float(r.uniform(-89, 89))
    scale = float(r.uniform(0.2, 1.0)) / 3600.0
    extra = [
        _card("EXTEND", True),
        _card("CTYPE1", "RA---TAN"), _card("CTYPE2", "DEC--TAN"),
        _card("CRVAL1", ra), _card("CRVAL2", dec),
        _card("CRPIX1", float(naxes[0] if naxes else 1) / 2 + 0.5),
        _card("CRPIX2", float(naxes[-1] if naxes else 1) / 2 + 0.5),
        _card("CD1_1", -scale), _card("CD1_2", 0.0), _card("CD2_1", 0.0), _card("CD2_2", scale),
        _card("CUNIT1", "deg"), _card("CUNIT2", "deg"),
        _card("RADESYS", "ICRS"), _card("EQUINOX", 2000.0),
        _card("DATE-OBS", "2026-%02d-%02dT%02d:%02d:%02d" % (int(r.integers(1, 13)), int(r.integers(1, 29)),
                                                             int(r.integers(0, 24)), int(r.integers(0, 60)),
                                                             int(r.integers(0, 60)))),
        _card("EXPTIME", float(r.uniform(10, 600)), "s"),
        _card("TELESCOP", "TTT3"), _card("INSTRUME", "SYNTH"),
        _card("FILTER", ["g", "r", "i", "z"][int(r.integers(0, 4))]),
        _card("GAIN", float(r.uniform(0.8, 2.5))), _card("RDNOISE", float(r.uniform(2, 9))),
        _card("AIRMASS", float(r.uniform(1.0, 2.2))), _card("MAGZPT", float(r.uniform(24, 27))),
        _card("BUNIT", "ADU"), _card("OBJECT", "FIELD%04d" % int(r.integers(0, 10000))),
        _card("OBSERVER", "SYNTH"), _card("SEEING", float(r.uniform(0.6, 2.5)), "arcsec"),
        _card("PROPID", "P%05d" % int(r.integers(0, 99999))),
    ]
    i = 0
    while len(cards) < ncards - 1:
        cards.append(extra[i] if i < len(extra) else ("COMMENT   synthetic padding card").ljust(FITS_CARD).encode("ascii"))
        i += 1
    cards = cards[: ncards - 1]
    cards.append(b"END".ljust(FITS_CARD))
    hdr = b"".join(cards)
    hdr += b" " * ((-len(hdr)) % FITS_RECORD)
    return hdr


# ---------------------------------------------------------------------------
# Pixel data
# ---------------------------------------------------------------------------

def sky_image_host(seed: int, n1: int, n2: int, bitpix: int = -32, background: float = 1000.0,
                   sigma: float = 50.0, n_sources: int = 200) -> np.ndarray:
    """A small sky image (host, numpy): Gaussian background plus Poisson point
    sources with Gaussian PSFs, returned as big-endian FITS bytes."""
    r = rng(seed)
    img = r.normal(background, sigma, size=(n2, n1)).astype(np.float64)
    for _ in range(n_sources):
        x, y = r.uniform(0, n1), r.uniform(0, n2)
        flux = float(r.poisson(float(r.uniform(2e3, 2e5))))
        fwhm = float(r.uniform(3, 7))
        s = fwhm / 2.3548
        x0, x1 = max(0, int(x - 4 * s)), min(n1, int(x + 4 * s) + 1)
        y0, y1 = max(0, int(y - 4 * s)), min(n2, int(y + 4 * s) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1]
        img[y0:y1, x0:x1] += flux / (2 * math.pi * s * s) * np.exp(-((xx - x) ** 2 + (yy - y) ** 2) / (2 * s * s))
    if bitpix == -32:
        arr = img.astype(">f4")
    elif bitpix == 16:
        arr = np.clip(np.round(img - 32768.0 + 1000.0), -32768, 32767).astype(">i2")
    else:
        raise ValueError("unsupported BITPIX")
    return np.frombuffer(arr.tobytes(), dtype=np.uint8)


def sky_image_device(seed: int, n1: int, n2: int, device="cuda", background: float = 1000.0,
                     sigma: float = 50.0, n_sources: int = 10000, out=None):
    """A large float32 sky image generated on the GPU with torch (so that a
    4 GiB image never crosses the host link): N(background, sigma^2) plus
    ``n_sources`` Poisson point sources with Gaussian PSFs (FWHM 3-7 px),
    stored big-endian as FITS requires.  Returns a uint8 tensor of
    n1*n2*4 bytes (or fills ``out``, which may be longer; the tail is
    zeroed, i.e. the data unit is zero-padded)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    npix = n1 * n2
    nbytes = npix * 4
    if out is None:
        out = torch.empty(nbytes, dtype=torch.uint8, device=device)
    f = out[:nbytes].view(torch.float32)
    rows_per = max(1, (1 << 26) // n1)
    for r0 in range(0, n2, rows_per):
        r1 = min(n2, r0 + rows_per)
        blk = f[r0 * n1: r1 * n1]
        blk.normal_(background, sigma, generator=g)
    # Point sources: small Gaussian stamps added with index_add_.
    hs = 10
    ax = torch.arange(-hs, hs + 1, device=device, dtype=torch.float32)
    cx = torch.rand(n_sources, generator=g, device=device) * (n1 - 2 * hs - 2) + hs + 1
    cy = torch.rand(n_sources, generator=g, device=device) * (n2 - 2 * hs - 2) + hs + 1
    lam = torch.rand(n_sources, generator=g, device=device) * (2e5 - 2e3) + 2e3
    flux = torch.poisson(lam, generator=g)
    fwhm = torch.rand(n_sources, generator=g, device=device) * 4 + 3
    s = fwhm / 2.3548
    ix = cx.floor().long()
    iy = cy.floor().long()
    dx = (ix[:, None].float() + ax[None, :]) - cx[:, None]
    dy = (iy[:, None].float() + ax[None, :]) - cy[:, None]
    gx = torch.exp(-dx * dx / (2 * s[:, None] ** 2))
    gy = torch.exp(-dy * dy / (2 * s[:, None] ** 2))
    stamp = (flux / (2 * math.pi * s * s))[:, None, None] * gy[:, :, None] * gx[:, None, :]
    offs = torch.arange(-hs, hs + 1, device=device)
    idx = (iy[:, None, None] + offs[None, :, None]) * n1 + (ix[:, None, None] + offs[None, None, :])
    f.index_add_(0, idx.reshape(-1), stamp.reshape(-1))
    # float32 -> big-endian bytes, in place, chunk by chunk.
    b = out[:nbytes].view(-1, 4)
    step = 1 << 26
    for i in range(0, b.shape[0], step):
        b[i: i + step] = b[i: i + step].flip(1)
    if out.numel() > nbytes:
        out[nbytes:].zero_()
    return out


def fits_file_host(seed: int, n1: int, n2: int, bitpix: int = -32, ncards: int = 36,
                   n_sources: int = 50) -> bytes:
    """A complete small single-HDU FITS file (header + zero-padded data unit)."""
    hdr = fits_header(seed, bitpix, [n1, n2], ncards)
    data = sky_image_host(seed + 1, n1, n2, bitpix, n_sources=n_sources).tobytes()
    data += bytes(padded_len(len(data)) - len(data))
    return hdr + data


# ---------------------------------------------------------------------------
# Message mixes for the batched and served forms
# ---------------------------------------------------------------------------

def message_mix(seed: int, count: int, median: int = 2 << 20, sigma: float = 1.0, lo: int = 16,
                hi: int = 64 << 20, frac_unaligned: float = 0.3, frac_long_iv: float = 0.05,
                aad_max: int = 4096, key_sizes=(16, 32)) -> List[Dict]:
    """Descriptors of independent messages: lognormal lengths (median, sigma)
    clipped to [lo, hi], ~frac_unaligned of them not a multiple of 16, keys of
    mixed sizes, 96-bit IVs except ~frac_long_iv with 8..128-byte IVs, AAD of
    0..aad_max bytes.  Payload bytes are not materialised here."""
    r = rng(seed)
    out = []
    for i in range(count):
        n = int(np.clip(r.lognormal(math.log(median), sigma), lo, hi))
        if r.random() < frac_unaligned:
            if n % 16 == 0:
                n += int(r.integers(1, 16)) if n + 16 <= hi else -int(r.integers(1, 16))
        else:
            n = max(16, n - n % 16)
        key_len = int(key_sizes[int(r.integers(0, len(key_sizes)))])
        if r.random() < frac_long_iv:
            iv_len = int(r.integers(8, 129))
            if iv_len == 12:
                iv_len = 13
        else:
            iv_len = 12
        out.append({
            "len": n,
            "key": r.integers(0, 256, size=key_len, dtype=np.uint8).tobytes(),
            "iv": r.integers(0, 256, size=iv_len, dtype=np.uint8).tobytes(),
            "aad_len": int(r.integers(0, aad_max + 1)),
            "seed": int(r.integers(0, 2 ** 31 - 1)),
        })
    return out
