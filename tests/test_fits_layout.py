"""FITS header parsing of the C ABI (gfc_fits_layout), checked on the CPU
against the oracle's FITS split -- no GPU needed."""
import pytest

import oracle
from paper_2602_23067_gb300 import workloads


@pytest.fixture(scope="module")
def native():
    from paper_2602_23067_gb300 import build

    build.build()
    from paper_2602_23067_gb300 import _native

    return _native


@pytest.mark.parametrize("n1,n2,bitpix,ncards", [(100, 60, -32, 36), (17, 3, 16, 36), (48, 48, -32, 40),
                                                 (2048, 2, -32, 80), (1, 1, 16, 36)])
def test_layout_matches_oracle_split(native, n1, n2, bitpix, ncards):
    hdr = workloads.fits_header(3, bitpix, [n1, n2], ncards=ncards)
    data = workloads.sky_image_host(4, n1, n2, bitpix, n_sources=1).tobytes()
    f = hdr + data + bytes(workloads.padded_len(len(data)) - len(data))
    L = native.gfc_fits_layout(f)
    header, padded, nbytes = oracle.fits_split(f)
    assert L.header_bytes == len(header)
    assert L.data_bytes == nbytes
    assert L.data_padded_bytes == len(padded)
    assert L.bitpix == bitpix and L.naxis == 2
    assert list(L.naxes[:2]) == [n1, n2]


def test_layout_rejects_non_fits(native):
    with pytest.raises(native.GcmError) as e:
        native.gfc_fits_layout(b"x" * 2880)
    assert e.value.code == native.GCM_ERR_INVALID_ARG
    hdr = workloads.fits_header(3, -32, [4, 4]).replace(b"END     ", b"XND     ")
    with pytest.raises(native.GcmError):
        native.gfc_fits_layout(hdr)
    bad = workloads.fits_header(3, -32, [4, 4]).replace(b"BITPIX  =                  -32",
                                                        b"BITPIX  =                  -31")
    with pytest.raises(native.GcmError):
        native.gfc_fits_layout(bad)


def test_header_only_file(native):
    hdr = workloads.fits_header(5, 8, [], ncards=10)
    L = native.gfc_fits_layout(hdr)
    assert L.naxis == 0 and L.data_bytes == 0 and L.data_padded_bytes == 0
    assert L.header_bytes == 2880
