"""The C ABI library loads and exports every function include/*.h declares
(no GPU needed: nothing here launches work)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^\s*(?:const\s+)?(?:int|void|char|size_t|int32_t|uint32_t|uint64_t|gcm_status)\s*\**\s*(g(?:cm|fc)_\w+)\s*\(",
                  re.M)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        with open(h) as f:
            names.update(DECL.findall(f.read()))
    return sorted(names)


@pytest.fixture(scope="module")
def native():
    from paper_2602_23067_gb300 import build

    build.build()
    from paper_2602_23067_gb300 import _native

    return _native


def test_header_declares_the_core_calls():
    names = declared_functions()
    for n in ("gcm_ctx_create", "gcm_ctx_destroy", "gcm_encrypt", "gcm_decrypt_verify", "gcm_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(native):
    for name in declared_functions():
        assert hasattr(native.lib, name), name


def test_binding_covers_every_declared_symbol(native):
    assert set(declared_functions()) <= set(native.SIGNATURES)


def test_only_abi_symbols_are_exported(native):
    out = subprocess.run(["nm", "-D", "--defined-only", native.LIB_PATH], capture_output=True, text=True).stdout
    syms = [ln.split()[-1] for ln in out.splitlines() if ln.strip()]
    exported = [s for s in syms if not s.startswith("_") and s not in ("_init", "_fini")]
    assert exported, out
    for s in exported:
        assert s.startswith("gcm_") or s.startswith("gfc_"), s
    assert not any("oracle" in s for s in syms)


def test_errors_without_a_device_are_reported_not_raised(native):
    # Argument checks run before any CUDA call.
    import ctypes

    rc = native.lib.gcm_encrypt(None, None, 16, None, 12, None, 0, None, 0, None, None, 0, None)
    assert rc == native.GCM_ERR_INVALID_ARG
    assert "NULL" in native.last_error()


def test_host_alloc_argument_errors(native):
    # gcm_host_alloc checks its arguments before any CUDA call.
    import ctypes

    out = ctypes.c_void_p(1)
    assert native.lib.gcm_host_alloc(0, 0, ctypes.byref(out)) == native.GCM_ERR_INVALID_ARG
    assert out.value is None
    assert native.lib.gcm_host_alloc(0, 16, None) == native.GCM_ERR_INVALID_ARG
    assert native.lib.gcm_host_free(None) == native.GCM_OK


def test_server_admission_argument_errors(native):
    # gcm_server_admission checks its server argument before anything else.
    import ctypes

    b, peak, waits = ctypes.c_size_t(7), ctypes.c_size_t(7), ctypes.c_uint64(7)
    rc = native.lib.gcm_server_admission(None, ctypes.byref(b), ctypes.byref(peak), ctypes.byref(waits))
    assert rc == native.GCM_ERR_INVALID_ARG
    assert (b.value, peak.value, waits.value) == (7, 7, 7)


def build_c_consumer(out_dir):
    """Compiles tests/abi_consumer.c (C99, warnings as errors) against the
    header and links it to the library; returns the executable's path."""
    lib_dir = os.path.join(ROOT, "paper_2602_23067_gb300")
    exe = os.path.join(out_dir, "abi_consumer")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "abi_consumer.c"), "-o", exe, "-L", lib_dir, "-lgcmgpu",
           "-Wl,-rpath," + lib_dir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_header_is_plain_c_and_links(native, tmp_path):
    # The boundary needs no C++ and no Python: a C99 program that includes
    # the header compiles without warnings and links against the library.
    assert os.path.exists(build_c_consumer(str(tmp_path)))


def test_batch_plan_argument_errors(native):
    # The plan calls check their handles before any CUDA call.
    import ctypes

    out = ctypes.c_void_p(1)
    msg = native.GcmMsg()
    rc = native.lib.gcm_batch_plan_create(None, ctypes.byref(msg), 1, 0, ctypes.byref(out))
    assert rc == native.GCM_ERR_INVALID_ARG
    assert out.value is None
    assert native.lib.gcm_batch_plan_create(None, ctypes.byref(msg), 1, 0, None) == native.GCM_ERR_INVALID_ARG
    assert native.lib.gcm_batch_plan_set(None, 0, ctypes.byref(msg), 1) == native.GCM_ERR_INVALID_ARG
    assert native.lib.gcm_batch_plan_launch(None, None) == native.GCM_ERR_INVALID_ARG
    assert native.lib.gcm_batch_plan_wait(None, None) == native.GCM_ERR_INVALID_ARG
    native.lib.gcm_batch_plan_destroy(None)


def test_batch_plan_binding_takes_device_tensors_only(native):
    # The binding refuses host buffers before it calls the library (a plan
    # is a device-memory batch).
    torch = pytest.importorskip("torch")
    from paper_2602_23067_gb300.api import BatchPlan

    host = torch.zeros(32, dtype=torch.uint8)
    msg = {"key": bytes(16), "iv": bytes(12), "aad": None, "inp": host, "out": host,
           "tag": torch.zeros(16, dtype=torch.uint8)}
    with pytest.raises(ValueError):
        BatchPlan(None, [msg], False)
