"""The C-ABI library builds, loads and exports every function include/ocm.h
declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

import paper_1111_0627_gb300 as ocm
from paper_1111_0627_gb300 import _native

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "ocm.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ocm_[a-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("ocm_solve", "ocm_backward", "ocm_workspace_size", "ocm_status_string",
                     "ocm_version"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_native.build())
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in _native.SIGNATURES, f"binding lacks {name}"


def test_host_only_entry_points():
    lib = ocm.load()
    assert lib.ocm_version() == 112
    assert lib.ocm_workspace_size(0, 5) == 0
    assert lib.ocm_workspace_size(5, 0) == 0
    small = lib.ocm_workspace_size(1000, 4000)
    big = lib.ocm_workspace_size(2000, 4000)
    assert small > 0 and big > small and small % 256 == 0
    single = lib.ocm_workspace_size_single(1000, 4000)
    assert single % 256 == 0 and 4 * 4000 + 20 * 1000 <= single - small <= 4 * 4000 + 20 * 1000 + 4096
    assert lib.ocm_workspace_size_single(0, 5) == 0
    assert lib.ocm_status_string(0) == b"ok"
    for code in range(-9, 0):
        assert lib.ocm_status_string(code) != b"unknown status"


def test_argument_errors_are_reported_before_any_device_work():
    lib = ocm.load()
    num, den, clen = ctypes.c_int64(0), ctypes.c_int32(0), ctypes.c_int32(0)
    # null CSR pointers
    rc = lib.ocm_solve(None, None, None, 4, 4, 0, ctypes.byref(num), ctypes.byref(den), None,
                       ctypes.byref(clen), None, 0, None, None, None)
    assert rc == -1
    fake = ctypes.c_void_p(256)   # never dereferenced: the size checks fail first
    rc = lib.ocm_solve(fake, fake, fake, 4, 4, 7, ctypes.byref(num), ctypes.byref(den), fake,
                       ctypes.byref(clen), fake, 10**9, None, None, None)
    assert rc == -1                                      # bad mode
    rc = lib.ocm_solve(fake, fake, fake, 4, 4, 0, ctypes.byref(num), ctypes.byref(den), fake,
                       ctypes.byref(clen), fake, 16, None, None, None)
    assert rc == -7                                      # workspace too small
    rc = lib.ocm_solve(fake, fake, fake, 4, 4, 0, ctypes.byref(num), ctypes.byref(den), fake,
                       ctypes.byref(clen), ctypes.c_void_p(256 + 8), 10**9, None, None, None)
    assert rc == -7                                      # workspace misaligned
    opt = _native.OcmOptions()
    opt.flags = 1024                                     # no such flag
    rc = lib.ocm_solve(fake, fake, fake, 4, 4, 0, ctypes.byref(num), ctypes.byref(den), fake,
                       ctypes.byref(clen), fake, 10**9, None, ctypes.byref(opt), None)
    assert rc == -1
    opt.flags = 256 | 512                                # chunks forced on and off at once
    rc = lib.ocm_solve(fake, fake, fake, 4, 4, 0, ctypes.byref(num), ctypes.byref(den), fake,
                       ctypes.byref(clen), fake, 10**9, None, ctypes.byref(opt), None)
    assert rc == -1
    opt.flags = 8 | 16                                   # both evaluation forms at once
    rc = lib.ocm_solve(fake, fake, fake, 4, 4, 0, ctypes.byref(num), ctypes.byref(den), fake,
                       ctypes.byref(clen), fake, 10**9, None, ctypes.byref(opt), None)
    assert rc == -1
    opt.flags = 4                                        # single lambda: larger workspace
    rc = lib.ocm_solve(fake, fake, fake, 4, 4, 0, ctypes.byref(num), ctypes.byref(den), fake,
                       ctypes.byref(clen), fake, lib.ocm_workspace_size(4, 4), None,
                       ctypes.byref(opt), None)
    assert rc == -7
    clen_g = ctypes.c_void_p(256)
    rc = lib.ocm_solve_batch(fake, fake, fake, fake, 1, 4, 4, 0, fake, fake, clen_g, fake, fake,
                             10**9, None, ctypes.byref(opt), None)
    assert rc == -1                                      # single lambda: not for batches
    opt.flags = 0
    opt.sweep_kind = 7                                   # no such sweep layout
    rc = lib.ocm_solve(fake, fake, fake, 4, 4, 0, ctypes.byref(num), ctypes.byref(den), fake,
                       ctypes.byref(clen), fake, 10**9, None, ctypes.byref(opt), None)
    assert rc == -1
    rc = lib.ocm_backward(fake, 0, fake, 4, fake, None)
    assert rc == -1
    rc = lib.ocm_backward_ratio(fake, 0, fake, fake, 4, fake, None)   # empty cycle
    assert rc == -1
    rc = lib.ocm_backward_ratio(fake, 2, None, fake, 4, fake, None)   # no transit times
    assert rc == -1


def test_no_cpu_fallback_in_the_package():
    """The product package never imports the oracle or a CPU solver."""
    pkg = os.path.dirname(ocm.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                text = open(os.path.join(root, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


@pytest.fixture
def fault_env():
    old = os.environ.get("OCM_FAULT")
    yield os.environ
    if old is None:
        os.environ.pop("OCM_FAULT", None)
    else:
        os.environ["OCM_FAULT"] = old


def _host_csr_call(lib, fn_name):
    """Calls an entry point with valid sizes and 256-byte aligned host
    addresses: with OCM_FAULT set it must return before any device work, so
    the addresses are never dereferenced (no GPU is needed)."""
    import numpy as np
    n, m = 8, 16
    buf = np.zeros(1 << 20, np.uint8)
    base = (buf.ctypes.data + 255) // 256 * 256
    num, den, clen = ctypes.c_int64(0), ctypes.c_int32(0), ctypes.c_int32(0)
    if fn_name == "ocm_solve":
        ws = lib.ocm_workspace_size(n, m)
        return lib.ocm_solve(base, base, base, n, m, 0, ctypes.byref(num), ctypes.byref(den),
                             base, ctypes.byref(clen), base, ws, None, None, None), (num, den)
    if fn_name == "ocm_solve_batch":
        ws = lib.ocm_workspace_size_batch(2, n, m)
        return lib.ocm_solve_batch(base, base, base, base, 2, n, m, 0, base, base, base, base,
                                   base, ws, None, None, None), (num, den)
    if fn_name == "ocm_scc":
        cnt = ctypes.c_int32(-1)
        ws = lib.ocm_workspace_size_scc(n, m)
        return lib.ocm_scc(base, base, n, m, base, ctypes.byref(cnt), base, ws, None), (cnt, den)
    raise ValueError(fn_name)


@pytest.mark.parametrize("fn_name", ["ocm_solve", "ocm_solve_batch", "ocm_scc"])
def test_injected_launch_failure_returns_cuda_error_without_device_work(fault_env, fn_name):
    lib = ocm.load()
    fault_env["OCM_FAULT"] = "launch"
    rc, (a, b) = _host_csr_call(lib, fn_name)
    assert rc == -8                                  # OCM_ERR_CUDA
    assert lib.ocm_status_string(rc) == b"CUDA runtime error"
    assert a.value in (0, -1) and b.value == 0       # outputs untouched


@pytest.mark.parametrize("fn_name", ["ocm_solve", "ocm_solve_batch"])
def test_injected_validation_failure_returns_bad_csr(fault_env, fn_name):
    lib = ocm.load()
    fault_env["OCM_FAULT"] = "validate"
    rc, (num, den) = _host_csr_call(lib, fn_name)
    assert rc == -2                                  # OCM_ERR_BAD_CSR
    assert (num.value, den.value) == (0, 0)


def test_python_layer_maps_injected_failures_to_ocm_error(fault_env):
    """ocm.OCMError carries the status and its text (the Python layer adds no
    recovery of its own)."""
    err = ocm.OCMError(-8, "ocm_solve")
    assert err.status == -8 and "CUDA" in str(err)
