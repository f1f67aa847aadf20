"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/*.h declares. No GPU needed (no compute call is made)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"DPSR_API\s+[\w\s\*]*?\b(dpsr_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2106_03452_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_boundary():
    names = _declared()
    for must in ("dpsr_plan_create", "dpsr_forward", "dpsr_backward", "dpsr_plan_destroy",
                 "dpsr_sync", "dpsr_strerror", "dpsr_plan_workspace_bytes"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2106_03452_gb300 import libdpsr
    for n in _declared():
        assert n in libdpsr._PROTOS, n
        assert hasattr(libdpsr, n), n


def test_host_only_calls(lib):
    from paper_2106_03452_gb300 import libdpsr as L
    assert L.dpsr_strerror(L.DPSR_EDEGENERATE).startswith("degenerate")
    assert L.dpsr_strerror(12345) == "unknown status"
    assert L.dpsr_plan_workspace_bytes(12, 100) == 0          # r not a power of two
    assert L.dpsr_plan_workspace_bytes(1024, 100) == 0        # above the maximum size
    assert L.dpsr_plan_workspace_bytes(512, 100) > 6 * 8 * 512 * 512 * 257   # six half spectra
    b128 = L.dpsr_plan_workspace_bytes(128, 20000)
    b256 = L.dpsr_plan_workspace_bytes(256, 100000)
    assert 4 * 128 * 128 * 66 * 8 < b128 < 2 * 4 * 128 * 128 * 66 * 8
    assert b256 > 7 * b128


def test_create_rejects_bad_arguments(lib):
    from paper_2106_03452_gb300 import libdpsr as L
    h = ctypes.c_void_p()
    for r, sigma in ((12, 2.0), (4, 2.0), (1024, 2.0), (64, -1.0), (64, float("nan"))):
        assert L.load().dpsr_plan_create(r, sigma, ctypes.byref(h)) == L.DPSR_EINVAL
    assert L.load().dpsr_forward(None, None, None, 10, None) == L.DPSR_EINVAL
    assert L.load().dpsr_backward(None, None, None, None) == L.DPSR_EINVAL
