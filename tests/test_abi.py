"""The C-ABI library loads and exports every symbol include/shl.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2511_04025_b300 import build, shl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(shl_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    L = ctypes.CDLL(shl.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(shl.SIGNATURES), set(names) - set(shl.SIGNATURES)


def test_binding_loads_without_gpu():
    shl.lib()
    o = shl.default_solve_opts()
    assert o.E == 1.0 and o.nu == 0.3 and o.E_void == 1e-6 and o.tol == 1e-10
    assert o.precision == shl.SHL_FP64 and o.density == shl.SHL_MASK


def test_create_without_device_reports_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(shl.ShlError) as e:
        shl.shl_create(0)
    assert e.value.status in (shl.SHL_ECUDA, shl.SHL_EINVAL)
