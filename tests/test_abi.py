"""The C-ABI library builds, loads and exports every entry point include/ls.h declares (no GPU).

Only host-side calls are made here (no CUDA work): ls_version, ls_last_error, ls_calc_rho and
argument errors that are raised before any device call.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_11403_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(ls_[a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    from paper_2212_11403_gb300 import ls
    assert sorted(ls.EXPORTED) == names


def test_version_and_error_strings(lib):
    lib.ls_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.ls_version()
    lib.ls_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
    out = ctypes.c_void_p()
    assert lib.ls_create(ctypes.byref(out), None, 10, 10) == -1  # LS_ERR_ARG before any CUDA call
    lib.ls_last_error.restype = ctypes.c_char_p
    assert b"null" in lib.ls_last_error()


def test_calc_rho_matches_oracle_and_rejects_bad_input(lib):
    from paper_2212_11403_gb300 import ls
    m = np.array([7e-8, 1e-8, 5e-8, 4e-8, 1.4e-7, 1e-4, 0.3, 2.0])
    for Ne, g in [(1.0, 1.0), (2.0, 1.0), (0.7, 1.3)]:
        np.testing.assert_array_equal(ls.ls_calc_rho(m, Ne, g), oracle.calc_rho(m, Ne, g))
    with pytest.raises(ls.LSError):
        ls.ls_calc_rho(np.array([-1.0]))
    with pytest.raises(ls.LSError):
        ls.ls_calc_rho(np.array([1e-3]), 1.0, 0.0)
