"""The C-ABI library builds, loads and exports every entry point that
include/ch.h declares (host-only checks; no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2105_01865_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "ch.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ch_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(n for n, _, _ in capi.SIGNATURES) == names


def test_error_strings(lib):
    for code in range(6):
        assert capi.ch_error_string(code).startswith("CH_")


def test_workspace_bytes_validates(lib):
    p = capi.make_params((16, 12, 10), 0.1, (0, 0, 1), 0.075, 10.0, 1e-3, capi.CH_F32, advect=True)
    n = capi.ch_workspace_bytes(p)
    N = 16 * 12 * 10
    assert n >= 3 * N * 4 + (16 * 12 * 10 + 16 * 12 * 10 + 17 * 12 * 10) * 4
    bad = capi.make_params((16, 12, 4), 0.1, (0, 0, 1), 0.075, 10.0, 1e-3)       # n < 5
    assert capi.ch_workspace_bytes(bad) == 0
    bad = capi.make_params((16, 12, 10), 0.1, (0, 0, 3), 0.075, 10.0, 1e-3)      # bad bc
    assert capi.ch_workspace_bytes(bad) == 0
    bad = capi.make_params((16, 12, 10), 0.1, (2, 0, 1), 0.075, 10.0, 1e-3)      # Dirichlet only in z
    assert capi.ch_workspace_bytes(bad) == 0
    ok = capi.make_params((16, 12, 10), 0.1, (0, 0, 2), 0.075, 10.0, 1e-3)       # Dirichlet z walls
    assert capi.ch_workspace_bytes(ok) > 0
    bad = capi.make_params((16, 12, 10), 0.1, (0, 0, 2), 0.075, 10.0, 1e-3, scheme=capi.CH_SCHEME_STANDARD)
    assert capi.ch_workspace_bytes(bad) == 0                                      # split scheme only
    bad = capi.make_params((16, 12, 10), 0.1, (0, 0, 1), 0.075, 10.0, -1.0)      # dt <= 0
    assert capi.ch_workspace_bytes(bad) == 0


def test_create_rejects_null_pointers_without_touching_the_gpu(lib):
    p = capi.make_params((16, 12, 10), 0.1, (0, 0, 1), 0.075, 10.0, 1e-3)
    out = ctypes.c_void_p()
    st = lib.ch_create(ctypes.byref(p), None, None, 0, None, ctypes.byref(out))
    assert st == capi.CH_EINVAL and not out.value
