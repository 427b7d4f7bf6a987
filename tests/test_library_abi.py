"""The C-ABI library builds, loads and exports every function of include/*.h.

Runs without a GPU: only host-side entry points are called.
"""
import ctypes
import math
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(fftls_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1412_8398_gb300 import build, fftls
    build.build()
    return fftls.load_library()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["fftls_create", "fftls_destroy", "fftls_solve", "fftls_effective_stiffness",
                     "fftls_reference_medium", "fftls_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_header(lib):
    from paper_1412_8398_gb300 import fftls, warmstart
    assert set(_declared_functions()) == set(fftls._SIGNATURES) | set(warmstart._NN_SIGNATURES)


def test_nn_host_calls(lib):
    from paper_1412_8398_gb300 import warmstart
    n = (ctypes.c_int * 3)(8, 8, 8)
    assert lib.fftls_nn_wgrad_scratch(1, 2, 8, n, 3) >= 2 * 8 * 28
    assert warmstart.parameter_count() == sum(co * ci * k ** 3 + co for _, ci, co, k, _ in warmstart.LAYERS)


def test_host_only_calls(lib):
    from paper_1412_8398_gb300 import fftls
    assert fftls.supported_length(512) and fftls.supported_length(96) and fftls.supported_length(1)
    assert fftls.supported_length(48) and fftls.supported_length(5) and fftls.supported_length(1000)
    assert fftls.supported_length(2048) and fftls.supported_length(1536)
    assert not fftls.supported_length(7) and not fftls.supported_length(4096) and not fftls.supported_length(0)
    l0, m0 = fftls.reference_medium([0.6, 600.0], [0.6, 600.0], 3, "AS")
    assert abs(m0 - math.sqrt(0.6 * 600.0)) < 1e-12 and abs(l0 + 2 * m0 / 3 - math.sqrt(1000.0)) < 1e-12
    l0, m0 = fftls.reference_medium([0.4, 4.0], [0.6, 6.0], 2, "DS")
    assert abs(m0 - 3.3) < 1e-14 and abs(l0 + m0 - 5.5) < 1e-14
    with pytest.raises(fftls.FftlsError):
        fftls.reference_medium([0.6, 0.0], [0.6, 0.0], 3, "AS")   # porous: default degenerates
    assert lib.fftls_status_string(5) == b"FFTLS_E_NOT_CONVERGED"
    assert lib.fftls_status_string(7) == b"FFTLS_E_TIMEOUT" and fftls.status_name(7) == "FFTLS_E_TIMEOUT"
    assert [fftls.status_name(i) == lib.fftls_status_string(i).decode() for i in range(8)] == [True] * 8


def test_plan_rows_match_header(lib):
    """The binding's tile-schedule row has the header's FFTLS_PLAN_FIELDS fields, and the plan calls
    refuse a missing context on the host."""
    from paper_1412_8398_gb300 import fftls
    text = open(os.path.join(ROOT, "include", "fftls.h")).read()
    assert len(fftls.PLAN_KEYS) == int(re.search(r"#define FFTLS_PLAN_FIELDS (\d+)", text).group(1))
    n = ctypes.c_int(0)
    assert lib.fftls_tile_plans(None, None, ctypes.byref(n)) == 1  # FFTLS_E_INVALID_ARG
    assert lib.fftls_set_tile_plans(None, None, 0) == 1
