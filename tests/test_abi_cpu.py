"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/fitrig.h declares; argument validation that needs no GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fitrig.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2509_21754_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"FITRIG_API\s+[\w\s\*]+?\b(fitrig_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("fitrig_plan_create", "fitrig_push_snapshot", "fitrig_detect",
                 "fitrig_candidates", "fitrig_plan_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    handle, path = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(fitrig_\w+)$", out, flags=re.M))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    for n in declared_symbols():
        getattr(handle, n)
    # nothing else leaks out of the library
    assert exported == set(declared_symbols())



def test_binding_wraps_every_declared_symbol():
    """The Python binding carries a function of the same name, and a ctypes
    signature, for every entry point of the header."""
    from paper_2509_21754_gb300 import fitrig as F
    names = declared_symbols()
    missing = [n for n in names if not callable(getattr(F, n, None))]
    assert not missing, missing
    untyped = [n for n in names if n not in F.SIGNATURES]
    assert not untyped, untyped

def test_status_strings(lib):
    from paper_2509_21754_gb300 import fitrig as F
    for s in range(10):
        assert F.status_string(s) and "unknown" not in F.status_string(s)
    assert "unknown" in F.status_string(99)


@pytest.mark.parametrize("args,code", [
    ((0, 10, 5, 2, 3.0, 1), 1),      # nx < 1
    ((10, 10, 5, 0, 3.0, 1), 1),     # window < 1
    ((10, 10, 5, 11, 3.0, 1), 1),    # window > min(nx, ny)
    ((10, 10, 2, 2, 3.0, 1), 1),     # fewer than 3 snapshots
    ((10, 10, 3, 2, 3.0, 2), 1),     # freq branch needs >= 4 snapshots
    ((10, 10, 5, 2, 0.0, 1), 1),     # nsigma <= 0
    ((10, 10, 5, 2, float("nan"), 1), 1),
    ((10, 10, 5, 2, 3.0, 4), 1),     # unknown branch
    ((300, 300, 5, 129, 3.0, 1), 9),  # windows above 128 are not implemented
    ((10, 10, 4099, 2, 3.0, 2), 9),  # transform longer than 4096 points
])
def test_plan_create_validation(lib, args, code):
    from paper_2509_21754_gb300 import fitrig as F
    h = ctypes.c_void_p()
    rc = F.load().fitrig_plan_create(*args, ctypes.byref(h))
    assert rc == code
    assert not h.value


def test_null_handles_are_rejected(lib):
    from paper_2509_21754_gb300 import fitrig as F
    L = F.load()
    n = ctypes.c_int32()
    d = ctypes.c_double()
    assert L.fitrig_detect(None, ctypes.byref(n)) == F.EINVAL
    assert L.fitrig_candidates(None, None, 0, ctypes.byref(n)) == F.EINVAL
    assert L.fitrig_push_snapshot(None, None, 0, 0, 0) == F.EINVAL
    assert L.fitrig_plan_set(None, 1, 0) == F.EINVAL
    assert L.fitrig_global_max(None, ctypes.byref(d)) == F.EINVAL
    assert L.fitrig_plan_destroy(None) == F.EINVAL
    assert L.fitrig_threshold_map(None, 10, 3.0, 0, 0, None, None, None) == F.EINVAL


def test_binding_raises_on_errors(lib):
    from paper_2509_21754_gb300 import fitrig as F
    with pytest.raises(F.FitrigError) as e:
        F.fitrig_plan_create(0, 10, 5, 2, 3.0)
    assert e.value.status == F.EINVAL


def test_new_entry_points_check_their_arguments_without_a_device(lib):
    """The block push and the caller-buffer candidates reject bad arguments
    before any device call."""
    import numpy as np
    from paper_2509_21754_gb300 import fitrig as F
    L = F.load()
    assert L.fitrig_push_snapshots(None, None, 1, F.F32, 0, 0, 0) == F.EINVAL
    buf = np.zeros((2, 4, 4), np.float32)
    assert L.fitrig_push_snapshots(None, ctypes.c_void_p(buf.ctypes.data), 2, F.F32, 0, 0, 0) == F.EINVAL
    with pytest.raises(F.FitrigError) as e:
        F.fitrig_push_snapshots(None, np.zeros((4, 4), np.float32))   # not a block
    assert e.value.status == F.EINVAL
    with pytest.raises(F.FitrigError) as e:
        F.fitrig_candidates(None, out=np.zeros(4, np.float32))         # wrong record type
    assert e.value.status == F.EINVAL
    assert L.fitrig_plan_set(None, F.OPT_HARMONICS, 8) == F.EINVAL
    assert L.fitrig_plan_set(None, F.OPT_REFINE, F.REFINE_CUBIC) == F.EINVAL
    assert L.fitrig_plan_set(None, F.OPT_CODING, F.CODING_DELTA) == F.EINVAL


def test_spectrum_map_checks_its_arguments_without_a_device(lib):
    """fitrig_spectrum_map rejects bad arguments before any device call."""
    from paper_2509_21754_gb300 import fitrig as F
    L = F.load()
    p = ctypes.c_void_p(16)   # never dereferenced: every call below fails validation
    ms = ctypes.c_float()
    assert L.fitrig_spectrum_map(None, 256, 8, 8, 1, p, p, 0, 0, ctypes.byref(ms)) == F.EINVAL
    assert L.fitrig_spectrum_map(p, 256, 8, 4, 1, p, p, 0, 0, None) == F.EINVAL       # stride < T
    assert L.fitrig_spectrum_map(p, 1, 8, 8, 1, p, p, 0, 0, None) == F.EINVAL         # n < 2
    assert L.fitrig_spectrum_map(p, 4097, 8, 8, 1, p, p, 0, 0, None) == F.EINVAL      # n > 4096
    assert L.fitrig_spectrum_map(p, 256, 8, 8, 3, p, p, 0, 0, None) == F.EINVAL       # harmonics
    assert L.fitrig_spectrum_map(p, 256, 8, 8, 64, p, p, 0, 0, None) == F.EINVAL
    assert L.fitrig_spectrum_map(p, 256, 8, 8, 1, p, p, 3, 0, None) == F.EINVAL       # method
    assert L.fitrig_spectrum_map(p, 300, 8, 8, 1, p, p, F.SPECTRUM_RADIX, 0, None) == F.EUNSUPPORTED
    assert L.fitrig_spectrum_map(p, 64, 8, 8, 1, p, p, F.SPECTRUM_RADIX, 0, None) == F.EUNSUPPORTED


def test_result_and_candidate_records_match_the_header():
    """The binding's record types have the sizes fitrig.h documents."""
    from paper_2509_21754_gb300 import fitrig as F
    assert F.RESULT_DTYPE.itemsize == 64
    assert F.CANDIDATE_DTYPE.itemsize == 32
