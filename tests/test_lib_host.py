"""Host-side checks of the C-ABI library that need no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_05045_gb300 import build
    build.build()
    import paper_2507_05045_gb300 as msp
    return msp.load_library()


def header_symbols():
    src = open(os.path.join(ROOT, "include", "msp.h")).read()
    return sorted(set(re.findall(r"MSP_API[^;]*?\b(msp_\w+)\s*\(", src, flags=re.S)))


def test_header_declares_the_python_symbol_list():
    import paper_2507_05045_gb300 as msp
    assert header_symbols() == sorted(msp.EXPORTED_SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in header_symbols():
        assert hasattr(lib, name), name


def test_version_and_error_strings(lib):
    assert b"sm_103a" in lib.msp_version()
    assert lib.msp_last_error() is not None


def test_validation_errors_before_any_device_use(lib):
    import paper_2507_05045_gb300 as msp
    A = np.array([[1, -2, 3]], dtype=np.int32)
    with pytest.raises(msp.MspError) as e:
        msp.Instance(A, [1])
    assert e.value.code == -1  # MSP_EINVAL
    with pytest.raises(msp.MspError) as e:
        msp.Instance(np.ones((1, 101), np.int32), [1])
    assert e.value.code == -2  # MSP_ERANGE
    with pytest.raises(msp.MspError) as e:
        msp.Instance(np.full((1, 3), 30000, np.int32), [1])
    assert e.value.code == -2  # row sum >= 2^16
    with pytest.raises(msp.MspError) as e:
        msp.Instance(np.ones((2, 3), np.int32), [1, -1])
    assert e.value.code == -1


def test_null_arguments_are_rejected(lib):
    out = ctypes.c_void_p()
    assert lib.msp_create(None, None, 1, 1, ctypes.byref(out)) == -1
    lib.msp_destroy(None)
    lib.msp_free_solutions(None)
    lib.msp_server_destroy(None)


def test_no_device_fails_loudly_without_cpu_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    import paper_2507_05045_gb300 as msp
    with pytest.raises(msp.MspError) as e:
        msp.solve_all(np.ones((1, 4), np.int32), [2])
    assert e.value.code == -4  # MSP_ECUDA


def test_checked_build_loads_and_exports_every_symbol():
    # the MSP_CHECKED variant of the library builds here (nvcc cross-compiles)
    # and loads without a GPU; it is run on the parity cases by
    # tests/test_gpu_checked.py
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2507_05045_gb300 import build, msp\n"
            "lib = msp.load_library(build.build(checked=True))\n"
            "print(lib.msp_version().decode())\n"
            "print(all(hasattr(lib, s) for s in msp.EXPORTED_SYMBOLS))\n") % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    version, exported = r.stdout.strip().splitlines()[-2:]
    assert "MSP_CHECKED" in version and exported == "True"


def test_surrogate_merged_rows_exceed_the_field_limit(lib):
    # eq. 2 merges rows 1 and 2 with a multiplier above the row-1 sum; the
    # merged (9,80) row reaches millions, past the 16-bit packed fields, so
    # the library rejects the instance before any device work
    import paper_2507_05045_gb300 as msp
    import msp_instances as mi
    A, d, _ = mi.generate(9, 80, 9080)
    W = int(A[0].sum()) + 1
    merged = A[0].astype(np.int64) + W * A[1].astype(np.int64)
    A2 = np.vstack([merged, A[2:]]).astype(np.int32)
    d2 = np.concatenate([[int(d[0]) + W * int(d[1])], d[2:]]).astype(np.int32)
    with pytest.raises(msp.MspError) as e:
        msp.Instance(A2, d2)
    assert e.value.code == -2  # MSP_ERANGE
