"""The C-ABI library builds, loads and exports every declared symbol (CPU
only: no compute call reaches a GPU here; only argument checks that return
before any CUDA call are exercised)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fei.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1310_1194_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fei_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("fei_reference_create", "fei_reference_destroy", "fei_integrate",
                 "fei_integrate_backward", "fei_plan_offsets", "fei_last_error_string"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_argument_errors_before_any_cuda_call(lib):
    lib.fei_reference_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    lib.fei_last_error_string.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    assert lib.fei_reference_create(0, ctypes.byref(h)) == 2
    assert b"degree" in lib.fei_last_error_string()
    assert lib.fei_reference_create(8, ctypes.byref(h)) == 2
    assert lib.fei_reference_create(3, None) == 1
    lib.fei_integrate.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4
    assert lib.fei_integrate(None, 1, None, 0, None, None, None, None) == 1
    lib.fei_plan_offsets.argtypes = [ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 5
    assert lib.fei_plan_offsets(None, 5, None, None, None, None, None) == 1
    assert lib.fei_reference_destroy(None) == 0
    lib.fei_sync_status.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]
    assert lib.fei_sync_status(None, 4, None, None, None) == 1
    assert lib.fei_sync_status(None, -1, None, None, None) == 1
    # plans: argument errors are reported before any CUDA call
    vp = ctypes.c_void_p
    lib.fei_plan_create.argtypes = [vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int, vp]
    assert lib.fei_plan_create(None, 1, 10, 0, None) == 1
    out = vp()
    assert lib.fei_plan_create(None, 1, 10, 0, ctypes.byref(out)) == 1
    assert out.value is None
    lib.fei_plan_execute.argtypes = [vp] * 6
    assert lib.fei_plan_execute(None, None, None, None, None, None) == 1
    lib.fei_plan_tune.argtypes = [vp] * 6
    assert lib.fei_plan_tune(None, None, None, None, None, None) == 1
    lib.fei_plan_choice.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    assert lib.fei_plan_choice(None, 3, None, None, None) == 1
    lib.fei_plan_set_choice.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64]
    assert lib.fei_plan_set_choice(None, 3, 0, 0) == 1
    lib.fei_plan_kernel.argtypes = [vp, ctypes.c_int, vp]
    assert lib.fei_plan_kernel(None, 3, None) == 1
    lib.fei_pipeline_create.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, vp]
    out = vp()
    assert lib.fei_pipeline_create(None, 1, 0, 0, ctypes.byref(out)) == 1 and out.value is None
    assert lib.fei_pipeline_create(None, 1, 0, 0, None) == 1
    lib.fei_integrate_host.argtypes = [vp] * 7
    assert lib.fei_integrate_host(None, None, None, None, None, None, None) == 1
    lib.fei_pipeline_info.argtypes = [vp] * 3
    assert lib.fei_pipeline_info(None, None, None) == 1
    lib.fei_pipeline_destroy.argtypes = [vp]
    assert lib.fei_pipeline_destroy(None) == 0
    assert lib.fei_plan_destroy(None) == 0
    lib.fei_integrate_backward_quadratic.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp, vp, vp, vp]
    assert lib.fei_integrate_backward_quadratic(None, 1, None, 0, None, None, None, None) == 1
    lib.fei_status_summary.argtypes = [vp, ctypes.c_int64, vp, vp]
    assert lib.fei_status_summary(None, 5, None, None) == 1
    assert lib.fei_status_summary(None, 0, None, None) == 0
    assert lib.fei_status_summary(None, -1, None, None) == 1


def test_python_binding_loads():
    from paper_1310_1194_gb300 import _lib
    assert _lib.lib is not None
    assert _lib.PRECISIONS["fp64"] == 0


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    """No CPU fallback: with libfei.so absent, importing the binding raises."""
    import importlib.util
    import os as _os
    import sys as _sys
    src = _os.path.join(ROOT, "paper_1310_1194_gb300", "_lib.py")
    text = open(src).read().replace('LIB_PATH = os.path.join(HERE, "_build", "libfei.so")',
                                    f'LIB_PATH = {str(tmp_path / "missing" / "libfei.so")!r}')
    path = tmp_path / "lib_missing.py"
    path.write_text(text)
    spec = importlib.util.spec_from_file_location("lib_missing", str(path))
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)
