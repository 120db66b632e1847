"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/ptn.h declares, and so does the benchmark's FMA-rate probe for include/ptn_peaks.h
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ptn.h")


def declared_functions(header=HEADER):
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*(ptn_[a-z0-9_]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ptn_solver_create", "ptn_solve_ip", "ptn_solve_admm", "ptn_solve_batch", "ptn_adjoint"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2409_20027_gb300 import build, ptn
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in ptn.h but not exported"
    assert set(declared_functions()) <= set(ptn.EXPORTS)
    assert lib is not None


def test_peaks_library_exports_its_header():
    from paper_2409_20027_gb300 import build
    names = declared_functions(os.path.join(ROOT, "include", "ptn_peaks.h"))
    assert names == ["ptn_peak_fma"]
    lib = ctypes.CDLL(build.build_peaks())
    for name in names:
        assert hasattr(lib, name)
    # invalid arguments are refused before any CUDA call
    lib.ptn_peak_fma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.ptn_peak_fma(2, 8, 10, None, None) == -1
    assert lib.ptn_peak_fma(0, 0, 10, None, None) == -1


def test_version_string_without_gpu():
    from paper_2409_20027_gb300 import ptn
    v = ptn.load().ptn_version().decode()
    assert "sm_103a" in v


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_2409_20027_gb300 import ptn
    with pytest.raises(OSError):
        ptn._open(str(tmp_path / "libptn.so"))


def test_entry_points_refuse_null_handles_and_pointers_without_a_gpu():
    # argument checks come before any CUDA call, so they answer on a machine without a GPU
    from paper_2409_20027_gb300 import ptn
    lib = ptn.load()
    INVALID = -1
    nx, nu = ctypes.c_int(), ctypes.c_int()
    assert lib.ptn_model_dims(1, ctypes.byref(nx), ctypes.byref(nu)) == 0 and (nx.value, nu.value) == (4, 1)
    assert lib.ptn_model_dims(1, None, None) == INVALID
    assert lib.ptn_model_dims(3, ctypes.byref(nx), ctypes.byref(nu)) == 0 and (nx.value, nu.value) == (32, 8)
    assert lib.ptn_model_dims(999, ctypes.byref(nx), ctypes.byref(nu)) == INVALID
    tb = (ctypes.c_int * 1)(8)
    assert lib.ptn_batch_prepare(None, 0, 1, tb, None, None) == INVALID
    assert lib.ptn_solve_batch_async(None, None, None, None, None, None, None, None, None) == INVALID
    assert lib.ptn_solve_ip(None, None, None, 8, None, None, None, None, None) == INVALID
    assert lib.ptn_set_options(None, None) == INVALID
    assert lib.ptn_set_reference(None, None, None) == INVALID
    assert lib.ptn_adjoint_checkpointed(None, 8, 4, None, None, None, None, 1.0, 1.0, None, None, None, None, None,
                                        None, None, None) == INVALID
    assert lib.ptn_last_error(None) is not None
    opt = ptn.Options()
    lib.ptn_default_options(ctypes.byref(opt))
    assert opt.costate_mode == 0 and opt.precision == ptn.PTN_FP32_FP64SOLVE
    # the struct mirror matches the C layout up to its last field (defaults read back)
    assert opt.armijo_eps32 == 1e-9 and opt.polish == 100.0 and opt.fp64_finish == 1
    # the static entry point checks its arguments first as well
    err = ctypes.create_string_buffer(256)
    rc = lib.ptn_solve_ip_static(None, None, None, None, 8, None, None, None, None, err, 256, None)
    assert rc == INVALID and b"NULL" in err.value
