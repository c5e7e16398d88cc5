"""The C-ABI library builds, loads without a GPU and exports every symbol
that include/oct_hydro.h declares; host-side validation rejects bad
arguments before touching the device (no compute call needs a GPU here)."""
import ctypes
import os
import re

import pytest

from paper_2210_06439_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "oct_hydro.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(oct_hydro_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = binding.load()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(binding.SIGNATURES)


def test_create_validates_arguments_on_host():
    L = binding.load()
    h = ctypes.c_void_p()
    assert L.oct_hydro_create(10, 8, 3, 5, 5.0 / 3.0, None) == binding.OCT_E_ARG
    for args in [(0, 8, 3, 5, 1.6), (4, 9, 3, 5, 1.6), (4, 8, 2, 5, 1.6), (4, 8, 3, 6, 1.6), (4, 8, 3, -1, 1.6),
                 (4, 8, 3, 5, 1.0), (4, 8, 3, 5, float("nan"))]:
        st = L.oct_hydro_create(*args, ctypes.byref(h))
        assert st == binding.OCT_E_ARG, args
        assert h.value is None
        assert L.oct_hydro_last_error().decode()


def test_null_handle_calls_fail_cleanly():
    L = binding.load()
    assert L.oct_hydro_rhs(None, None, None, None, None) == binding.OCT_E_ARG
    assert L.oct_hydro_rk_step(None, None, None, None) == binding.OCT_E_ARG
    assert L.oct_hydro_set_params(None, 0, 0.4, 1e-12, 1e-3, 0.1) == binding.OCT_E_ARG
    assert L.oct_hydro_state_len(None) == -1
    assert L.oct_hydro_step_launches(None) == -1
    assert L.oct_hydro_host_copy_bytes(None, None, None) == binding.OCT_E_ARG
    L.oct_hydro_destroy(None)


def test_create_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = binding.load()
    h = ctypes.c_void_p()
    st = L.oct_hydro_create(4, 8, 3, 5, 5.0 / 3.0, ctypes.byref(h))
    assert st in (binding.OCT_E_CUDA, binding.OCT_E_NOMEM)
    assert h.value is None


def test_build_flags_target_sm103a_only():
    assert "arch=compute_103a,code=sm_103a" in build.NVCC_FLAGS
    assert os.path.exists(build.LIB)
