"""The C ABI: the library builds, loads and exports every symbol the header declares; host-side
argument checks and the no-device error path need no GPU."""
import ctypes
import os
import re

import pytest

from paper_2605_25346_b300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "diffreach.h")).read()
    return sorted(set(re.findall(r"\b(dr_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    build.build()
    lib = _lib.load()
    names = _declared()
    assert set(names) == set(_lib.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name


def test_create_without_device_reports_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    lib = _lib.load()
    ctx = ctypes.c_void_p()
    code = lib.dr_create(ctypes.byref(ctx), 0, None)
    assert code == _lib.DR_ERR_CUDA
    assert not ctx
    assert b"device" in lib.dr_last_error(None)


def test_null_context_arguments_are_rejected():
    lib = _lib.load()
    assert lib.dr_set_horizon(None, 5) == _lib.DR_ERR_ARG
    assert lib.dr_set_options(None, None) == _lib.DR_ERR_ARG
    assert lib.dr_kernel_launches(None) == 0


def test_wait_expiry_check_refuses_bad_budgets():
    # the budget is checked before any device query, with or without a GPU
    lib = _lib.load()
    assert lib.dr_check_wait_expiry(0.0) == _lib.DR_ERR_ARG
    assert lib.dr_check_wait_expiry(-1.0) == _lib.DR_ERR_ARG
    assert lib.dr_check_wait_expiry(3.0) == _lib.DR_ERR_ARG
    assert lib.dr_check_wait_expiry(float("nan")) == _lib.DR_ERR_ARG


def test_wait_expiry_check_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    lib = _lib.load()
    assert lib.dr_check_wait_expiry(0.1) == _lib.DR_ERR_CUDA  # no device to wait on
