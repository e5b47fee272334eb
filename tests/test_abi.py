"""The C-ABI library builds, loads and exports every entry point that
include/lbm.h declares; argument validation that needs no GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2208_13769_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = _declared()
    for n in ("lbm_create", "lbm_set_material", "lbm_set_boundary", "lbm_step", "lbm_read_fields",
              "lbm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    L = C.CDLL(lbm.library_path() if os.path.exists(lbm.library_path()) else lbm.lib()._name)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings():
    for s in range(7):
        assert lbm.status_string(s)
    assert lbm.status_string(99) == "unknown status"


def test_create_rejects_bad_descriptors_without_touching_the_gpu():
    L = lbm.lib()
    h = C.c_void_p()
    assert L.lbm_create(None, C.byref(h)) == lbm.LBM_E_INVALID
    d = lbm.lbm_desc()
    d.nx, d.ny, d.dX = 2, 8, 1.0
    assert L.lbm_create(C.byref(d), C.byref(h)) == lbm.LBM_E_INVALID and not h.value
    d.nx, d.ny, d.dX = 8, 8, 0.0
    assert L.lbm_create(C.byref(d), C.byref(h)) == lbm.LBM_E_INVALID
    d.dX, d.storage = 1.0, 7
    assert L.lbm_create(C.byref(d), C.byref(h)) == lbm.LBM_E_INVALID
    d.storage, d.scheme = 0, 5
    assert L.lbm_create(C.byref(d), C.byref(h)) == lbm.LBM_E_INVALID
    d.scheme, d.nx = 1, 0
    assert L.lbm_create(C.byref(d), C.byref(h)) == lbm.LBM_E_INVALID
    assert L.lbm_create(C.byref(d), None) == lbm.LBM_E_INVALID


def test_null_context_calls_fail_cleanly():
    L = lbm.lib()
    assert L.lbm_step(None, 1) == lbm.LBM_E_INVALID
    assert L.lbm_set_material(None, 1.0, 1.0, 1.0, 1.0, None) == lbm.LBM_E_INVALID
    assert L.lbm_set_boundary(None, 0, 0, None, None, None) == lbm.LBM_E_INVALID
    assert L.lbm_fields_size(None, 1) == 0
    assert L.lbm_destroy(None) == lbm.LBM_OK
    assert L.lbm_sync(None) == lbm.LBM_E_INVALID


def test_checkpoint_calls_reject_null_arguments_without_touching_the_gpu():
    L = lbm.lib()
    assert L.lbm_state_size(None) == 0
    buf = (C.c_uint8 * 64)()
    assert L.lbm_read_state(None, buf, 64) == lbm.LBM_E_INVALID
    assert L.lbm_write_state(None, buf, 64) == lbm.LBM_E_INVALID


def test_injected_allocation_failure_is_reported_before_any_cuda_call(monkeypatch):
    """LBM_FAULT=alloc makes lbm_create fail as if device memory were
    exhausted; it needs no GPU and leaves no context behind."""
    monkeypatch.setenv("LBM_FAULT", "alloc")
    L = lbm.lib()
    d = lbm.lbm_desc()
    d.nx, d.ny, d.dX = 16, 16, 1.0
    h = C.c_void_p()
    assert L.lbm_create(C.byref(d), C.byref(h)) == lbm.LBM_E_OOM and not h.value


def test_set_hole_rejects_null_arguments_without_touching_the_gpu():
    L = lbm.lib()
    hole = (C.c_int32 * 4)(4, 8, 4, 8)
    assert L.lbm_set_hole(None, hole, None) == lbm.LBM_E_INVALID


def test_measurement_and_batch_tuning_calls_reject_bad_arguments_without_touching_the_gpu():
    L = lbm.lib()
    out = (C.c_double * 4)()
    assert L.lbm_profile_interior(None, 10, out) == lbm.LBM_E_INVALID
    t, ms = lbm.lbm_tuning(), C.c_double()
    assert L.lbm_batch_autotune(None, 1, 16, C.byref(t), C.byref(ms)) == lbm.LBM_E_INVALID
    arr = (C.c_void_p * 1)(None)
    assert L.lbm_batch_autotune(arr, 1, 16, C.byref(t), C.byref(ms)) == lbm.LBM_E_INVALID  # NULL member
    assert L.lbm_batch_autotune(arr, 0, 16, C.byref(t), C.byref(ms)) == lbm.LBM_E_INVALID
    h = C.c_void_p()
    assert L.lbm_batch_create_tuned(arr, 1, None, C.byref(t), C.byref(h)) == lbm.LBM_E_INVALID
