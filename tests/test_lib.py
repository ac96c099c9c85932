"""The C-ABI library builds, loads and exports every declared entry point;
host-side argument validation (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2403_09990_gb300 import purse as P

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "purse.h")


def declared_functions():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:purse_status|const char\*)\s+(\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_symbol():
    L = P.lib()
    names = declared_functions()
    assert {"purse_create", "purse_sample", "megb_solve", "purse_destroy"} <= set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", P.library_path()], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert getattr(L, n) is not None
    assert "sm_103a" in P.version()


def test_binding_declares_every_symbol():
    assert set(declared_functions()) == set(P._SIGS)


def _status(fn, *args):
    return getattr(P.lib(), fn)(*args)


def test_argument_validation_without_gpu():
    L = P.lib()
    h = ctypes.c_void_p()
    model = np.zeros((2, 3))
    r = np.ones(2)
    # too few constraints
    assert L.purse_create(0, 2, model.ctypes.data, model.ctypes.data, r.ctypes.data, None, ctypes.byref(h)) == 1
    assert b"n must be" in L.purse_last_error()
    # bad kind, non-finite input, non-positive radius, missing intrinsics
    m3 = np.zeros((3, 3))
    r3 = np.ones(3)
    assert L.purse_create(7, 3, m3.ctypes.data, m3.ctypes.data, r3.ctypes.data, None, ctypes.byref(h)) == 1
    bad = m3.copy()
    bad[1, 1] = np.nan
    assert L.purse_create(0, 3, bad.ctypes.data, m3.ctypes.data, r3.ctypes.data, None, ctypes.byref(h)) == 1
    r_bad = np.array([1.0, 0.0, 1.0])
    assert L.purse_create(0, 3, m3.ctypes.data, m3.ctypes.data, r_bad.ctypes.data, None, ctypes.byref(h)) == 1
    assert L.purse_create(1, 3, m3.ctypes.data, m3.ctypes.data, r3.ctypes.data, None, ctypes.byref(h)) == 1
    # NULL handles are rejected before any CUDA call
    prm = P.make_params()
    assert L.purse_sample(None, ctypes.byref(prm), 0, None, 1, 1, None, None, None, None, None) == 1
    assert L.megb_solve(None, 0, 10, None, 0, None, 0, None, None, None) == 1
    assert L.purse_sync(None, None) == 1
    assert L.purse_destroy(None) == 0
    with pytest.raises(P.PurseError) as e:
        P.purse_destroy(None) or P._check(1, "x")
    assert e.value.status == 1


def test_regression_create_validation_without_gpu():
    L = P.lib()
    h = ctypes.c_void_p()
    hyp = np.tile(np.concatenate([np.eye(3).reshape(9), np.zeros(3)]), (3, 1))
    bR, bt = np.full(3, 0.1), np.full(3, 0.01)
    assert L.purse_create_regression(0, hyp.ctypes.data, bR.ctypes.data, bt.ctypes.data, ctypes.byref(h)) == 1
    bad = hyp.copy()
    bad[1, 0] = 2.0                                    # not a rotation
    assert L.purse_create_regression(3, bad.ctypes.data, bR.ctypes.data, bt.ctypes.data, ctypes.byref(h)) == 1
    assert b"rotation" in L.purse_last_error()
    z = np.array([0.1, 0.0, 0.1])
    assert L.purse_create_regression(3, hyp.ctypes.data, z.ctypes.data, bt.ctypes.data, ctypes.byref(h)) == 1
    assert L.purse_create_regression(3, None, bR.ctypes.data, bt.ctypes.data, ctypes.byref(h)) == 1


def test_noise_matrix_validation_without_gpu():
    L = P.lib()
    assert L.purse_set_noise(None, None) == 1
    assert b"NULL handle" in L.purse_last_error()
