"""Failure detection on the host paths (CPU only): PURSE_FAULT injection.

The library reads PURSE_FAULT at every call and refuses the named operation on the host, before
any CUDA call, with the status a real failure of that kind returns: ``alloc`` -> PURSE_ERR_NOMEM,
``launch`` -> PURSE_ERR_CUDA, ``nan_input`` -> PURSE_ERR_ARG (the validation sees a NaN),
``empty_seed`` -> PURSE_ERR_EMPTY.  These tests call entry points that need no device once the
fault is injected; the ones that need a handle (empty_seed, the bounded device wait of
``stall``, recovery after each fault) are in test_gpu_faults.py.
"""
import ctypes

import numpy as np
import pytest

from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn

ARG, CUDA, EMPTY, NOMEM = 1, 2, 3, 5


def _create(p):
    L = P.lib()
    model = np.ascontiguousarray(p.model, dtype=np.float64)
    obs = np.ascontiguousarray(p.obs, dtype=np.float64)
    radii = np.ascontiguousarray(p.radii, dtype=np.float64)
    K = P.purse_intrinsics(*p.K) if p.kind == 1 else None
    h = ctypes.c_void_p()
    st = L.purse_create(p.kind, len(radii), model.ctypes.data, obs.ctypes.data, radii.ctypes.data,
                        ctypes.byref(K) if K is not None else None, ctypes.byref(h))
    return st, h, obs


def _release(st, h):
    if st == 0:
        P.lib().purse_destroy(h)


@pytest.mark.parametrize("kind", [0, 1])
def test_alloc_fault_refuses_purse_create_before_the_device(monkeypatch, kind):
    monkeypatch.setenv("PURSE_FAULT", "alloc")
    p = syn.purse_3d3d(8, 0) if kind == 0 else syn.purse_2d3d(12, 0)
    st, h, _ = _create(p)
    assert st == NOMEM and not h.value
    assert b"injected fault (PURSE_FAULT=alloc)" in P.lib().purse_last_error()


def test_alloc_fault_refuses_purse_batch_create(monkeypatch):
    monkeypatch.setenv("PURSE_FAULT", "alloc")
    L = P.lib()
    ps = [syn.purse_3d3d(5, 1), syn.purse_2d3d(7, 2)]
    offs = np.array([0, 5, 12], dtype=np.int32)
    kinds = np.array([0, 1], dtype=np.int32)
    model = np.concatenate([q.model for q in ps])
    obs = np.concatenate([ps[0].obs, np.c_[ps[1].obs, np.zeros(7)]])
    radii = np.concatenate([q.radii for q in ps])
    Ks = (P.purse_intrinsics * 2)(P.purse_intrinsics(0, 0, 0, 0), P.purse_intrinsics(*ps[1].K))
    b = ctypes.c_void_p()
    st = L.purse_batch_create(2, kinds.ctypes.data, offs.ctypes.data, model.ctypes.data, obs.ctypes.data,
                              radii.ctypes.data, Ks, ctypes.byref(b))
    assert st == NOMEM and not b.value
    assert b"PURSE_FAULT=alloc" in L.purse_last_error()


def test_nan_input_fault_is_caught_by_the_validation_and_leaves_the_caller_array(monkeypatch):
    monkeypatch.setenv("PURSE_FAULT", "nan_input")
    p = syn.purse_3d3d(8, 3)
    st, h, obs = _create(p)
    assert st == ARG and not h.value
    assert b"non-finite" in P.lib().purse_last_error()
    assert np.all(np.isfinite(obs)) and np.array_equal(obs, p.obs)


def test_nan_input_fault_in_the_regression_constructor(monkeypatch):
    monkeypatch.setenv("PURSE_FAULT", "nan_input")
    p = syn.purse_reg(10, 0)
    L = P.lib()
    hyp = np.ascontiguousarray(np.concatenate([p.rot_hyp.reshape(-1, 9), p.obs], axis=1))
    br = np.ascontiguousarray(p.radii_rot)
    bt = np.ascontiguousarray(p.radii)
    h = ctypes.c_void_p()
    st = L.purse_create_regression(len(bt), hyp.ctypes.data, br.ctypes.data, bt.ctypes.data, ctypes.byref(h))
    assert st == ARG and b"non-finite" in L.purse_last_error()
    assert np.all(np.isfinite(hyp))


def test_launch_fault_refuses_handle_free_calls(monkeypatch):
    monkeypatch.setenv("PURSE_FAULT", "launch")
    L = P.lib()
    buf = np.zeros(64).ctypes.data  # never dereferenced: the call is refused first
    assert L.megb_solve_noalloc(0, 10, buf, 10, buf, 10, buf, None, None) == CUDA
    assert b"injected fault (PURSE_FAULT=launch)" in L.purse_last_error()
    assert L.purse_rng_words(1, 1, 0, 0, 0, 4, 4, buf, None, 0, None) == CUDA
    assert b"purse_rng_words" in L.purse_last_error()


def test_argument_errors_come_before_injected_faults(monkeypatch):
    monkeypatch.setenv("PURSE_FAULT", "launch,alloc")
    L = P.lib()
    buf = np.zeros(64).ctypes.data
    assert L.megb_solve_noalloc(0, 5000, buf, 10, buf, 10, buf, None, None) == ARG   # n_iters > 4096
    assert L.purse_rng_words(1, 300, 0, 0, 0, 4, 4, buf, None, 0, None) == ARG       # phase > 255


def test_fault_list_matches_whole_site_names(monkeypatch):
    # "nan_inputs" and "xalloc" name no site: purse_create sees neither fault (on a machine
    # without a GPU it then fails on the device, with PURSE_ERR_CUDA)
    monkeypatch.setenv("PURSE_FAULT", "nan_inputs,xalloc")
    p = syn.purse_3d3d(8, 0)
    st, h, _ = _create(p)
    assert st not in (ARG, NOMEM), P.lib().purse_last_error()
    _release(st, h)
    # several sites: the first one met on the path wins (validation before allocation)
    monkeypatch.setenv("PURSE_FAULT", "alloc,nan_input")
    st, h, _ = _create(p)
    assert st == ARG
    monkeypatch.setenv("PURSE_FAULT", "")
    st, h, _ = _create(p)
    assert st not in (ARG, NOMEM)
    _release(st, h)
