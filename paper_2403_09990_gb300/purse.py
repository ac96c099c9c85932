"""Thin ctypes binding of libpurse (include/purse.h).

Argument marshalling only: every function forwards to the C ABI function of
the same name with raw device pointers (``tensor.data_ptr()``) and the
current CUDA stream.  Nothing here computes a step of the method, and there
is no CPU fallback: if the library is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

PURSE_3D3D, PURSE_2D3D, PURSE_REG = 0, 1, 2
STATUS = {0: "PURSE_OK", 1: "PURSE_ERR_ARG", 2: "PURSE_ERR_CUDA", 3: "PURSE_ERR_EMPTY", 4: "PURSE_ERR_TIMEOUT",
          5: "PURSE_ERR_NOMEM", 6: "PURSE_ERR_NUMERIC", 7: "PURSE_ERR_STATE"}


class PurseError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__(f"{fn}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class purse_intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double)]


class purse_params(ctypes.Structure):
    _fields_ = [("n_iter", ctypes.c_int), ("n_perturb", ctypes.c_int), ("n_keep", ctypes.c_int),
                ("n_steps", ctypes.c_int), ("omega0", ctypes.c_double), ("v0", ctypes.c_double),
                ("gamma", ctypes.c_double), ("rot_perturb", ctypes.c_double), ("trans_perturb", ctypes.c_double),
                ("perturb_units", ctypes.c_int), ("sampler", ctypes.c_int), ("precision", ctypes.c_int)]


class purse_tune_result(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("config", ctypes.c_int), ("ms", ctypes.c_float), ("default_config", ctypes.c_int),
                ("default_ms", ctypes.c_float), ("n_tried", ctypes.c_int)]


TUNE_WALK, TUNE_MEGB, TUNE_DIST, TUNE_BATCH = 0, 1, 2, 3


def make_params(n_iter=5, n_perturb=150, n_keep=10, n_steps=15, omega0=1.0, v0=2.0, gamma=0.5, rot_perturb=0.2,
                trans_perturb=0.1, perturb_units=0, sampler=0, precision=0) -> purse_params:
    return purse_params(n_iter, n_perturb, n_keep, n_steps, omega0, v0, gamma, rot_perturb, trans_perturb,
                        perturb_units, sampler, precision)


_LIB = None
_VP = ctypes.c_void_p
_SIGS = {
    "purse_create": [ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP, ctypes.POINTER(_VP)],
    "purse_create_regression": [ctypes.c_int, _VP, _VP, _VP, ctypes.POINTER(_VP)],
    "purse_set_noise": [_VP, _VP],
    "purse_destroy": [_VP],
    "purse_eval": [_VP, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP, _VP, _VP],
    "purse_dist": [_VP, ctypes.c_int, _VP, ctypes.c_longlong, _VP, _VP],
    "purse_ransag": [_VP, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_int), _VP],
    "purse_sample": [_VP, ctypes.POINTER(purse_params), ctypes.c_uint64, _VP, ctypes.c_int, ctypes.c_int, _VP, _VP,
                     _VP, _VP, _VP],
    "purse_sample_plain": [_VP, ctypes.POINTER(purse_params), ctypes.c_uint64, _VP, ctypes.c_int, ctypes.c_int, _VP,
                           _VP, _VP, _VP],
    "purse_last_evals": [_VP, ctypes.POINTER(ctypes.c_ulonglong), _VP],
    "megb_solve": [_VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP, _VP],
    "megb_solve_mean": [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP,
                        _VP],
    "megb_backward": [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP, ctypes.c_int, _VP, _VP, ctypes.c_int, _VP, _VP,
                      _VP, _VP, _VP, _VP],
    "megb_solve_exact": [_VP, ctypes.c_int, _VP, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP, _VP],
    "megb_solve_noalloc": [ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP, _VP],
    "purse_rng_words": [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                        ctypes.c_int, ctypes.c_int, _VP, _VP, ctypes.c_int, _VP],
    "purse_sync": [_VP, _VP],
    "purse_batch_create": [ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(_VP)],
    "purse_batch_create_regression": [ctypes.c_int, _VP, _VP, _VP, _VP, _VP],
    "purse_batch_destroy": [_VP],
    "purse_batch_set_noise": [_VP, _VP],
    "purse_batch_solve": [_VP, ctypes.POINTER(purse_params), ctypes.POINTER(purse_params), ctypes.c_uint64, _VP,
                          ctypes.c_int, ctypes.c_int, _VP, _VP],
    "purse_batch_tune": [_VP, ctypes.POINTER(purse_params), ctypes.POINTER(purse_params), ctypes.c_uint64, _VP,
                         ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                         ctypes.POINTER(ctypes.c_float), _VP],
    "purse_batch_copy_farthest": [_VP, _VP, _VP],
    "purse_batch_copy_samples": [_VP, ctypes.c_int, _VP, _VP, _VP, _VP, _VP],
    "purse_batch_set_grad": [_VP, ctypes.c_int],
    "purse_batch_copy_snap": [_VP, ctypes.c_int, _VP, _VP, _VP],
    "purse_batch_backward": [_VP, _VP, _VP, _VP, _VP, _VP],
    "purse_batch_sync": [_VP, ctypes.POINTER(ctypes.c_ulonglong), _VP],
    "purse_tune_walk": [_VP, ctypes.POINTER(purse_params), ctypes.c_uint64, _VP, ctypes.c_int, ctypes.c_int, _VP, _VP,
                        ctypes.POINTER(purse_tune_result), _VP],
    "purse_tune_megb": [_VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int, _VP, ctypes.c_int, _VP,
                        ctypes.POINTER(purse_tune_result), _VP],
    "purse_tune_dist": [_VP, ctypes.c_int, _VP, ctypes.c_longlong, _VP, ctypes.POINTER(purse_tune_result), _VP],
    "purse_tune_cache_get": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.c_char_p,
                             ctypes.POINTER(purse_tune_result)],
    "purse_tune_cache_put": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.c_char_p,
                             ctypes.c_int, ctypes.c_float],
    "purse_tune_cache_clear": [],
    "purse_last_error": [],
    "purse_version": [],
}


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """The loaded libpurse.so (built in-tree on first use)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libpurse.so not built ({path})")
            path = _build.build()
        L = ctypes.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name in ("purse_last_error", "purse_version") else ctypes.c_int
        _LIB = L
    return _LIB


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status: int, fn: str):
    if status != 0:
        raise PurseError(status, fn, lib().purse_last_error().decode())


def purse_create(kind: int, model, obs, radii, K=None) -> int:
    """Host arrays (numpy float64, contiguous) -> handle."""
    import numpy as np
    model = np.ascontiguousarray(model, dtype=np.float64)
    obs = np.ascontiguousarray(obs, dtype=np.float64)
    radii = np.ascontiguousarray(radii, dtype=np.float64)
    Kp = ctypes.byref(purse_intrinsics(*K)) if K is not None else None
    h = _VP()
    _check(lib().purse_create(kind, radii.shape[0], model.ctypes.data, obs.ctypes.data, radii.ctypes.data, Kp,
                              ctypes.byref(h)), "purse_create")
    return h.value


def purse_create_regression(hyp, beta_rot, beta_t) -> int:
    """Host arrays: hypotheses (n, 12) (R row-major, t), radii (n,) each -> handle."""
    import numpy as np
    hyp = np.ascontiguousarray(hyp, dtype=np.float64).reshape(-1, 12)
    beta_rot = np.ascontiguousarray(beta_rot, dtype=np.float64)
    beta_t = np.ascontiguousarray(beta_t, dtype=np.float64)
    h = _VP()
    _check(lib().purse_create_regression(hyp.shape[0], hyp.ctypes.data, beta_rot.ctypes.data, beta_t.ctypes.data,
                                         ctypes.byref(h)), "purse_create_regression")
    return h.value


def purse_set_noise(h, lam=None):
    """Noise matrices Lambda_i (n, d, d) of eq. 4 for the handle, or None for the identity."""
    import numpy as np
    if lam is None:
        _check(lib().purse_set_noise(h, None), "purse_set_noise")
        return
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    _check(lib().purse_set_noise(h, lam.ctypes.data), "purse_set_noise")


def purse_destroy(h: int):
    _check(lib().purse_destroy(h), "purse_destroy")


def purse_eval(h, precision, poses, n_poses, margin=None, active=None, grad=None, stream=None):
    _check(lib().purse_eval(h, precision, _ptr(poses), n_poses, _ptr(margin), _ptr(active), _ptr(grad),
                            _stream(stream)), "purse_eval")


def purse_dist(h, mode, poses, n_poses, dist, stream=None):
    _check(lib().purse_dist(h, mode, _ptr(poses), n_poses, _ptr(dist), _stream(stream)), "purse_dist")


def purse_ransag(h, seed, n_trials, max_seeds, seeds, stream=None) -> int:
    n = ctypes.c_int(0)
    _check(lib().purse_ransag(h, seed, n_trials, max_seeds, _ptr(seeds), ctypes.byref(n), _stream(stream)),
           "purse_ransag")
    return n.value


def purse_sample(h, params: purse_params, seed, seeds, s0, n_samples, q, t, trace=None, stream=None, snap=None):
    _check(lib().purse_sample(h, ctypes.byref(params), seed, _ptr(seeds), s0, n_samples, _ptr(q), _ptr(t),
                              _ptr(trace), _ptr(snap), _stream(stream)), "purse_sample")


def purse_sample_plain(h, params: purse_params, seed, seeds, s0, n_samples, q, t, trace=None, stream=None):
    _check(lib().purse_sample_plain(h, ctypes.byref(params), seed, _ptr(seeds), s0, n_samples, _ptr(q), _ptr(t),
                                    _ptr(trace), _stream(stream)), "purse_sample_plain")


def purse_last_evals(h, stream=None) -> int:
    v = ctypes.c_ulonglong(0)
    _check(lib().purse_last_evals(h, ctypes.byref(v), _stream(stream)), "purse_last_evals")
    return v.value


def megb_solve(h, precision, n_iters, q, n_rot, t, n_tr, result, farthest=None, stream=None):
    _check(lib().megb_solve(h, precision, n_iters, _ptr(q), n_rot, _ptr(t), n_tr, _ptr(result), _ptr(farthest),
                            _stream(stream)), "megb_solve")


def megb_solve_mean(h, precision, n_iters, n_last, q, n_rot, t, n_tr, result, farthest=None, stream=None):
    _check(lib().megb_solve_mean(h, precision, n_iters, n_last, _ptr(q), n_rot, _ptr(t), n_tr, _ptr(result),
                                 _ptr(farthest), _stream(stream)), "megb_solve_mean")


def megb_backward(h, precision, n_iters, q, snap_rot, n_rot, t, snap_tr, n_tr, farthest, result, grad_result,
                  grad_obs, grad_radii, stream=None):
    _check(lib().megb_backward(h, precision, n_iters, _ptr(q), _ptr(snap_rot), n_rot, _ptr(t), _ptr(snap_tr), n_tr,
                               _ptr(farthest), _ptr(result), _ptr(grad_result), _ptr(grad_obs), _ptr(grad_radii),
                               _stream(stream)), "megb_backward")


def megb_solve_exact(h, precision, q, n_rot, t, n_tr, result, ref=None, stream=None):
    _check(lib().megb_solve_exact(h, precision, _ptr(q), n_rot, _ptr(t), n_tr, _ptr(ref), _ptr(result),
                                  _stream(stream)), "megb_solve_exact")


def megb_solve_noalloc(precision, n_iters, q, n_rot, t, n_tr, result, farthest=None, stream=None):
    _check(lib().megb_solve_noalloc(precision, n_iters, _ptr(q), n_rot, _ptr(t), n_tr, _ptr(result), _ptr(farthest),
                                    _stream(stream)), "megb_solve_noalloc")


def purse_rng_words(seed, phase, j, i, w0, n_streams, n_words, words, lattice=None, unit=0, stream=None):
    _check(lib().purse_rng_words(seed, phase, j, i, w0, n_streams, n_words, _ptr(words), _ptr(lattice), unit,
                                 _stream(stream)), "purse_rng_words")


def _tune_dict(r):
    return {"op": r.op, "config": r.config, "ms": r.ms, "default_config": r.default_config, "default_ms": r.default_ms,
            "n_tried": r.n_tried}


def purse_tune_walk(h, params: purse_params, seed, seeds, s0, n_samples, q, t, stream=None) -> dict:
    r = purse_tune_result()
    _check(lib().purse_tune_walk(h, ctypes.byref(params), seed, _ptr(seeds), s0, n_samples, _ptr(q), _ptr(t),
                                 ctypes.byref(r), _stream(stream)), "purse_tune_walk")
    return _tune_dict(r)


def purse_tune_megb(h, precision, n_iters, q, n_rot, t, n_tr, result, stream=None) -> dict:
    r = purse_tune_result()
    _check(lib().purse_tune_megb(h, precision, n_iters, _ptr(q), n_rot, _ptr(t), n_tr, _ptr(result), ctypes.byref(r),
                                 _stream(stream)), "purse_tune_megb")
    return _tune_dict(r)


def purse_tune_dist(h, mode, poses, n_poses, dist, stream=None) -> dict:
    r = purse_tune_result()
    _check(lib().purse_tune_dist(h, mode, _ptr(poses), n_poses, _ptr(dist), ctypes.byref(r), _stream(stream)),
           "purse_tune_dist")
    return _tune_dict(r)


def purse_tune_cache_get(op, kind, n, n_samples, variant, gpu=None):
    """The cached choice as a dict, or None."""
    r = purse_tune_result()
    st = lib().purse_tune_cache_get(op, kind, n, n_samples, variant, gpu.encode() if gpu else None, ctypes.byref(r))
    if st == 7:
        return None
    _check(st, "purse_tune_cache_get")
    return _tune_dict(r)


def purse_tune_cache_put(op, kind, n, n_samples, variant, gpu, config, ms=0.0):
    _check(lib().purse_tune_cache_put(op, kind, n, n_samples, variant, gpu.encode() if gpu else None, config, ms),
           "purse_tune_cache_put")


def purse_tune_cache_clear():
    _check(lib().purse_tune_cache_clear(), "purse_tune_cache_clear")


def purse_sync(h, stream=None):
    _check(lib().purse_sync(h, _stream(stream)), "purse_sync")


def purse_batch_create(purses) -> int:
    """Batch handle from a list of synthetic.Purse-like objects."""
    import numpy as np
    kinds = np.array([int(p.kind) for p in purses], dtype=np.int32)
    offsets = np.zeros(len(purses) + 1, dtype=np.int32)
    offsets[1:] = np.cumsum([p.radii.shape[0] for p in purses])
    model = np.ascontiguousarray(np.concatenate([p.model for p in purses]), dtype=np.float64)
    obs = np.ascontiguousarray(np.concatenate(
        [p.obs if p.obs.shape[1] == 3 else np.concatenate([p.obs, np.zeros((p.obs.shape[0], 1))], 1) for p in purses]),
        dtype=np.float64)
    radii = np.ascontiguousarray(np.concatenate([p.radii for p in purses]), dtype=np.float64)
    Ks = (purse_intrinsics * len(purses))()
    for i, p in enumerate(purses):
        if p.K is not None:
            Ks[i] = purse_intrinsics(*p.K)
    h = _VP()
    _check(lib().purse_batch_create(len(purses), kinds.ctypes.data, offsets.ctypes.data, model.ctypes.data,
                                    obs.ctypes.data, radii.ctypes.data, ctypes.cast(Ks, _VP), ctypes.byref(h)),
           "purse_batch_create")
    return h.value


def purse_batch_create_regression(purses) -> int:
    """Batch handle from a list of pose-regression synthetic.Purse-like objects (rot_hyp, obs, radii_rot,
    radii)."""
    import numpy as np
    offsets = np.zeros(len(purses) + 1, dtype=np.int32)
    offsets[1:] = np.cumsum([p.radii.shape[0] for p in purses])
    hyp = np.ascontiguousarray(np.concatenate(
        [np.concatenate([np.asarray(p.rot_hyp).reshape(-1, 9), np.asarray(p.obs).reshape(-1, 3)], axis=1)
         for p in purses]), dtype=np.float64)
    br = np.ascontiguousarray(np.concatenate([p.radii_rot for p in purses]), dtype=np.float64)
    bt = np.ascontiguousarray(np.concatenate([p.radii for p in purses]), dtype=np.float64)
    h = _VP()
    _check(lib().purse_batch_create_regression(len(purses), offsets.ctypes.data, hyp.ctypes.data, br.ctypes.data,
                                               bt.ctypes.data, ctypes.byref(h)), "purse_batch_create_regression")
    return h.value


def purse_batch_set_noise(b, purses):
    """Noise matrices of every PURSE of the batch from the objects' lam (n x 3 x 3 or n x 2 x 2), in
    the CSR order of purse_batch_create; None (or PURSEs without lam) clears them."""
    import numpy as np
    if purses is None or all(getattr(p, "lam", None) is None for p in purses):
        _check(lib().purse_batch_set_noise(b, None), "purse_batch_set_noise")
        return
    rows = []
    for p in purses:
        lam = getattr(p, "lam", None)
        n = p.radii.shape[0]
        L = np.zeros((n, 3, 3))
        if lam is None:
            L[:] = np.eye(3)
        else:
            d = np.asarray(lam).shape[-1]
            L[:, :d, :d] = lam
            if d == 2:
                L[:, 2, 2] = 1.0
        rows.append(L.reshape(n, 9))
    arr = np.ascontiguousarray(np.concatenate(rows), dtype=np.float64)
    _check(lib().purse_batch_set_noise(b, arr.ctypes.data), "purse_batch_set_noise")


def purse_batch_destroy(b):
    _check(lib().purse_batch_destroy(b), "purse_batch_destroy")


def purse_batch_solve(b, p3d: purse_params, p2d: purse_params, seed, seeds, n_samples, n_iters, results, stream=None):
    _check(lib().purse_batch_solve(b, ctypes.byref(p3d), ctypes.byref(p2d), seed, _ptr(seeds), n_samples, n_iters,
                                   _ptr(results), _stream(stream)), "purse_batch_solve")


def purse_batch_tune(b, p3d, p2d, seed, seeds, n_samples, stream=None):
    c, w, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_float(0)
    _check(lib().purse_batch_tune(b, ctypes.byref(p3d), ctypes.byref(p2d), seed, _ptr(seeds), n_samples,
                                  ctypes.byref(c), ctypes.byref(w), ctypes.byref(ms), _stream(stream)),
           "purse_batch_tune")
    return c.value, w.value, ms.value


def purse_batch_copy_farthest(b, out, stream=None):
    _check(lib().purse_batch_copy_farthest(b, _ptr(out), _stream(stream)), "purse_batch_copy_farthest")


def purse_batch_copy_samples(b, p, q_rot=None, t_rot=None, q_tr=None, t_tr=None, stream=None):
    _check(lib().purse_batch_copy_samples(b, p, _ptr(q_rot), _ptr(t_rot), _ptr(q_tr), _ptr(t_tr), _stream(stream)),
           "purse_batch_copy_samples")


def purse_batch_set_grad(b, enable):
    _check(lib().purse_batch_set_grad(b, int(enable)), "purse_batch_set_grad")


def purse_batch_copy_snap(b, p, snap_rot=None, snap_tr=None, stream=None):
    _check(lib().purse_batch_copy_snap(b, p, _ptr(snap_rot), _ptr(snap_tr), _stream(stream)), "purse_batch_copy_snap")


def purse_batch_backward(b, results, grad_results, grad_obs, grad_radii, stream=None):
    _check(lib().purse_batch_backward(b, _ptr(results), _ptr(grad_results), _ptr(grad_obs), _ptr(grad_radii),
                                      _stream(stream)), "purse_batch_backward")


def purse_batch_sync(b, stream=None) -> int:
    v = ctypes.c_ulonglong(0)
    _check(lib().purse_batch_sync(b, ctypes.byref(v), _stream(stream)), "purse_batch_sync")
    return v.value


def version() -> str:
    return lib().purse_version().decode()


class Purse:
    """Owning wrapper of a PURSE handle built from a synthetic.Purse-like object."""

    def __init__(self, p):
        self.kind = int(p.kind)
        self.n = int(p.radii.shape[0])
        if self.kind == PURSE_REG:
            import numpy as np
            hyp = np.concatenate([np.asarray(p.rot_hyp).reshape(-1, 9), np.asarray(p.obs).reshape(-1, 3)], axis=1)
            self.h = purse_create_regression(hyp, p.radii_rot, p.radii)
        else:
            self.h = purse_create(self.kind, p.model, p.obs, p.radii, p.K if self.kind == PURSE_2D3D else None)
            if getattr(p, "lam", None) is not None:
                purse_set_noise(self.h, p.lam)

    def close(self):
        if self.h:
            purse_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
