"""Step I of CLOSURE for 3D-3D in FP64 (oracle side): RANSAG.

Section IV, Step I (Example 2): each trial picks three distinct constraints,
takes one point inside each of their noise balls, fits a pose to the three
pairs with Arun's method (SVD of the cross-covariance, with the determinant
correction that keeps a proper rotation), and keeps the pose if it satisfies
every constraint of eq. (5).  S0 is the accepted poses in trial order, at
most ``max_seeds`` of them, from ``n_trials`` trials.

Random draws: trial tau uses the Philox streams (phase 5, j, 0, tau) of
oracle.philox; j = 0 gives the index triple, j = 1..3 the ball points.

Step I for pose regression (Example 3, the convex-combination sampler):
trial tau draws weights uniform on the simplex, w_i = e_i / sum_j e_j with
e_i = -log u_i and u_i = ((word_i >> 8) + 1/2) 2^-24 from words 0..N-1 of
stream (5, 0, 0, tau), and forms the pose t = sum w_i t_i,
R = proj_SO3(sum w_i R_i); it is kept if it lies in the PURSE.

Parity: pinned in tests/test_oracle_ransag.py (exact recovery of a
noise-free pose, least-squares optimality of the fitted rotation, every
accepted seed inside the PURSE) and tests/test_oracle_reg.py (simplex
weights, seeds inside the regression PURSE).
"""
from __future__ import annotations

import numpy as np

from . import philox
from .purse import in_purse
from .so3 import proj_so3


def arun(A, B):
    """Least-squares (R, t) with B ~ R A + t for corresponding rows (..., n, 3)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    abar = A.mean(axis=-2)
    bbar = B.mean(axis=-2)
    H = np.einsum('...ni,...nj->...ij', A - abar[..., None, :], B - bbar[..., None, :])
    U, _, Vt = np.linalg.svd(H)
    V = np.swapaxes(Vt, -1, -2)
    Ut = np.swapaxes(U, -1, -2)
    d = np.sign(np.linalg.det(V @ Ut))
    D = np.ones(H.shape[:-2] + (3,))
    D[..., 2] = d
    R = (V * D[..., None, :]) @ Ut
    t = bbar - np.einsum('...ij,...j->...i', R, abar)
    return R, t


def ransag_trials(purse, seed: int, trials):
    """Candidate pose and acceptance of each trial index in ``trials``."""
    tau = np.asarray(trials, dtype=np.int64)
    words = philox.stream_words(seed, philox.PHASE_RANSAG, 0, 0, tau, 3)
    idx = philox.distinct_triple(words, purse.n)                       # (T, 3)
    pts = np.stack([philox.ball_points(seed, philox.PHASE_RANSAG, c + 1, 0, tau)[0]
                    for c in range(3)], axis=1)                         # (T, 3, 3)
    lam = getattr(purse, "lam", None)
    if lam is not None:  # a point of the noise ellipsoid {e : e^T Lambda e <= r^2}: e = r U^-1 u
        U = np.swapaxes(np.linalg.cholesky(lam[idx]), -1, -2)
        pts = np.linalg.solve(U, pts[..., None])[..., 0]
    Bp = purse.obs[idx] + purse.radii[idx][..., None] * pts
    R, t = arun(purse.model[idx], Bp)
    ok = in_purse(purse, R, t)
    return R, t, ok, idx


def ransag_3d3d(purse, seed: int, n_trials: int, max_seeds: int, chunk: int = 1 << 14):
    """S0 as an (n, 12) array (R row-major, t) and the accepted trial indices."""
    seeds, acc = [], []
    for start in range(0, n_trials, chunk):
        tau = np.arange(start, min(n_trials, start + chunk))
        R, t, ok, _ = ransag_trials(purse, seed, tau)
        for n in np.nonzero(ok)[0]:
            if len(seeds) == max_seeds:
                break
            seeds.append(np.concatenate([R[n].reshape(9), t[n]]))
            acc.append(int(tau[n]))
        if len(seeds) == max_seeds:
            break
    return np.array(seeds).reshape(-1, 12), np.array(acc, dtype=np.int64)


def simplex_weights(seed: int, trials, n: int):
    """Weights (T, n) uniform on the simplex for the trials (Dirichlet(1, ..., 1) by -log u)."""
    words = philox.stream_words(seed, philox.PHASE_RANSAG, 0, 0, np.asarray(trials, np.int64), n)
    u = ((words >> np.uint64(8)).astype(np.float64) + 0.5) * 2.0 ** -24
    e = -np.log(u)
    return e / e.sum(axis=-1, keepdims=True)


def convex_trials(purse, seed: int, trials):
    """Candidate pose and acceptance of each trial of the convex-combination sampler."""
    w = simplex_weights(seed, trials, purse.n)
    t = w @ purse.obs
    R = proj_so3(np.einsum('tn,nij->tij', w, purse.rot_hyp))
    return R, t, in_purse(purse, R, t)


def convex_seeds(purse, seed: int, n_trials: int, max_seeds: int, chunk: int = 1 << 14):
    """S0 of a regression PURSE as an (n, 12) array and the accepted trial indices."""
    seeds, acc = [], []
    for start in range(0, n_trials, chunk):
        tau = np.arange(start, min(n_trials, start + chunk))
        R, t, ok = convex_trials(purse, seed, tau)
        for n in np.nonzero(ok)[0]:
            if len(seeds) == max_seeds:
                break
            seeds.append(np.concatenate([R[n].reshape(9), t[n]]))
            acc.append(int(tau[n]))
        if len(seeds) == max_seeds:
            break
    return np.array(seeds).reshape(-1, 12), np.array(acc, dtype=np.int64)
