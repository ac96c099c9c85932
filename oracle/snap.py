"""Boundary snap of the samples (FP64, oracle side), for differentiating the balls.

The walks of Alg. 2-5 end near the PURSE boundary after discrete decisions,
so the samples are piecewise constant in the observations y_i and radii r_i.
Reading used here (not in the paper; needed for a derivative): each final
sample is moved along the ray of its walk's last move direction -- rotations
x(tau) = (Exp(tau omega) R*, t*) for the rotation-boundary sampler,
translations x(tau) = (R*, t* + tau v) for the translation-boundary sampler --
to the boundary:
* tau_hi = the smallest ladder value gamma^m, m = N_T-1 down to 0, with
  x(tau_hi) outside S (none: the sample stays, with no active constraint);
* bisection of [0, tau_hi] keeps x(lo) in S and x(hi) outside, to
  |hi - lo| <= 2^-40 tau_hi;
* the snapped sample is x(lo) and the active constraint j* is the one with
  the smallest margin there.
At the snapped sample h_j*(x(tau*)) = r_j*, so by the implicit-function
theorem d tau*/d r_j* = 1 / h'(tau*) and d tau*/d y_j* = -(d h_j*/d y_j*) / h'(tau*)
with h'(tau) = d h_j*(x(tau)) / d tau.  With noise matrices (eq. 4) h is the norm
|g|_Lambda, whose gradient in the residual g is Lambda g / |g|_Lambda.

Parity: pinned in tests/test_oracle_snap.py (snapped samples on the
boundary and inside S; central finite differences of tau* against the
implicit derivatives, identity norm and noise matrices).
"""
from __future__ import annotations

import numpy as np

from .purse import KIND_3D3D, in_purse, margins, margin_gradient
from .so3 import exp_so3


def ray_pose(R, t, direction, tau, rotation: bool):
    tau = np.asarray(tau, dtype=np.float64)
    if rotation:
        return exp_so3(tau[..., None] * direction) @ R, t
    return R, t + tau[..., None] * direction


def snap(purse, R, t, direction, ladder, rotation: bool, bisections: int = 60):
    """(R_snap, t_snap, tau*, j* (-1 = not snapped)) for samples (W, 3, 3), (W, 3), directions (W, 3)."""
    R = np.asarray(R, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    W = R.shape[0]
    hi = np.full(W, -1.0)
    for tau in sorted(ladder):                       # smallest ladder value first
        Rx, tx = ray_pose(R, t, direction, np.full(W, tau), rotation)
        out = ~in_purse(purse, Rx, tx) & (hi < 0)
        hi[out] = tau
    ok = hi > 0
    lo = np.zeros(W)
    h = np.where(ok, hi, 0.0)
    for _ in range(bisections):
        mid = 0.5 * (lo + h)
        Rx, tx = ray_pose(R, t, direction, mid, rotation)
        feas = in_purse(purse, Rx, tx)
        lo = np.where(ok & feas, mid, lo)
        h = np.where(ok & ~feas, mid, h)
    Rs, ts = ray_pose(R, t, direction, lo, rotation)
    m = margins(purse, Rs, ts)
    jstar = np.where(ok, np.argmin(m, axis=1), -1)
    return Rs, ts, lo, jstar


def ray_derivatives(purse, Rs, ts, direction, jstar, rotation: bool):
    """h'(tau*) and d h_j*/d y_j* at the snapped samples (rows with j* < 0 are zero)."""
    W = Rs.shape[0]
    G = margin_gradient(purse, Rs, ts)                              # (W, N, 6): d|g_i| / d(phi, rho)
    rows = np.arange(W)
    j = np.maximum(jstar, 0)
    g = G[rows, j]
    dh_dtau = np.einsum('wc,wc->w', g[:, :3] if rotation else g[:, 3:], direction)
    # d|g_j| / d y_j at fixed pose: 3D-3D y = b_j, |g| = |b - (R a + t)|; 2D-3D y = z_j (pixels)
    X = np.einsum('wij,wj->wi', Rs, purse.model[j]) + ts
    if purse.kind == KIND_3D3D:
        e = purse.obs[j] - X
    else:
        fx, fy, cx, cy = purse.K
        e = purse.obs[j] - np.stack([fx * X[:, 0] / X[:, 2] + cx, fy * X[:, 1] / X[:, 2] + cy], 1)
    lam = getattr(purse, "lam", None)
    if lam is None:
        dh_dy = e / np.linalg.norm(e, axis=1, keepdims=True)
    else:  # |g|_Lambda: the gradient in g = y - (projection of) X is Lambda g / |g|_Lambda
        le = np.einsum('wij,wj->wi', lam[j], e)
        dh_dy = le / np.sqrt((e * le).sum(axis=1, keepdims=True))
    valid = jstar >= 0
    return np.where(valid, dh_dtau, 0.0), np.where(valid[:, None], dh_dy, 0.0)
