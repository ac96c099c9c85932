"""PURSE constraints in FP64 (oracle side).

* 3D-3D (Example 2, eq. 3): g_i = b_i - (R a_i + t).
* 2D-3D (Example 1, eq. 2): g_i = z_i - pi(K (R Z_i + t)) in pixels, with
  pi(P) = (P_x / P_z, P_y / P_z) and K = [[fx, 0, cx], [0, fy, cy], [0, 0, 1]];
  a keypoint with P_z <= 0 (behind the camera) violates its constraint.
* PURSE (eq. 5) with Lambda_i = I, beta_i = r_i: all |g_i| <= r_i; with general
  positive definite Lambda_i (eq. 4) all sqrt(g_i^T Lambda_i g_i) <= r_i.
* margins r_i - |g_i| (-inf behind the camera) and dist(R, t, dS) =
  min_i margins (eq. 11).
* pose regression (Example 3, eq. PURSEreg): per hypothesis (R_i, t_i) two
  constraints, |vec(R) - vec(R_i)| <= beta_i^R (Frobenius) and
  |t - t_i| <= beta_i^t; the margins are the N rotation margins followed by
  the N translation margins.
* SE(3) gradient of h_i = |g_i| (with noise matrices |g_i|_Lambda_i) under the world-frame left
  perturbation R <- Exp(phi) R, t <- t + rho, returned as d h_i / d(phi, rho) (6 values).
Pinned in tests/test_oracle_purse.py against a direct scalar restatement of
eq. 2/3, cheirality cases and central finite differences of the gradient (also
with noise matrices).
"""
from __future__ import annotations

import numpy as np

KIND_3D3D = 0
KIND_2D3D = 1
KIND_REG = 2


def transform(model, R, t):
    """R a_i + t for every keypoint: (..., N, 3)."""
    return np.einsum('...ij,nj->...ni', R, model) + np.asarray(t)[..., None, :]


def lam_norm(g, lam):
    """|g|_Lambda = sqrt(g^T Lambda g) (eq. 4) of residuals g (..., N, d), Lambda (N, d, d)."""
    return np.sqrt(np.maximum(np.einsum('...ni,nij,...nj->...n', g, lam, g), 0.0))


def residual_norms(purse, R, t):
    """|g_i| (..., N) -- |g_i|_Lambda_i when the PURSE carries noise matrices -- and the in-front
    mask (all True for 3D-3D)."""
    X = transform(purse.model, R, t)
    lam = getattr(purse, "lam", None)
    if purse.kind == KIND_3D3D:
        g = purse.obs - X
        h = np.linalg.norm(g, axis=-1) if lam is None else lam_norm(g, lam)
        return h, np.ones(g.shape[:-1], dtype=bool)
    fx, fy, cx, cy = purse.K
    Pz = X[..., 2]
    front = Pz > 0
    Pzs = np.where(front, Pz, 1.0)
    u = fx * X[..., 0] / Pzs + cx
    v = fy * X[..., 1] / Pzs + cy
    gu = purse.obs[:, 0] - u
    gv = purse.obs[:, 1] - v
    if lam is not None:
        return lam_norm(np.stack([gu, gv], axis=-1), lam), front
    return np.sqrt(gu * gu + gv * gv), front


def margins(purse, R, t):
    """r_i - |g_i|, -inf for keypoints behind the camera; for a regression PURSE the 2N margins
    beta_i^R - |R - R_i|_F, then beta_i^t - |t - t_i|."""
    if purse.kind == KIND_REG:
        R = np.asarray(R, dtype=np.float64)
        t = np.asarray(t, dtype=np.float64)
        dR = np.sqrt(((R[..., None, :, :] - purse.rot_hyp) ** 2).sum(axis=(-2, -1)))
        dt = np.linalg.norm(t[..., None, :] - purse.obs, axis=-1)
        mR, mt = purse.radii_rot - dR, purse.radii - dt
        lead = np.broadcast_shapes(mR.shape[:-1], mt.shape[:-1])
        mR = np.broadcast_to(mR, lead + mR.shape[-1:])
        mt = np.broadcast_to(mt, lead + mt.shape[-1:])
        return np.concatenate([mR, mt], axis=-1)
    h, front = residual_norms(purse, R, t)
    return np.where(front, purse.radii - h, -np.inf)


def dist_to_boundary(purse, R, t):
    """eq. 11: min_i (beta_i - |g_i|)."""
    return margins(purse, R, t).min(axis=-1)


def in_purse(purse, R, t):
    """eq. 5: every constraint satisfied."""
    return (margins(purse, R, t) >= 0.0).all(axis=-1)


def norm_direction(e, lam):
    """d|e| / de: e / |e|, or with noise matrices (eq. 4) Lambda e / |e|_Lambda."""
    if lam is None:
        return e / np.linalg.norm(e, axis=-1, keepdims=True)
    le = np.einsum('nij,...nj->...ni', lam, e)
    return le / np.sqrt(np.einsum('...ni,...ni->...n', e, le))[..., None]


def margin_gradient(purse, R, t):
    """d|g_i| / d(phi, rho) under R <- Exp(phi) R, t <- t + rho; shape (..., N, 6).  With noise
    matrices the norm is |g_i|_Lambda_i, whose gradient in g is Lambda_i g_i / |g_i|_Lambda_i."""
    X = transform(purse.model, R, t)
    RA = X - np.asarray(t)[..., None, :]
    lam = getattr(purse, "lam", None)
    # d X / d phi = -[R a]x ; d X / d rho = I
    dX = np.concatenate([-_hat(RA), np.broadcast_to(np.eye(3), RA.shape + (3,))], -1)  # (...,N,3,6)
    if purse.kind == KIND_3D3D:
        e = X - purse.obs                       # = -g_i ; |g_i| = |e|
        return np.einsum('...i,...ij->...j', norm_direction(e, lam), dX)
    fx, fy, cx, cy = purse.K
    Kp = np.array([[fx, 0, cx], [0, fy, cy], [0, 0, 1.0]])
    P = X @ Kp.T
    Px, Py, Pz = P[..., 0], P[..., 1], P[..., 2]
    e = np.stack([Px / Pz - purse.obs[:, 0], Py / Pz - purse.obs[:, 1]], -1)  # = -g_i
    z = np.zeros_like(Pz)
    J = np.stack([np.stack([1 / Pz, z, -Px / Pz ** 2], -1),
                  np.stack([z, 1 / Pz, -Py / Pz ** 2], -1)], -2)   # (...,N,2,3)
    return np.einsum('...i,...ij,jk,...kl->...l', norm_direction(e, lam), J, Kp, dX)


def _hat(v):
    z = np.zeros(v.shape[:-1])
    return np.stack([
        np.stack([z, -v[..., 2], v[..., 1]], -1),
        np.stack([v[..., 2], z, -v[..., 0]], -1),
        np.stack([-v[..., 1], v[..., 0], z], -1),
    ], -2)
