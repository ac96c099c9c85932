"""Rotation helpers in FP64 (oracle side).

Quaternions are (w, x, y, z), Hamilton product, R(q) maps v to q v q*.
* exp_so3 / log_so3: Rodrigues' formula and its inverse through the unit
  quaternion (accurate at both small angles and near pi).
* dist_so3: the geodesic distance of Section II, arccos((tr(C^T R) - 1)/2);
  dist_quat evaluates the same angle as 2*atan2(|vec(c* q)|, |c.q|).
* proj_so3: nearest rotation (Frobenius) through the SVD, as used for the
  average rotation of Alg. 2 (line "R-bar").
* slerp: the geodesic step of Alg. 6, SLERP(A, B, tau) = A Exp(tau Log(A^T B)).
Pinned in tests/test_oracle_so3.py against closed forms and invariants.
"""
from __future__ import annotations

import numpy as np


def hat(v):
    v = np.asarray(v, dtype=np.float64)
    z = np.zeros(v.shape[:-1])
    return np.stack([
        np.stack([z, -v[..., 2], v[..., 1]], -1),
        np.stack([v[..., 2], z, -v[..., 0]], -1),
        np.stack([-v[..., 1], v[..., 0], z], -1),
    ], -2)


def exp_so3(v):
    """Rodrigues: R = I + sin(th)/th [v]x + (1 - cos th)/th^2 [v]x^2."""
    v = np.asarray(v, dtype=np.float64)
    th = np.linalg.norm(v, axis=-1)
    small = th < 1e-6
    ths = np.where(small, 1.0, th)
    a = np.where(small, 1.0 - th ** 2 / 6.0, np.sin(ths) / ths)
    b = np.where(small, 0.5 - th ** 2 / 24.0, (1.0 - np.cos(ths)) / ths ** 2)
    V = hat(v)
    I = np.broadcast_to(np.eye(3), V.shape)
    return I + a[..., None, None] * V + b[..., None, None] * (V @ V)


def quat_from_R(R):
    """Unit quaternion (w >= 0) of a rotation matrix (Shepperd's method)."""
    R = np.asarray(R, dtype=np.float64)
    shp = R.shape[:-2]
    R = R.reshape(-1, 3, 3)
    q = np.empty((R.shape[0], 4))
    for n, M in enumerate(R):
        tr = M[0, 0] + M[1, 1] + M[2, 2]
        d = np.array([tr, M[0, 0], M[1, 1], M[2, 2]])
        k = int(np.argmax(d))
        if k == 0:
            s = 2.0 * np.sqrt(1.0 + tr)
            q[n] = [0.25 * s, (M[2, 1] - M[1, 2]) / s, (M[0, 2] - M[2, 0]) / s, (M[1, 0] - M[0, 1]) / s]
        elif k == 1:
            s = 2.0 * np.sqrt(1.0 + M[0, 0] - M[1, 1] - M[2, 2])
            q[n] = [(M[2, 1] - M[1, 2]) / s, 0.25 * s, (M[0, 1] + M[1, 0]) / s, (M[0, 2] + M[2, 0]) / s]
        elif k == 2:
            s = 2.0 * np.sqrt(1.0 + M[1, 1] - M[0, 0] - M[2, 2])
            q[n] = [(M[0, 2] - M[2, 0]) / s, (M[0, 1] + M[1, 0]) / s, 0.25 * s, (M[1, 2] + M[2, 1]) / s]
        else:
            s = 2.0 * np.sqrt(1.0 + M[2, 2] - M[0, 0] - M[1, 1])
            q[n] = [(M[1, 0] - M[0, 1]) / s, (M[0, 2] + M[2, 0]) / s, (M[1, 2] + M[2, 1]) / s, 0.25 * s]
    q /= np.linalg.norm(q, axis=-1, keepdims=True)
    q *= np.where(q[:, :1] < 0, -1.0, 1.0)
    return q.reshape(shp + (4,))


def R_from_quat(q):
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def quat_mul(p, q):
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    pw, pv = p[..., :1], p[..., 1:]
    qw, qv = q[..., :1], q[..., 1:]
    w = pw * qw - (pv * qv).sum(-1, keepdims=True)
    v = pw * qv + qw * pv + np.cross(pv, qv)
    return np.concatenate([w, v], -1)


def quat_conj(q):
    q = np.asarray(q, dtype=np.float64)
    return np.concatenate([q[..., :1], -q[..., 1:]], -1)


def quat_log(q):
    """Rotation vector (axis * angle) of a unit quaternion, angle in [0, pi]."""
    q = np.asarray(q, dtype=np.float64)
    q = q * np.where(q[..., :1] < 0, -1.0, 1.0)
    v = q[..., 1:]
    s = np.linalg.norm(v, axis=-1)
    th = 2.0 * np.arctan2(s, q[..., 0])
    small = s < 1e-300
    scale = np.where(small, 2.0, th / np.where(small, 1.0, s))
    return v * scale[..., None]


def quat_exp(v):
    """Unit quaternion of the rotation vector v."""
    v = np.asarray(v, dtype=np.float64)
    th = np.linalg.norm(v, axis=-1)
    small = th < 1e-12
    k = np.where(small, 0.5, np.sin(0.5 * th) / np.where(small, 1.0, th))
    return np.concatenate([np.cos(0.5 * th)[..., None], v * k[..., None]], -1)


def log_so3(R):
    return quat_log(quat_from_R(R))


def dist_so3(C, R):
    """Geodesic distance of Section II: arccos((tr(C^T R) - 1) / 2)."""
    C = np.asarray(C, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    tr = np.einsum('...ij,...ij->...', C, R)
    return np.arccos(np.clip((tr - 1.0) / 2.0, -1.0, 1.0))


def dist_quat(c, q):
    """The same angle from unit quaternions: 2 atan2(|vec(c* q)|, |c . q|)."""
    d = quat_mul(quat_conj(c), q)
    return 2.0 * np.arctan2(np.linalg.norm(d[..., 1:], axis=-1), np.abs(d[..., 0]))


def proj_so3(M):
    """Nearest rotation to M in the Frobenius norm."""
    U, _, Vt = np.linalg.svd(np.asarray(M, dtype=np.float64))
    d = np.sign(np.linalg.det(U @ Vt))
    D = np.ones(U.shape[:-2] + (3,))
    D[..., 2] = d
    return (U * D[..., None, :]) @ Vt


def slerp(a, b, tau):
    """Point at fraction tau along the shorter geodesic from unit quaternion a to b."""
    a = np.asarray(a, dtype=np.float64)
    d = quat_mul(quat_conj(a), b)
    out = quat_mul(a, quat_exp(np.asarray(tau)[..., None] * quat_log(d)))
    out /= np.linalg.norm(out, axis=-1, keepdims=True)
    return out * np.where(out[..., :1] < 0, -1.0, 1.0)
