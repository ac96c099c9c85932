"""Seeded synthetic PURSE instances.

This module only draws problem instances: keypoints, a ground-truth pose and
bounded measurement noise, following the generative model of eq. (1) with the
3D-3D residual of eq. (3) and the 2D-3D reprojection residual of eq. (2)
(pinhole intrinsics, pixel units).  It contains none of the CLOSURE steps
(walks, distances to the boundary, ball solvers); both the CUDA path and the
CPU oracle receive the arrays it returns.

The LM-O, 3DMatch and LM datasets of Section V are not available; these
instances stand in for them with the sizes of the published settings:

* ``purse_3d3d``  -- model points uniform in [-0.1, 0.1]^3 m, ground-truth
  rotation uniform on SO(3), translation uniform in [-0.5, 0.5]^3 m,
  observations b_i = R a_i + t + n_i with n_i uniform in the ball of radius
  r_i, r_i ~ U[0.005, 0.02] m (point-cloud registration, Example 2).
* ``purse_2d3d``  -- pinhole fx = fy = 600, cx = 320, cy = 240 (640x480),
  3D keypoints uniform in [-0.1, 0.1]^3 m, object depth U[0.5, 1.5] m with
  the projected origin uniform in the central half of the image, pixel noise
  uniform in the disk of radius r_i, r_i ~ U[2, 10] px (object pose
  estimation, Example 1).
* ``purse_octahedron`` -- noise-free 3D-3D instance with model points at
  L * (+-e_x, +-e_y, +-e_z) and equal radii; its ball radii have a closed form.
* ``purse_reg`` -- pose-regression PURSE (Example 3): ten pose hypotheses
  (R_i, t_i) scattered around a ground-truth pose (rotation noise of about
  0.03 rad, translation noise of about 0.01 m, the LM setting's ten hypotheses)
  with radii beta_i^R (Frobenius distance of rotation matrices) and beta_i^t
  (metres) each exceeding the hypothesis' distance to the ground truth by a
  random slack, so the ground truth lies in the PURSE.
* ``purse_3d3d_ellipsoidal`` / ``purse_2d3d_ellipsoidal`` -- the same instances with the noise
  bounded in the general norm of eq. 4: random positive definite Lambda_i (eigenvalues in
  [0.5, 2]), noise uniform in {e : sqrt(e^T Lambda_i e) <= r_i}; ``purse_octahedron_ellipsoidal``
  -- the octahedral instance with one Lambda for every constraint (closed-form translation ball).
* ``purse_reg_nested`` -- a regression PURSE whose first hypothesis is the
  ground truth with the smallest balls, each contained in every other
  hypothesis' ball: the PURSE is then that pair of balls and its geodesic balls
  are known in closed form.

All randomness comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

KIND_3D3D = 0
KIND_2D3D = 1
KIND_REG = 2


@dataclass
class Purse:
    """One PURSE instance (eq. 5 with Lambda_i = I and beta_i = r_i)."""

    kind: int                      # KIND_3D3D, KIND_2D3D or KIND_REG
    model: np.ndarray              # (N, 3) a_i (3D-3D) or Z_i (2D-3D); zeros for KIND_REG
    obs: np.ndarray                # (N, 3) b_i, (N, 2) pixel z_i, or (N, 3) hypotheses t_i (KIND_REG)
    radii: np.ndarray              # (N,) r_i > 0 (KIND_REG: beta_i^t)
    K: tuple | None = None         # (fx, fy, cx, cy) for 2D-3D, None otherwise
    R_gt: np.ndarray = field(default_factory=lambda: np.eye(3))
    t_gt: np.ndarray = field(default_factory=lambda: np.zeros(3))
    rot_hyp: np.ndarray | None = None    # (N, 3, 3) hypotheses R_i (KIND_REG)
    radii_rot: np.ndarray | None = None  # (N,) beta_i^R, Frobenius distance (KIND_REG)
    lam: np.ndarray | None = None        # (N, d, d) noise matrices Lambda_i of eq. 4 (None: identity)

    @property
    def n(self) -> int:
        return int(self.radii.shape[0])

    def seed_pose(self) -> np.ndarray:
        """Ground-truth pose packed as 12 doubles (R row-major, then t)."""
        return np.concatenate([self.R_gt.reshape(9), self.t_gt]).astype(np.float64)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform rotation from a uniform unit quaternion (Shoemake 1992)."""
    u1, u2, u3 = rng.random(3)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    w = b * np.cos(2 * np.pi * u3)
    x = a * np.sin(2 * np.pi * u2)
    y = a * np.cos(2 * np.pi * u2)
    z = b * np.sin(2 * np.pi * u3)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _in_ball(rng: np.random.Generator, n: int, dim: int, radii: np.ndarray) -> np.ndarray:
    """n points uniform in the dim-ball of the given radii (strictly inside)."""
    g = rng.standard_normal((n, dim))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    rho = radii * rng.random(n) ** (1.0 / dim) * (1.0 - 1e-9)
    return g * rho[:, None]


def purse_3d3d(n: int = 8, seed: int = 0, r_lo: float = 0.005, r_hi: float = 0.02,
               extent: float = 0.1, t_extent: float = 0.5) -> Purse:
    rng = np.random.default_rng(seed)
    a = rng.uniform(-extent, extent, (n, 3))
    R = _random_rotation(rng)
    t = rng.uniform(-t_extent, t_extent, 3)
    r = rng.uniform(r_lo, r_hi, n)
    b = a @ R.T + t + _in_ball(rng, n, 3, r)
    return Purse(KIND_3D3D, a, b, r, None, R, t)


def purse_2d3d(n: int = 16, seed: int = 0, r_lo: float = 2.0, r_hi: float = 10.0,
               K: tuple = (600.0, 600.0, 320.0, 240.0), width: int = 640, height: int = 480,
               extent: float = 0.1, z_lo: float = 0.5, z_hi: float = 1.5) -> Purse:
    rng = np.random.default_rng(seed)
    fx, fy, cx, cy = K
    Z = rng.uniform(-extent, extent, (n, 3))
    R = _random_rotation(rng)
    depth = rng.uniform(z_lo, z_hi)
    u0 = rng.uniform(0.25 * width, 0.75 * width)
    v0 = rng.uniform(0.25 * height, 0.75 * height)
    t = np.array([(u0 - cx) * depth / fx, (v0 - cy) * depth / fy, depth])
    r = rng.uniform(r_lo, r_hi, n)
    P = Z @ R.T + t
    pix = np.stack([fx * P[:, 0] / P[:, 2] + cx, fy * P[:, 1] / P[:, 2] + cy], axis=1)
    z = pix + _in_ball(rng, n, 2, r)
    return Purse(KIND_2D3D, Z, z, r, (fx, fy, cx, cy), R, t)


def purse_octahedron(L: float = 0.1, r: float = 0.01, seed: int = 0) -> Purse:
    """Model points L*(+-e_k), exact observations b_i = R_g a_i + t_g, equal radii."""
    rng = np.random.default_rng(seed)
    a = L * np.concatenate([np.eye(3), -np.eye(3)])
    R = _random_rotation(rng)
    t = rng.uniform(-0.5, 0.5, 3)
    b = a @ R.T + t
    return Purse(KIND_3D3D, a, b, np.full(6, r), None, R, t)


def _rotation_exp(v: np.ndarray) -> np.ndarray:
    """Rotation matrices exp([v]x) of rotation vectors v (..., 3) (Rodrigues' formula)."""
    v = np.asarray(v, dtype=np.float64)
    th = np.linalg.norm(v, axis=-1)[..., None, None]
    k = v / np.where(th[..., 0] > 0, th[..., 0], 1.0)
    Kx = np.zeros(v.shape[:-1] + (3, 3))
    Kx[..., 0, 1], Kx[..., 0, 2], Kx[..., 1, 2] = -k[..., 2], k[..., 1], -k[..., 0]
    Kx = Kx - np.swapaxes(Kx, -1, -2)
    return np.eye(3) + np.sin(th) * Kx + (1.0 - np.cos(th)) * (Kx @ Kx)


def purse_reg(n: int = 10, seed: int = 0, rot_sigma: float = 0.03, t_sigma: float = 0.01,
              slack_rot: tuple = (0.01, 0.04), slack_t: tuple = (0.003, 0.012)) -> Purse:
    rng = np.random.default_rng(seed)
    R = _random_rotation(rng)
    t = rng.uniform(-0.3, 0.3, 3) + np.array([0.0, 0.0, 1.0])
    Ri = _rotation_exp(rng.normal(size=(n, 3)) * rot_sigma) @ R
    ti = t + rng.normal(size=(n, 3)) * t_sigma
    bR = np.linalg.norm((Ri - R).reshape(n, 9), axis=1) + rng.uniform(*slack_rot, n)
    bt = np.linalg.norm(ti - t, axis=1) + rng.uniform(*slack_t, n)
    return Purse(KIND_REG, np.zeros((n, 3)), ti, bt, None, R, t, Ri, bR)


def purse_reg_nested(n: int = 10, seed: int = 0, beta_rot: float = 0.04, beta_t: float = 0.006) -> Purse:
    """Hypothesis 0 = ground truth with radii (beta_rot, beta_t); every other hypothesis' radii exceed
    its distance to hypothesis 0 plus those radii, so its balls contain hypothesis 0's."""
    p = purse_reg(n, seed)
    Ri, ti = p.rot_hyp.copy(), p.obs.copy()
    Ri[0], ti[0] = p.R_gt, p.t_gt
    bR = np.linalg.norm((Ri - Ri[0]).reshape(n, 9), axis=1) + beta_rot + 0.01
    bt = np.linalg.norm(ti - ti[0], axis=1) + beta_t + 0.002
    bR[0], bt[0] = beta_rot, beta_t
    return Purse(KIND_REG, np.zeros((n, 3)), ti, bt, None, p.R_gt, p.t_gt, Ri, bR)


def _spd(rng: np.random.Generator, n: int, d: int, lo: float, hi: float) -> np.ndarray:
    """n random symmetric positive definite d x d matrices with eigenvalues uniform in [lo, hi]."""
    Q, _ = np.linalg.qr(rng.normal(size=(n, d, d)))
    ev = rng.uniform(lo, hi, (n, d))
    return np.einsum('nij,nj,nkj->nik', Q, ev, Q)


def _in_ellipsoid(rng: np.random.Generator, lam: np.ndarray, radii: np.ndarray) -> np.ndarray:
    """One point uniform in each {e : e^T Lambda_i e <= r_i^2} (strictly inside)."""
    n, d, _ = lam.shape
    u = _in_ball(rng, n, d, np.ones(n))
    U = np.linalg.cholesky(lam).transpose(0, 2, 1)        # Lambda = U^T U, U upper triangular
    return radii[:, None] * np.linalg.solve(U, u[..., None])[..., 0]


def purse_3d3d_ellipsoidal(n: int = 8, seed: int = 0, ev: tuple = (0.5, 2.0)) -> Purse:
    """3D-3D PURSE with noise bounded in the norm of eq. 4: Lambda_i with eigenvalues in ev, noise
    uniform in {e : |e|_Lambda_i <= r_i}."""
    p = purse_3d3d(n, seed)
    rng = np.random.default_rng(seed + 7919)
    lam = _spd(rng, n, 3, *ev)
    b = p.model @ p.R_gt.T + p.t_gt + _in_ellipsoid(rng, lam, p.radii)
    return Purse(KIND_3D3D, p.model, b, p.radii, None, p.R_gt, p.t_gt, lam=lam)


def purse_2d3d_ellipsoidal(n: int = 16, seed: int = 0, ev: tuple = (0.5, 2.0)) -> Purse:
    """2D-3D PURSE with pixel noise bounded in the norm of eq. 4 (2 x 2 Lambda_i)."""
    p = purse_2d3d(n, seed)
    rng = np.random.default_rng(seed + 7919)
    lam = _spd(rng, n, 2, *ev)
    fx, fy, cx, cy = p.K
    P = p.model @ p.R_gt.T + p.t_gt
    pix = np.stack([fx * P[:, 0] / P[:, 2] + cx, fy * P[:, 1] / P[:, 2] + cy], axis=1)
    z = pix + _in_ellipsoid(rng, lam, p.radii)
    return Purse(KIND_2D3D, p.model, z, p.radii, p.K, p.R_gt, p.t_gt, lam=lam)


def purse_octahedron_ellipsoidal(L: float = 0.1, r: float = 0.01, seed: int = 0, ev=(0.5, 2.0)) -> Purse:
    """The octahedral PURSE with one noise matrix Lambda for all six constraints: its translations form
    the ellipsoid {d : d^T Lambda d <= r^2}, whose enclosing ball has the radius r / sqrt(lambda_min)."""
    p = purse_octahedron(L, r, seed)
    lam = _spd(np.random.default_rng(seed + 1), 1, 3, *ev)
    return Purse(KIND_3D3D, p.model, p.obs, p.radii, None, p.R_gt, p.t_gt, lam=np.repeat(lam, 6, axis=0))


def purse_batch(n_purses: int = 4096, seed: int = 0, n_lo: int = 4, n_hi: int = 64) -> list[Purse]:
    """Batch of PURSEs: kind chosen by a fair coin, N ~ U{n_lo..n_hi}."""
    rng = np.random.default_rng(seed)
    kinds = rng.integers(0, 2, n_purses)
    ns = rng.integers(n_lo, n_hi + 1, n_purses)
    subseeds = rng.integers(0, 2**62, n_purses)
    out = []
    for k, n, s in zip(kinds, ns, subseeds):
        out.append(purse_3d3d(int(n), int(s)) if k == KIND_3D3D else purse_2d3d(int(n), int(s)))
    return out


def seed_array(purses_or_poses) -> np.ndarray:
    """Stack seed poses (12 doubles each: R row-major, then t)."""
    arr = [p.seed_pose() if isinstance(p, Purse) else np.asarray(p, np.float64).reshape(12)
           for p in purses_or_poses]
    return np.stack(arr).astype(np.float64)
