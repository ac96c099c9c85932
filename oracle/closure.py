"""Step II of CLOSURE in FP64 (oracle side): the strategic random walks.

Restates, in the paper's order and notation,
* the centre statistics of Alg. 2: R-bar = proj_SO3(sum R_j), t-bar = mean t_j;
* "walk away from the centre" (Section IV, Step II): omega = omega0 (u + u~)
  with (u, theta) the axis-angle of R_0 R-bar^T, and
  v = v0 S ((t_0 - t-bar)/|t_0 - t-bar| + v~), S the PCA scaling (2D-3D only);
* the parallel rotation-boundary sampler (Alg. 3, serial form Alg. 2) and the
  parallel translation-boundary sampler (Alg. 5, serial form Alg. 4):
  perturbation -> dist (eq. 11) -> top_k_indices -> step ladder
  Delta T = gamma^(m-1) -> in_purse -> find_farthest (m0 = smallest feasible
  m, then the best-ranked feasible k).

Readings of the paper used here (where it is silent or ambiguous):
* update_rotation(R*, omega, dT) = Exp(dT omega) R*, translation unchanged;
  update_translation(t*, R_jk, v, dT) = t* + dT v (R_jk unused).
* perturbation(t_p) is a point uniform in the ball of radius t_p * sigma_t
  (hat-box direction, radius whose cube is uniform; oracle.philox),
  perturbation(theta_p) is Exp of a vector uniform in the ball of radius
  theta_p * sigma_t / rho_a, where sigma_t is the PURSE translation scale
  (mean r_i for 3D-3D, mean r_i * t-bar_z / f for 2D-3D, mean beta_i^t for
  pose regression) and rho_a the RMS spread of the model points (pose
  regression: sigma_t sqrt(2) / mean beta_i^R, so that the rotation radius is
  theta_p times the angle scale of the rotation balls); ``perturb_units = 1``
  uses t_p, theta_p raw.
* Ties in top_k_indices go to the lower index; k0 is the best-ranked
  feasible k at m0; when nothing is feasible the walk keeps its pose.
* u = 0 when the angle of R_0 R-bar^T is <= 1e-9 rad, the direction term of
  v is 0 when |t_0 - t-bar| <= 1e-9 (1 + |t-bar|).
* PCA scaling S = U diag(sigma_k / sigma_1) U^T of the covariance of the
  seed translations when there are >= 4 seeds and sigma_1 > 0; otherwise
  S = u1 u1^T + (rho_a / |t-bar|)(I - u1 u1^T) with u1 = t-bar/|t-bar| (the
  viewing ray, along which a 2D-3D PURSE is long).
* Walk w starts from seed (w mod |S0|); its random draws are the Philox
  streams of oracle.philox named by w; perturbations 2b and 2b + 1 of an
  iteration come from one Philox block.

Parity: pinned in tests/test_oracle_walk.py (octahedral PURSE with
closed-form radii and Prop. 1, membership of every output sample, the
needle shape of a 2D-3D PURSE, seeds-versus-walks spread) and in
tests/test_oracle_velocity.py (start velocities: unit random parts, mean
projection 1 on the outward axis and direction, distance to the centre
growing at rates omega0 and v0; PCA scaling against the axes and ratios of a
known anisotropic seed cloud, the viewing ray with few seeds; both samplers
on the appendix's unit-ball toy set).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import philox
from .purse import KIND_2D3D, KIND_3D3D, KIND_REG, dist_to_boundary, in_purse
from .so3 import exp_so3, log_so3, proj_so3, quat_from_R


@dataclass
class Params:
    """Simulation parameters P of Alg. 1 (names of Alg. 2-5)."""
    n_walk: int = 2          # N_W
    n_iter: int = 5          # N_I
    n_perturb: int = 150     # N_P
    n_keep: int = 10         # N_P*
    n_steps: int = 15        # N_T
    omega0: float = 1.0      # omega_0
    v0: float = 2.0          # v_0
    gamma: float = 0.5       # time-step decay
    rot_perturb: float = 0.2     # theta_p (R_p)
    trans_perturb: float = 0.1   # t_p
    perturb_units: int = 0       # 0: relative to the PURSE scale, 1: raw units


def preset_2d3d(**kw) -> Params:
    """LM-O setting of Section V-B."""
    p = Params(n_walk=2, n_iter=5, n_perturb=150, n_keep=10, n_steps=15, omega0=1.0, v0=2.0,
               gamma=0.5, rot_perturb=0.2, trans_perturb=0.1)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def preset_3d3d(**kw) -> Params:
    """3DMatch setting of Section V-B."""
    p = Params(n_walk=2, n_iter=5, n_perturb=150, n_keep=10, n_steps=15, omega0=0.5, v0=0.0,
               gamma=0.5, rot_perturb=0.0, trans_perturb=0.1)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def preset_reg(**kw) -> Params:
    """LM (pose regression) setting of Section V-C: N_W = 20, N_I = 5, N_T = 10, no rotation
    perturbation, no centre velocity."""
    p = Params(n_walk=20, n_iter=5, n_perturb=150, n_keep=10, n_steps=10, omega0=0.5, v0=0.0,
               gamma=0.5, rot_perturb=0.0, trans_perturb=0.1)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def unpack_seeds(seeds):
    seeds = np.asarray(seeds, dtype=np.float64).reshape(-1, 12)
    return seeds[:, :9].reshape(-1, 3, 3), seeds[:, 9:]


@dataclass
class Stats:
    Rbar: np.ndarray
    tbar: np.ndarray
    S: np.ndarray            # PCA velocity scaling (identity for 3D-3D)
    sigma_t: float
    rho_a: float
    r_trans: float           # radius of perturbation(t_p)
    r_rot: float             # radius of perturbation(theta_p)


def center_stats(purse, seeds, params: Params) -> Stats:
    R0, t0 = unpack_seeds(seeds)
    Rbar = proj_so3(R0.sum(axis=0))
    tbar = t0.mean(axis=0)
    a = purse.model
    rho_a = float(np.sqrt(((a - a.mean(axis=0)) ** 2).sum(axis=1).mean()))
    if purse.kind == KIND_REG:
        # translation scale mean beta^t; rotation scale mean beta^R / sqrt(2), the angle of a
        # Frobenius distance (|R - R'|_F = 2 sqrt(2) sin(theta / 2) ~ sqrt(2) theta); written through
        # rho_a so that r_rot = theta_p sigma_t / rho_a is that angle scale times theta_p
        sigma_t = float(purse.radii.mean())
        rho_a = float(sigma_t * np.sqrt(2.0) / purse.radii_rot.mean())
        S = np.eye(3)
    elif purse.kind == KIND_3D3D:
        sigma_t = float(noise_scales(purse).mean())
        S = np.eye(3)
    else:
        fx, fy, _, _ = purse.K
        sigma_t = float(noise_scales(purse).mean() * tbar[2] / (0.5 * (fx + fy)))
        S = pca_scaling(t0, tbar, rho_a)
    if params.perturb_units:
        r_trans, r_rot = params.trans_perturb, params.rot_perturb
    else:
        r_trans = params.trans_perturb * sigma_t
        r_rot = params.rot_perturb * sigma_t / rho_a
    return Stats(Rbar, tbar, S, sigma_t, rho_a, float(r_trans), float(r_rot))


def noise_scales(purse):
    """Radius of each noise region: r_i, or with a noise matrix (eq. 4) the geometric mean
    r_i det(Lambda_i)^(-1/(2d)) of the semi-axes of {e : e^T Lambda_i e <= r_i^2}."""
    lam = getattr(purse, "lam", None)
    if lam is None:
        return np.asarray(purse.radii, dtype=np.float64)
    d = lam.shape[-1]
    return purse.radii * np.linalg.det(lam) ** (-1.0 / (2 * d))


def pca_scaling(t0, tbar, rho_a):
    if t0.shape[0] >= 4:
        d = t0 - tbar
        cov = d.T @ d / t0.shape[0]
        lam, U = np.linalg.eigh(cov)
        sig = np.sqrt(np.maximum(lam, 0.0))
        if sig[-1] > 0:
            return U @ np.diag(sig / sig[-1]) @ U.T
    n = np.linalg.norm(tbar)
    u1 = tbar / n
    ratio = min(1.0, rho_a / n)
    P = np.outer(u1, u1)
    return P + ratio * (np.eye(3) - P)


def init_angular_velocity(R0, Rbar, omega0, seed, walk_ids):
    """omega = omega0 (u + u~), (u, theta) the axis-angle of R_0 R-bar^T."""
    phi = log_so3(R0 @ Rbar.T)
    th = np.linalg.norm(phi, axis=-1)
    u = np.where((th > 1e-9)[..., None], phi / np.where(th > 1e-9, th, 1.0)[..., None], 0.0)
    ut, _ = philox.ball_points(seed, philox.PHASE_OMEGA, 0, 0, walk_ids, unit=True)
    return omega0 * (u + ut)


def init_center_velocity(t0, tbar, v0, S, seed, walk_ids):
    """v = v0 S ((t_0 - t-bar)/|t_0 - t-bar| + v~)."""
    dv = t0 - tbar
    n = np.linalg.norm(dv, axis=-1)
    thr = 1e-9 * (1.0 + np.linalg.norm(tbar))
    dirn = np.where((n > thr)[..., None], dv / np.where(n > thr, n, 1.0)[..., None], 0.0)
    vt, _ = philox.ball_points(seed, philox.PHASE_V, 0, 0, walk_ids, unit=True)
    return v0 * ((dirn + vt) @ S.T)


def top_k_indices(d, k):
    """Indices of the k largest d_j per row; ties go to the lower j."""
    return np.argsort(-d, axis=-1, kind='stable')[..., :k]


def step_ladder(params: Params):
    """Delta T = (1, gamma, ..., gamma^(N_T - 1))."""
    return params.gamma ** np.arange(params.n_steps, dtype=np.float64)


@dataclass
class Candidates:
    d: np.ndarray      # (W, N_P) distances to the boundary of the perturbed poses
    J: np.ndarray      # (W, N_P*) top-k perturbation indices
    Rc: np.ndarray     # rotations of the candidates: (W, N_T, 3, 3) [R] or (W, N_P, 3, 3) [t]
    tc: np.ndarray     # translations: (W, N_P, 3) [R] or (W, N_T, 3) [t]
    I: np.ndarray      # (W, N_P*, N_T) in_purse of candidate (k, m)


def rotation_walk_candidates(purse, R, t, omega, i, walk_ids, seed, params: Params, stats: Stats):
    """One iteration of Alg. 3 up to in_purse."""
    delta = philox.hatbox_points(seed, philox.PHASE_R_PERTURB, i, walk_ids, params.n_perturb)
    tj = t[:, None, :] + stats.r_trans * delta                    # t* + perturbation(t_p)
    d = dist_to_boundary(purse, R[:, None], tj)                   # eq. 11
    J = top_k_indices(d, params.n_keep)
    dT = step_ladder(params)
    Rm = exp_so3(dT[None, :, None] * omega[:, None, :]) @ R[:, None]   # update_rotation
    W = R.shape[0]
    tk = tj[np.arange(W)[:, None], J]                             # t_{j_k}
    I = in_purse(purse, Rm[:, None, :, :, :], tk[:, :, None, :])  # (W, N_P*, N_T)
    return Candidates(d, J, Rm, tj, I)


def translation_walk_candidates(purse, R, t, v, i, walk_ids, seed, params: Params, stats: Stats):
    """One iteration of Alg. 5 up to in_purse."""
    phi = philox.hatbox_points(seed, philox.PHASE_T_PERTURB, i, walk_ids, params.n_perturb)
    Rj = exp_so3(stats.r_rot * phi) @ R[:, None]                  # perturbation(theta_p) R*
    d = dist_to_boundary(purse, Rj, t[:, None])                   # eq. 11
    J = top_k_indices(d, params.n_keep)
    dT = step_ladder(params)
    tm = t[:, None, :] + dT[None, :, None] * v[:, None, :]        # update_translation
    W = R.shape[0]
    Rk = Rj[np.arange(W)[:, None], J]                             # R_{j_k}
    I = in_purse(purse, Rk[:, :, None, :, :], tm[:, None, :, :])  # (W, N_P*, N_T)
    return Candidates(d, J, Rj, tm, I)


def find_farthest(I):
    """m0 = min{m : some k feasible}, k0 = best-ranked feasible k at m0; -1 if none."""
    W = I.shape[0]
    anyk = I.any(axis=1)                      # (W, N_T)
    has = anyk.any(axis=1)
    m0 = np.where(has, np.argmax(anyk, axis=1), -1)
    col = I[np.arange(W), :, np.maximum(m0, 0)]   # (W, N_P*)
    k0 = np.where(has, np.argmax(col, axis=1), -1)
    return m0, k0


def apply_rotation_step(R, t, c: Candidates, m0, k0):
    W = R.shape[0]
    mv = m0 >= 0
    w = np.arange(W)[mv]
    R, t = R.copy(), t.copy()
    R[mv] = c.Rc[w, m0[mv]]
    t[mv] = c.tc[w, c.J[w, k0[mv]]]
    return R, t


def apply_translation_step(R, t, c: Candidates, m0, k0):
    W = R.shape[0]
    mv = m0 >= 0
    w = np.arange(W)[mv]
    R, t = R.copy(), t.copy()
    R[mv] = c.Rc[w, c.J[w, k0[mv]]]
    t[mv] = c.tc[w, m0[mv]]
    return R, t


def start_walks(seeds, walk_ids):
    R0, t0 = unpack_seeds(seeds)
    s = np.asarray(walk_ids) % R0.shape[0]
    return R0[s].copy(), t0[s].copy()


def sample_rotation_boundary(purse, seeds, params: Params, seed: int, walk_ids, stats: Stats | None = None):
    """Alg. 3: returns (R*, t*) of every walk after N_I iterations."""
    walk_ids = np.asarray(walk_ids, dtype=np.int64)
    stats = stats or center_stats(purse, seeds, params)
    R, t = start_walks(seeds, walk_ids)
    omega = init_angular_velocity(R, stats.Rbar, params.omega0, seed, walk_ids)
    for i in range(params.n_iter):
        c = rotation_walk_candidates(purse, R, t, omega, i, walk_ids, seed, params, stats)
        m0, k0 = find_farthest(c.I)
        R, t = apply_rotation_step(R, t, c, m0, k0)
    return R, t


def sample_translation_boundary(purse, seeds, params: Params, seed: int, walk_ids, stats: Stats | None = None):
    """Alg. 5: returns (R*, t*) of every walk after N_I iterations."""
    walk_ids = np.asarray(walk_ids, dtype=np.int64)
    stats = stats or center_stats(purse, seeds, params)
    R, t = start_walks(seeds, walk_ids)
    v = init_center_velocity(t, stats.tbar, params.v0, stats.S, seed, walk_ids)
    for i in range(params.n_iter):
        c = translation_walk_candidates(purse, R, t, v, i, walk_ids, seed, params, stats)
        m0, k0 = find_farthest(c.I)
        R, t = apply_translation_step(R, t, c, m0, k0)
    return R, t


def as_samples(R, t):
    """(q (W,4) with w >= 0, t (W,3)), the layout the library emits."""
    return quat_from_R(R), np.asarray(t, dtype=np.float64)
