"""Pins of the oracle's walk initialisation and of its samplers on the unit-ball toy (CPU only).

Section IV Step II ("walk away from the center") fixes the start velocities:
omega = omega0 (u + u~), (u, theta) the axis-angle of the relative rotation of R_0 against
R-bar, and v = v0 ((t_0 - t-bar)/|t_0 - t-bar| + v~), u~ and v~ random unit vectors, so that
the walks point away from the centre of the seeds.  The appendix on the dS_t sampler rescales
v by the PCA of the seed translations, whose first weight vector lies along the longest axis
of S_t.  The checks below build the geometry with scipy (not with the oracle's SO(3) helpers)
and test what these definitions imply:
* omega / omega0 - u and v / v0 - dir are unit vectors for every walk, and their mean
  projections on u and on dir are 1 (E[u~ . u] = 0): a flipped sign gives -1, a body-frame
  axis (R-bar^T R_0) gives u . R-bar^T u;
* moving along omega (left multiplication, the update of Alg. 2) increases the geodesic
  distance to R-bar at rate omega0 on average; moving along v increases |t - t-bar| at rate v0;
* with >= 4 seeds drawn from an anisotropic Gaussian the scaling S has the covariance axes
  as eigenvectors and the ratios sigma_k / sigma_1 as eigenvalues (within sampling error);
  with fewer seeds its longest axis is the viewing ray (the needle direction of a 2D-3D
  PURSE).
The appendix's intuitive example (unit ball; "R" the in-plane coordinates, "t" the axis
coordinate) runs the oracle's rotation and translation samplers on that toy set: the
rotation sampler pushes the in-plane radius to 1, the translation sampler pushes |z| to 1.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.stats import special_ortho_group

from oracle import closure

N_WALK = 20000


def _unit(x):
    x = np.asarray(x, dtype=np.float64)
    return x / np.linalg.norm(x)


@pytest.fixture(scope="module")
def rel_rotation():
    rng = np.random.default_rng(11)
    Rbar = Rotation.from_rotvec([0.9, -1.4, 0.6]).as_matrix()
    u = _unit(rng.normal(size=3))
    theta = 0.35
    R0 = Rotation.from_rotvec(theta * u).as_matrix() @ Rbar   # R_0 R-bar^T = Exp(theta u)
    return Rbar, R0, u, theta


def test_angular_velocity_points_away_from_the_mean_rotation(rel_rotation):
    Rbar, R0, u, theta = rel_rotation
    omega0 = 0.7
    w = np.arange(N_WALK)
    om = closure.init_angular_velocity(np.broadcast_to(R0, (N_WALK, 3, 3)), Rbar, omega0, 5, w)
    rnd = om / omega0 - u
    assert np.allclose(np.linalg.norm(rnd, axis=1), 1.0, atol=1e-12)      # u~ is a unit vector
    proj = (om / omega0) @ u
    se = np.sqrt(1.0 / 3.0 / N_WALK)
    assert abs(proj.mean() - 1.0) < 5 * se                                  # E[(u + u~) . u] = 1
    # a body-frame axis (R-bar^T R_0) would project on u by u . R-bar^T u, far from 1 here
    assert abs(u @ (Rbar.T @ u) - 1.0) > 0.1
    # the random part is isotropic: its mean vanishes
    assert np.linalg.norm(rnd.mean(axis=0)) < 5 * se
    # walking along omega (R <- Exp(tau omega) R) moves away from R-bar at rate omega0
    tau = 1e-4
    d0 = np.linalg.norm(Rotation.from_matrix(R0 @ Rbar.T).as_rotvec())
    Rt = Rotation.from_rotvec(tau * om) * Rotation.from_matrix(R0)
    d1 = np.linalg.norm((Rt * Rotation.from_matrix(Rbar).inv()).as_rotvec(), axis=1)
    rate = (d1 - d0) / tau
    assert abs(d0 - theta) < 1e-12
    assert abs(rate.mean() - omega0) < 5 * omega0 * se + 1e-3


def test_angular_velocity_at_the_centre_is_a_random_unit_vector():
    R = Rotation.from_rotvec([0.2, 0.1, -0.3]).as_matrix()
    om = closure.init_angular_velocity(np.broadcast_to(R, (4096, 3, 3)), R, 1.3, 2, np.arange(4096))
    assert np.allclose(np.linalg.norm(om, axis=1), 1.3, atol=1e-12)
    assert np.linalg.norm(om.mean(axis=0)) < 5 * 1.3 * np.sqrt(1.0 / 3.0 / 4096)


def test_center_velocity_points_away_from_the_mean_translation():
    rng = np.random.default_rng(3)
    tbar = np.array([0.1, -0.2, 0.9])
    d = _unit(rng.normal(size=3))
    t0 = tbar + 0.03 * d
    v0 = 1.7
    w = np.arange(N_WALK)
    v = closure.init_center_velocity(np.broadcast_to(t0, (N_WALK, 3)), tbar, v0, np.eye(3), 9, w)
    assert np.allclose(np.linalg.norm(v / v0 - d, axis=1), 1.0, atol=1e-12)
    se = np.sqrt(1.0 / 3.0 / N_WALK)
    assert abs(((v / v0) @ d).mean() - 1.0) < 5 * se
    # |t - t-bar| grows at rate v0 on average along v
    tau = 1e-6
    rate = (np.linalg.norm(t0 + tau * v - tbar, axis=1) - 0.03) / tau
    assert abs(rate.mean() - v0) < 5 * v0 * se + 1e-3
    # with a scaling S the velocity is S (dir + v~): S^-1 v / v0 - dir is a unit vector
    Q = special_ortho_group.rvs(3, random_state=4)
    S = Q @ np.diag([1.0, 0.4, 0.1]) @ Q.T
    vs = closure.init_center_velocity(np.broadcast_to(t0, (N_WALK, 3)), tbar, v0, S, 9, w)
    back = np.linalg.solve(S, (vs / v0).T).T
    assert np.allclose(np.linalg.norm(back - d, axis=1), 1.0, atol=1e-9)
    assert abs((back @ d).mean() - 1.0) < 5 * se


def test_pca_scaling_follows_the_seed_covariance():
    rng = np.random.default_rng(21)
    U = special_ortho_group.rvs(3, random_state=22)
    sig = np.array([0.05, 0.02, 0.008])
    n = 40000
    tbar = np.array([0.05, -0.03, 1.1])
    t0 = tbar + (rng.normal(size=(n, 3)) * sig) @ U.T
    S = closure.pca_scaling(t0, t0.mean(axis=0), 0.1)
    lam, V = np.linalg.eigh(S)
    lam, V = lam[::-1], V[:, ::-1]
    # eigenvalues sigma_k / sigma_1 within the sampling error of n Gaussian seeds (~1 %)
    assert np.allclose(lam, sig / sig[0], rtol=0.03), lam
    # eigenvectors along the covariance axes; the first along the longest axis
    assert np.all(np.abs(np.sum(V * U, axis=0)) > 0.999), np.sum(V * U, axis=0)
    # a velocity drawn isotropically then scaled favours the longest axis (the mean |cosine| to
    # a fixed axis is 1/2 for isotropic directions)
    g = rng.normal(size=(4096, 3))
    gs = g @ S.T
    share = np.abs(gs @ U[:, 0]) / np.linalg.norm(gs, axis=1)
    assert share.mean() > 0.7


def test_pca_scaling_with_few_seeds_is_longest_along_the_viewing_ray():
    tbar = np.array([0.12, -0.05, 0.8])
    seeds = tbar + np.array([[0.0, 0.0, 0.0], [1e-3, 0.0, 0.0], [0.0, 2e-3, 1e-3]])
    rho_a = 0.09
    S = closure.pca_scaling(seeds, seeds.mean(axis=0), rho_a)
    lam, V = np.linalg.eigh(S)
    ray = _unit(seeds.mean(axis=0))
    assert abs(abs(V[:, -1] @ ray) - 1.0) < 1e-12
    assert abs(lam[-1] - 1.0) < 1e-12
    assert np.all(lam[:2] < 0.5)


# --------------------------------------------------------------------------- unit-ball toy walk
# The appendix's intuitive example: S = {x^2 + y^2 + z^2 <= 1}, the "rotation" part is (x, y)
# and the "translation" part is z.  It is embedded in poses as (x, y) = the first two components
# of Log(R) and z = t_z; a walk from R = I with angular velocity omega keeps Log(R) = alpha omega,
# so (x, y) = alpha omega_xy as long as alpha |omega| < pi.

def _toy_xyz(R, t):
    R, t = np.broadcast_arrays(np.asarray(R, dtype=np.float64), np.asarray(t, dtype=np.float64)[..., None])
    t = t[..., 0]
    rv = Rotation.from_matrix(R.reshape(-1, 3, 3)).as_rotvec().reshape(R.shape[:-2] + (3,))
    return rv[..., 0], rv[..., 1], t[..., 2]


def _toy_dist(purse, R, t):
    x, y, z = _toy_xyz(R, t)
    return 1.0 - np.sqrt(x * x + y * y + z * z)


def _toy_in(purse, R, t):
    x, y, z = _toy_xyz(R, t)
    return x * x + y * y + z * z <= 1.0


def _toy_stats(r_trans, r_rot):
    return closure.Stats(Rbar=np.eye(3), tbar=np.zeros(3), S=np.eye(3), sigma_t=1.0, rho_a=1.0,
                         r_trans=r_trans, r_rot=r_rot)


def test_unit_ball_toy_rotation_sampler(monkeypatch):
    monkeypatch.setattr(closure, "dist_to_boundary", _toy_dist)
    monkeypatch.setattr(closure, "in_purse", _toy_in)
    prm = closure.Params(n_walk=1, n_iter=20, n_perturb=150, n_keep=10, n_steps=15, omega0=1.0, v0=0.0,
                         gamma=0.5, rot_perturb=0.0, trans_perturb=0.1)
    w = np.arange(256)
    seeds = np.concatenate([np.eye(3).ravel(), np.zeros(3)])[None]
    om = closure.init_angular_velocity(np.broadcast_to(np.eye(3), (256, 3, 3)), np.eye(3), 1.0, 4, w)
    R, t = closure.sample_rotation_boundary(None, seeds, prm, 4, w, stats=_toy_stats(0.1, 0.0))
    x, y, z = _toy_xyz(R, t)
    rho = np.hypot(x, y)
    assert np.all(x * x + y * y + z * z <= 1.0)
    keep = np.hypot(om[:, 0], om[:, 1]) > 0.6       # walks whose alpha stays below pi
    assert keep.sum() > 100
    # Step 1 keeps |z| small (perturbations that drag away from the boundary), Step 2 pushes the
    # in-plane radius to the boundary of the "R" set
    assert rho[keep].min() > 0.95 and np.median(rho[keep]) > 0.99, np.sort(rho[keep])[:5]
    assert np.median(np.abs(z[keep])) < 0.1


def test_unit_ball_toy_translation_sampler(monkeypatch):
    monkeypatch.setattr(closure, "dist_to_boundary", _toy_dist)
    monkeypatch.setattr(closure, "in_purse", _toy_in)
    prm = closure.Params(n_walk=1, n_iter=20, n_perturb=150, n_keep=10, n_steps=15, omega0=0.0, v0=1.0,
                         gamma=0.5, rot_perturb=0.1, trans_perturb=0.0, perturb_units=1)
    w = np.arange(256)
    seeds = np.concatenate([np.eye(3).ravel(), np.zeros(3)])[None]
    v = closure.init_center_velocity(np.zeros((256, 3)), np.zeros(3), 1.0, np.eye(3), 6, w)
    R, t = closure.sample_translation_boundary(None, seeds, prm, 6, w, stats=_toy_stats(0.0, 0.1))
    x, y, z = _toy_xyz(R, t)
    assert np.all(x * x + y * y + z * z <= 1.0)
    keep = np.abs(v[:, 2]) > 0.5
    assert keep.sum() > 50
    assert np.abs(z[keep]).min() > 0.95 and np.median(np.abs(z[keep])) > 0.99, np.sort(np.abs(z[keep]))[:5]
    assert np.median(np.hypot(x[keep], y[keep])) < 0.1
