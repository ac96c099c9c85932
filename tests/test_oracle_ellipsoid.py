"""Pins of the oracle for noise bounded in the general norm of eq. 4, |e|_Lambda = sqrt(e^T Lambda e)
(CPU only).

* Lambda = I gives the isotropic margins; Lambda = c I scales every residual norm by sqrt(c);
* the norm equals |diag(sqrt(ev)) Q^T e| of an eigendecomposition (an independent formula);
* the synthetic ellipsoidal PURSEs contain their ground truth, and the noise-region draws map a
  unit-ball point u to e = r U^-1 u with e^T Lambda e = r^2 |u|^2 (Lambda = U^T U);
* the octahedral PURSE with one Lambda: its translations form the ellipsoid d^T Lambda d <= r^2,
  so the exact ball of the walk samples stays inside r / sqrt(lambda_min) and comes close to it.
"""
import numpy as np

from oracle import closure, megb as om, purse as op, ransag, so3
from paper_2403_09990_gb300 import synthetic as syn


def test_identity_and_scaled_matrices():
    p = syn.purse_2d3d(16, 2)
    rng = np.random.default_rng(1)
    R = so3.exp_so3(rng.normal(size=(20, 3)) * 0.02) @ p.R_gt
    t = p.t_gt + rng.normal(size=(20, 3)) * 0.005
    h0, f0 = op.residual_norms(p, R, t)
    p.lam = np.repeat(np.eye(2)[None], p.n, axis=0)
    h1, f1 = op.residual_norms(p, R, t)
    assert np.allclose(h0, h1, atol=1e-12) and np.array_equal(f0, f1)
    p.lam = 4.0 * p.lam
    h2, _ = op.residual_norms(p, R, t)
    assert np.allclose(h2, 2.0 * h0, rtol=1e-12)


def test_norm_against_eigendecomposition():
    for maker, d in ((syn.purse_3d3d_ellipsoidal, 3), (syn.purse_2d3d_ellipsoidal, 2)):
        p = maker(seed=4)
        rng = np.random.default_rng(2)
        g = rng.normal(size=(7, p.n, d))
        ev, Q = np.linalg.eigh(p.lam)
        ref = np.linalg.norm(np.sqrt(ev)[None] * np.einsum('nij,kni->knj', Q, g), axis=-1)
        assert np.allclose(op.lam_norm(g, p.lam), ref, rtol=1e-12)
        assert np.all(op.margins(p, p.R_gt, p.t_gt) > 0) and op.in_purse(p, p.R_gt, p.t_gt)


def test_noise_region_draw_identity():
    p = syn.purse_3d3d_ellipsoidal(8, 5)
    rng = np.random.default_rng(3)
    u = rng.normal(size=(8, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True) * 1.3
    U = np.swapaxes(np.linalg.cholesky(p.lam), -1, -2)
    e = p.radii[:, None] * np.linalg.solve(U, u[..., None])[..., 0]
    q = np.einsum('ni,nij,nj->n', e, p.lam, e)
    assert np.allclose(q, p.radii ** 2 * (u ** 2).sum(axis=1), rtol=1e-12)
    seeds, _ = ransag.ransag_3d3d(p, 0, 20000, 64)
    assert len(seeds) > 0
    assert np.all(op.in_purse(p, seeds[:, :9].reshape(-1, 3, 3), seeds[:, 9:]))


def test_ellipsoidal_octahedron_translation_ball():
    p = syn.purse_octahedron_ellipsoidal(seed=3)
    dstar = 0.01 / np.sqrt(np.linalg.eigvalsh(p.lam[0]).min())
    prm = closure.preset_3d3d(v0=0.02, rot_perturb=0.2, n_iter=8)
    R, t = closure.sample_translation_boundary(p, p.seed_pose()[None], prm, 5, np.arange(1000))
    assert np.all(op.in_purse(p, R, t))
    c, d = om.meb_exact_translation(t)
    assert d <= dstar * (1 + 1e-9) and d >= 0.97 * dstar, (d, dstar)
    assert np.linalg.norm(c - p.t_gt) <= 0.05 * dstar
