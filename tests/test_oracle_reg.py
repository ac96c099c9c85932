"""Pins of the oracle for the pose-regression PURSE (Example 3, eq. PURSEreg), CPU only.

* margins: the Frobenius distance of two rotations is 2 sqrt(2) sin(theta / 2) of their
  geodesic angle theta (an independent formula), translations are plain distances;
* the ground truth lies in the synthetic PURSE;
* the convex-combination sampler: weights on the simplex with the Dirichlet(1) moments,
  seeds inside the PURSE in trial order;
* nested hypotheses: the PURSE is one rotation ball of angle 2 asin(beta / (2 sqrt 2)) and
  one translation ball, so the exact balls of the walk samples lie inside them (Prop. 1),
  the rotation ball close to it, and every sample is in the PURSE; the dS_t walks fill the
  translation ball the same way.
"""
import numpy as np

from oracle import closure, megb as om, purse as op, ransag, so3
from paper_2403_09990_gb300 import synthetic as syn


def test_regression_margins_against_geodesic_angles():
    p = syn.purse_reg(10, 3)
    rng = np.random.default_rng(0)
    R = so3.exp_so3(rng.normal(size=(50, 3)) * 0.05) @ p.R_gt
    t = p.t_gt + rng.normal(size=(50, 3)) * 0.01
    m = op.margins(p, R, t)
    assert m.shape == (50, 20)
    for k in range(50):
        ang = np.array([so3.dist_so3(Ri, R[k]) for Ri in p.rot_hyp])
        assert np.allclose(m[k, :10], p.radii_rot - 2 * np.sqrt(2) * np.sin(ang / 2), atol=1e-12)
        assert np.allclose(m[k, 10:], p.radii - np.linalg.norm(t[k] - p.obs, axis=1), atol=1e-15)
    assert np.all(op.margins(p, p.R_gt, p.t_gt) > 0)
    assert op.in_purse(p, p.R_gt, p.t_gt)


def test_simplex_weights_and_convex_seeds():
    p = syn.purse_reg(10, 0)
    w = ransag.simplex_weights(0, np.arange(50000), 10)
    assert np.all(w > 0) and np.allclose(w.sum(axis=1), 1.0)
    assert np.allclose(w.mean(axis=0), 0.1, atol=3e-3)
    assert abs((w ** 2).mean() - 2.0 / (10 * 11)) < 1e-3          # Dirichlet(1): E w_i^2 = 2 / (n (n + 1))
    seeds, acc = ransag.convex_seeds(p, 0, 5000, 300)
    assert len(seeds) == 300 and np.all(np.diff(acc) > 0)
    R = seeds[:, :9].reshape(-1, 3, 3)
    assert np.allclose(R @ np.swapaxes(R, 1, 2), np.eye(3), atol=1e-12)
    assert np.all(op.in_purse(p, R, seeds[:, 9:]))


def test_nested_hypotheses_closed_form_balls():
    p = syn.purse_reg_nested(10, 0, beta_rot=0.04, beta_t=0.006)
    Dstar = 2 * np.arcsin(0.04 / (2 * np.sqrt(2)))
    prm = closure.preset_reg()
    seeds, _ = ransag.convex_seeds(p, 0, 5000, 50)
    R, t = closure.sample_rotation_boundary(p, seeds, prm, 5, np.arange(600))
    assert np.all(op.in_purse(p, R, t))
    q, tt = closure.as_samples(R, t)
    C, D = om.meb_exact_rotation(q, q[0])
    c, d = om.meb_exact_translation(tt)
    assert D <= Dstar * (1 + 1e-9) and D >= 0.97 * Dstar, (D, Dstar)
    assert so3.dist_quat(C, so3.quat_from_R(p.R_gt)) <= 0.05 * Dstar
    assert d <= 0.006 * (1 + 1e-9) and np.linalg.norm(c - p.t_gt) <= 0.006


def test_nested_hypotheses_translation_walks():
    """The dS_t sampler on the nested PURSE: the translations fill one ball of radius beta_t around
    t_gt, so the exact ball of the walk samples lies inside it and comes close to it (Prop. 1), and
    every sample keeps its rotation within the rotation ball."""
    p = syn.purse_reg_nested(10, 1, beta_rot=0.04, beta_t=0.006)
    prm = closure.preset_reg(rot_perturb=0.2, v0=0.02)
    seeds, _ = ransag.convex_seeds(p, 2, 5000, 50)
    R, t = closure.sample_translation_boundary(p, seeds, prm, 9, np.arange(600))
    assert np.all(op.in_purse(p, R, t))
    c, d = om.meb_exact_translation(t)
    assert d <= 0.006 * (1 + 1e-9) and d >= 0.97 * 0.006, d
    assert np.linalg.norm(c - p.t_gt) <= 0.05 * 0.006
