"""Pins of the oracle's PURSE constraints (CPU only).

The generator draws each observation as the ground-truth image of a keypoint
plus a noise vector inside the ball (or disk) of radius r_i; the oracle's
residual at the ground-truth pose must therefore be exactly that noise, and
the ground truth must lie in the PURSE.  Frame changes leave the residuals
unchanged, the SE(3) gradient matches central differences.
"""
import numpy as np
import pytest

from oracle import purse as op
from oracle import so3
from paper_2403_09990_gb300 import synthetic as syn


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ground_truth_in_purse_3d3d(seed):
    p = syn.purse_3d3d(8, seed)
    m = op.margins(p, p.R_gt, p.t_gt)
    assert np.all(m > 0)
    assert op.in_purse(p, p.R_gt, p.t_gt)
    # the residual norm at the ground truth is the drawn noise norm
    h, _ = op.residual_norms(p, p.R_gt, p.t_gt)
    noise = p.obs - (p.model @ p.R_gt.T + p.t_gt)
    assert np.allclose(h, np.linalg.norm(noise, axis=1), atol=1e-15)
    assert np.all(np.linalg.norm(noise, axis=1) < p.radii)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ground_truth_in_purse_2d3d(seed):
    p = syn.purse_2d3d(16, seed)
    assert op.in_purse(p, p.R_gt, p.t_gt)
    fx, fy, cx, cy = p.K
    X = p.model @ p.R_gt.T + p.t_gt
    pix = np.stack([fx * X[:, 0] / X[:, 2] + cx, fy * X[:, 1] / X[:, 2] + cy], 1)
    h, front = op.residual_norms(p, p.R_gt, p.t_gt)
    assert front.all()
    assert np.allclose(h, np.linalg.norm(p.obs - pix, axis=1), atol=1e-9)
    # a far-away translation leaves the PURSE; a pose behind the camera violates every constraint
    assert not op.in_purse(p, p.R_gt, p.t_gt + np.array([0.5, 0, 0]))
    m = op.margins(p, p.R_gt, p.t_gt * np.array([1, 1, -1]))
    assert np.all(np.isneginf(m))
    assert op.dist_to_boundary(p, p.R_gt, -p.t_gt) == -np.inf


def test_margins_invariant_under_frame_change():
    rng = np.random.default_rng(3)
    R = so3.exp_so3(rng.normal(size=3))
    t = rng.normal(size=3) * 0.01
    for p in [syn.purse_3d3d(8, 4), syn.purse_2d3d(16, 4)]:
        Rp = p.R_gt @ so3.exp_so3(rng.normal(size=3) * 0.01)
        tp = p.t_gt + rng.normal(size=3) * 0.003
        m0 = op.margins(p, Rp, tp)
        # model frame change Z' = Q Z + s with R' = R Q^T, t' = t - R Q^T s
        Q = so3.exp_so3(rng.normal(size=3))
        s = rng.normal(size=3)
        p2 = syn.Purse(p.kind, p.model @ Q.T + s, p.obs, p.radii, p.K)
        m1 = op.margins(p2, Rp @ Q.T, tp - Rp @ Q.T @ s)
        assert np.allclose(m0, m1, atol=1e-9)
        if p.kind == syn.KIND_3D3D:
            # world frame change b' = G b + g with R' = G R, t' = G t + g
            p3 = syn.Purse(p.kind, p.model, p.obs @ R.T + t, p.radii)
            assert np.allclose(op.margins(p3, R @ Rp, R @ tp + t), m0, atol=1e-12)


def test_dist_and_membership_consistent():
    p = syn.purse_2d3d(16, 5)
    rng = np.random.default_rng(5)
    Rs = so3.exp_so3(rng.normal(size=(500, 3)) * 0.02) @ p.R_gt
    ts = p.t_gt + rng.normal(size=(500, 3)) * np.array([0.003, 0.003, 0.03])
    d = op.dist_to_boundary(p, Rs, ts)
    assert np.array_equal(d >= 0, op.in_purse(p, Rs, ts))
    assert 0 < (d >= 0).mean() < 1


@pytest.mark.parametrize("kind,lam", [(0, False), (1, False), (0, True), (1, True)])
def test_gradient_matches_central_differences(kind, lam):
    if lam:
        p = syn.purse_3d3d_ellipsoidal(8, 6) if kind == 0 else syn.purse_2d3d_ellipsoidal(16, 6)
    else:
        p = syn.purse_3d3d(8, 6) if kind == 0 else syn.purse_2d3d(16, 6)
    rng = np.random.default_rng(7)
    R = so3.exp_so3(rng.normal(size=3) * 0.01) @ p.R_gt
    t = p.t_gt + rng.normal(size=3) * 0.002
    G = op.margin_gradient(p, R, t)
    h = 1e-6
    fd = np.zeros_like(G)
    for c in range(6):
        e = np.zeros(6)
        e[c] = h
        hp, _ = op.residual_norms(p, so3.exp_so3(e[:3]) @ R, t + e[3:])
        hm, _ = op.residual_norms(p, so3.exp_so3(-e[:3]) @ R, t - e[3:])
        fd[:, c] = (hp - hm) / (2 * h)
    scale = np.abs(fd).max()
    assert np.abs(G - fd).max() < 1e-6 * scale + 1e-9
