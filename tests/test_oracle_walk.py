"""Pins of the oracle's boundary samplers (Alg. 2-5) (CPU only).

The octahedral 3D-3D PURSE (model points L(+-e_k), exact observations,
equal radii r) has closed-form balls: pairing +-a_k gives |t - t_g| <= r with
equality reachable, so d* = r, c* = t_g; at t = t_g a rotation by theta about
the unit axis u moves point L e_k by 2 sin(theta/2) L sqrt(1 - (u.e_k)^2), the
largest feasible angle is along a cube diagonal, so
D* = 2 arcsin(r sqrt(6) / (4 L)) with centre R_g.  Prop. 1 says the ball of any
subset of S is no larger; the walks must come close to it (synthetic eta).
A walk that ranks perturbations the wrong way, scans the ladder from the
small end, or skips in_purse fails one of these.
"""
import numpy as np
import pytest

from oracle import closure, megb, purse as op, ransag, so3
from paper_2403_09990_gb300 import synthetic as syn

K = 200


@pytest.fixture(scope="module")
def octa():
    L, r = 0.1, 0.01
    p = syn.purse_octahedron(L, r, 0)
    return p, 2 * np.arcsin(r * np.sqrt(6) / (4 * L)), r


def test_octahedral_rotation_boundary(octa):
    p, Dstar, dstar = octa
    prm = closure.preset_3d3d(n_iter=5)
    R, t = closure.sample_rotation_boundary(p, p.seed_pose()[None], prm, 0, np.arange(512))
    assert op.in_purse(p, R, t).all()
    q, tt = closure.as_samples(R, t)
    C, D, _ = megb.megb_rotation(q, K)
    assert D <= Dstar * (1 + 1 / np.sqrt(K))          # Prop. 1 (+ the GGD bound)
    assert D >= 0.9 * Dstar                             # the walks reach the boundary
    assert so3.dist_quat(C, so3.quat_from_R(p.R_gt)) < 0.2 * Dstar
    c, d, _ = megb.megb_translation(tt, K)
    assert d <= dstar * (1 + 1 / np.sqrt(K))


def test_octahedral_translation_boundary(octa):
    p, Dstar, dstar = octa
    prm = closure.preset_3d3d(n_iter=5, v0=0.02, rot_perturb=0.2)
    R, t = closure.sample_translation_boundary(p, p.seed_pose()[None], prm, 0, np.arange(512))
    assert op.in_purse(p, R, t).all()
    c, d, _ = megb.megb_translation(t, K)
    assert 0.9 * dstar <= d <= dstar * (1 + 1 / np.sqrt(K))
    assert np.linalg.norm(c - p.t_gt) < 0.2 * dstar


def test_walks_spread_beyond_ransag_seeds():
    # Fig. 5 claim: boundary samples enclose a larger ball than the interior seeds
    p = syn.purse_3d3d(8, 0)
    seeds, _ = ransag.ransag_3d3d(p, 0, 40000, 64)
    prm = closure.preset_3d3d()
    R, t = closure.sample_rotation_boundary(p, seeds, prm, 0, np.arange(256))
    assert op.in_purse(p, R, t).all()
    q, _ = closure.as_samples(R, t)
    q0 = so3.quat_from_R(seeds[:, :9].reshape(-1, 3, 3))
    assert megb.megb_rotation(q, K)[1] > 1.2 * megb.megb_rotation(q0, K)[1]


def test_2d3d_samplers_stay_in_purse_and_translation_walk_follows_the_depth_axis():
    p = syn.purse_2d3d(16, 0)
    prm = closure.preset_2d3d()
    w = np.arange(256)
    R, t = closure.sample_rotation_boundary(p, p.seed_pose()[None], prm, 0, w)
    R2, t2 = closure.sample_translation_boundary(p, p.seed_pose()[None], prm, 0, w)
    assert op.in_purse(p, R, t).all() and op.in_purse(p, R2, t2).all()
    # the PURSE is a needle along the viewing ray: the translation sampler
    # spreads much further than the rotation sampler's translations
    d_rot = megb.megb_translation(t, K)[1]
    d_tra = megb.megb_translation(t2, K)[1]
    assert d_tra > 3 * d_rot
    ray = p.t_gt / np.linalg.norm(p.t_gt)
    spread = t2 - t2.mean(0)
    along = np.abs(spread @ ray).max()
    across = np.linalg.norm(spread - np.outer(spread @ ray, ray), axis=1).max()
    assert along > 2 * across


def test_walks_are_reproducible_per_walk_id():
    p = syn.purse_2d3d(16, 1)
    prm = closure.preset_2d3d(n_iter=3)
    seeds = p.seed_pose()[None]
    R, t = closure.sample_rotation_boundary(p, seeds, prm, 7, np.arange(64))
    Rs, ts = closure.sample_rotation_boundary(p, seeds, prm, 7, np.array([5, 33, 60]))
    assert np.array_equal(R[[5, 33, 60]], Rs) and np.array_equal(t[[5, 33, 60]], ts)
    R3, _ = closure.sample_rotation_boundary(p, seeds, prm, 8, np.arange(64))
    assert not np.allclose(R3, R)


def test_find_farthest_and_top_k_semantics():
    I = np.zeros((3, 4, 5), bool)
    I[0, 3, 2] = I[0, 1, 4] = I[0, 2, 2] = True      # m0 = 2, best-ranked feasible k = 2
    I[2, 0, 0] = True
    m0, k0 = closure.find_farthest(I)
    assert list(m0) == [2, -1, 0] and list(k0) == [2, -1, 0]
    d = np.array([[0.5, 2.0, 2.0, -1.0, 3.0, 2.0]])
    assert list(closure.top_k_indices(d, 4)[0]) == [4, 1, 2, 5]
