"""Pins of the oracle's ball solvers (CPU only).

* exact ball: Welzl's recursion equals brute force over support sets;
  the ball of a rectangle's corners is its circumcircle (Fig. 2 example);
* translation GGD (Badoiu-Clarkson): r* <= d_K <= (1 + 1/sqrt(K)) r* and
  |c_K - c*| <= r*/sqrt(K) against the exact ball;
* rotation GGD: on samples along one geodesic the ball is known in closed
  form (centre at the middle of the arc, radius half its length) and the
  one-dimensional Badoiu-Clarkson bound holds; on the six rotations
  Exp(+-theta e_k) C the centre is C and the radius theta;
* invariants: containment, diam/2 <= radius <= diam, sign invariance.
"""
import numpy as np
import pytest

from oracle import megb, so3

rng = np.random.default_rng(11)


@pytest.mark.parametrize("dim,n", [(2, 7), (3, 9), (4, 9), (3, 3)])
def test_welzl_equals_bruteforce(dim, n):
    for trial in range(5):
        P = rng.normal(size=(n, dim))
        c1, r1 = megb.welzl_meb(P)
        c2, r2 = megb.meb_bruteforce(P)
        assert abs(r1 - r2) < 1e-10 * max(1, r2)
        assert np.allclose(c1, c2, atol=1e-9)
        assert np.all(np.linalg.norm(P - c1, axis=1) <= r1 + 1e-12)


def test_rectangle_corners():
    w, h = 3.0, 1.0
    P = np.array([[0, 0, 0], [w, 0, 0], [0, h, 0], [w, h, 0]], float) + 5.0
    c, r = megb.welzl_meb(P)
    assert np.allclose(c, [w / 2 + 5, h / 2 + 5, 5])
    assert abs(r - 0.5 * np.hypot(w, h)) < 1e-12
    for K in [10, 100, 1000]:
        cK, dK, _ = megb.megb_translation(P, K)
        assert r - 1e-12 <= dK <= r * (1 + 1 / np.sqrt(K))


@pytest.mark.parametrize("n", [20, 200, 2000])
def test_translation_ggd_badoiu_clarkson_bound(n):
    P = rng.normal(size=(n, 3)) * np.array([0.01, 0.02, 0.05]) + rng.normal(size=3)
    cs, rs = megb.welzl_meb(P)
    for K in [1, 10, 50, 200]:
        cK, dK, f = megb.megb_translation(P, K)
        assert rs * (1 - 1e-12) <= dK <= rs * (1 + 1 / np.sqrt(K)) + 1e-15
        assert np.linalg.norm(cK - cs) <= rs / np.sqrt(K) + 1e-15
        # containment and the farthest points are real samples
        assert np.all(np.linalg.norm(P - cK, axis=1) <= dK + 1e-15)
        assert f.min() >= 0 and f.max() < n
    diam = max(np.linalg.norm(P - p, axis=1).max() for p in P)
    assert diam / 2 - 1e-15 <= dK <= diam


def test_rotation_ggd_on_one_geodesic():
    C0 = so3.quat_from_R(so3.exp_so3(rng.normal(size=3)))
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    ang = rng.uniform(-0.4, 0.9, 300)
    qs = so3.quat_mul(so3.quat_exp(ang[:, None] * u), C0[None])
    mid, half = 0.5 * (ang.max() + ang.min()), 0.5 * (ang.max() - ang.min())
    Cstar = so3.quat_mul(so3.quat_exp(mid * u), C0)
    for K in [1, 10, 100, 400]:
        C, D, f = megb.megb_rotation(qs, K)
        assert half * (1 - 1e-12) <= D <= half * (1 + 1 / np.sqrt(K)) + 1e-12
        assert so3.dist_quat(C, Cstar) <= half / np.sqrt(K) + 1e-12


def test_rotation_ggd_octahedral_configuration():
    C0 = so3.quat_from_R(so3.exp_so3(rng.normal(size=3)))
    theta = 0.2
    axes = np.concatenate([np.eye(3), -np.eye(3)])
    qs = so3.quat_mul(so3.quat_exp(theta * axes), C0[None])
    qs = np.concatenate([qs, so3.quat_mul(so3.quat_exp(rng.normal(size=(50, 3)) * 0.03), C0[None])])
    K = 400
    C, D, f = megb.megb_rotation(qs, K)
    assert theta * (1 - 1e-12) <= D <= theta * (1 + 1 / np.sqrt(K))
    assert so3.dist_quat(C, C0) <= theta / np.sqrt(K)


def test_rotation_ggd_invariants_and_sign_invariance():
    C0 = so3.quat_from_R(so3.exp_so3(rng.normal(size=3)))
    qs = so3.quat_mul(so3.quat_exp(rng.normal(size=(500, 3)) * np.array([0.02, 0.05, 0.1])), C0[None])
    C, D, f = megb.megb_rotation(qs, 200)
    d = so3.dist_quat(C[None], qs)
    assert np.all(d <= D + 1e-15)
    diam = max(so3.dist_quat(q[None], qs).max() for q in qs)
    assert diam / 2 <= D <= diam
    flip = qs * np.where(rng.random(len(qs)) < 0.5, -1.0, 1.0)[:, None]
    C2, D2, f2 = megb.megb_rotation(flip, 200)
    assert np.array_equal(f, f2) and abs(D - D2) < 1e-14
    # near-flat cluster: the ball of the quaternions in R^4 (Step III embedding)
    # projected to the sphere is a centre no better than the GGD one by more than the bound
    cw, rw = megb.welzl_meb(megb.canonical(qs))
    cw /= np.linalg.norm(cw)
    Dw = so3.dist_quat(cw[None], qs).max()
    assert D <= Dw * (1 + 1 / np.sqrt(200))
    assert Dw <= D * (1 + 1 / np.sqrt(200))


def test_replay_reproduces_free_run():
    qs = so3.quat_from_R(so3.exp_so3(rng.normal(size=(100, 3)) * 0.1))
    C, D, f = megb.megb_rotation(qs, 50)
    Cs = megb.megb_rotation_replay(qs, f)
    assert np.allclose(Cs[-1], C, atol=1e-15)
    ts = rng.normal(size=(100, 3))
    c, d, g = megb.megb_translation(ts, 50)
    assert np.allclose(megb.megb_translation_replay(ts, g)[-1], c, atol=1e-15)


def test_exact_translation_ball_closed_forms_and_jung():
    # rectangle corners: the circumcircle; random clouds: brute force, diam/2 <= r <= diam sqrt(3/8)
    w, h = 2.0, 0.5
    P = np.array([[0, 0, 0], [w, 0, 0], [0, h, 0], [w, h, 0]], float) - 1.0
    c, r = megb.meb_exact_translation(P)
    assert np.allclose(c, [w / 2 - 1, h / 2 - 1, -1]) and abs(r - 0.5 * np.hypot(w, h)) < 1e-12
    for _ in range(5):
        P = rng.normal(size=(10, 3)) * np.array([0.01, 0.03, 0.02])
        c, r = megb.meb_exact_translation(P)
        c2, r2 = megb.meb_bruteforce(P)
        assert abs(r - r2) < 1e-12 and np.allclose(c, c2, atol=1e-10)
        diam = max(np.linalg.norm(P - p, axis=1).max() for p in P)
        assert diam / 2 - 1e-15 <= r <= diam * np.sqrt(3 / 8) + 1e-15


def test_exact_rotation_ball_closed_forms():
    C0 = so3.quat_from_R(so3.exp_so3(rng.normal(size=3)))
    # six rotations Exp(+-theta e_k) C0 plus interior ones: centre C0, radius theta (by symmetry)
    theta = 0.3
    axes = np.concatenate([np.eye(3), -np.eye(3)])
    qs = so3.quat_mul(so3.quat_exp(theta * axes), C0[None])
    qs = np.concatenate([qs, so3.quat_mul(so3.quat_exp(rng.normal(size=(40, 3)) * 0.02), C0[None])])
    C, D = megb.meb_exact_rotation(qs, qs[0])
    assert so3.dist_quat(C, C0) < 1e-10 and abs(D - theta) < 1e-10
    # samples along one geodesic: the middle of the arc, half its length
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    ang = rng.uniform(-0.5, 0.8, 200)
    qs = so3.quat_mul(so3.quat_exp(ang[:, None] * u), C0[None])
    C, D = megb.meb_exact_rotation(qs, qs[0])
    mid, half = 0.5 * (ang.max() + ang.min()), 0.5 * (ang.max() - ang.min())
    assert so3.dist_quat(C, so3.quat_mul(so3.quat_exp(mid * u), C0)) < 1e-9 and abs(D - half) < 1e-10


def test_exact_rotation_ball_sign_and_left_invariance():
    C0 = so3.quat_from_R(so3.exp_so3(rng.normal(size=3)))
    qs = so3.quat_mul(so3.quat_exp(rng.normal(size=(300, 3)) * np.array([0.03, 0.05, 0.1])), C0[None])
    C, D = megb.meb_exact_rotation(qs, qs[0])
    flip = qs * np.where(rng.random(len(qs)) < 0.5, -1.0, 1.0)[:, None]
    C2, D2 = megb.meb_exact_rotation(flip, qs[5])
    assert so3.dist_quat(C, C2) < 1e-12 and abs(D - D2) < 1e-12
    G = so3.quat_from_R(so3.exp_so3(rng.normal(size=3)))
    C3, D3 = megb.meb_exact_rotation(so3.quat_mul(G[None], qs), G)
    assert so3.dist_quat(C3, so3.quat_mul(G, C)) < 1e-10 and abs(D3 - D) < 1e-12
    # never worse than the geodesic-descent ball by more than its (1 + 1/sqrt K) bound
    Cg, Dg, _ = megb.megb_rotation(qs, 400)
    assert D <= Dg * (1 + 1e-9) and Dg <= D * (1 + 1 / np.sqrt(400))


def _random_quats(rng, n, spread):
    v = rng.normal(size=(n, 3)) * spread
    q = np.array([so3.quat_exp(x) for x in v])
    return q * np.where(q[:, :1] < 0, -1.0, 1.0)


def test_mean_output_rule_with_one_iterate_is_the_plain_descent():
    rng = np.random.default_rng(5)
    qs, ts = _random_quats(rng, 300, 0.2), rng.normal(size=(300, 3))
    C, D, f = megb.megb_rotation(qs, 50)
    Cm, Dm, fm = megb.megb_rotation_mean(qs, 50, 1)
    assert np.array_equal(f, fm) and np.allclose(C, Cm, atol=1e-14) and abs(D - Dm) < 1e-14
    c, d, g = megb.megb_translation(ts, 50)
    cm, dm, gm = megb.megb_translation_mean(ts, 50, 1)
    assert np.array_equal(g, gm) and np.allclose(c, cm, atol=1e-14) and abs(d - dm) < 1e-14


def test_mean_output_rule_projection_equals_quaternion_eigenvector():
    # proj_SO3(sum R(q_t)) maximises trace(R(p)^T sum R(q_t)) = sum (4 (p.q_t)^2 - 1) over unit p, so
    # its quaternion is the principal eigenvector of sum q_t q_t^T (Horn's identity, no SVD)
    rng = np.random.default_rng(6)
    qs = _random_quats(rng, 500, 0.3)
    K, n_last = 60, 10
    C, D, f = megb.megb_rotation_mean(qs, K, n_last)
    Cs = megb.megb_rotation_replay(qs, f)[K - n_last + 1:]
    w, V = np.linalg.eigh(Cs.T @ Cs)
    e = V[:, -1] * (1.0 if V[0, -1] >= 0 else -1.0)
    assert np.abs(C - e).max() < 1e-12
    assert abs(D - so3.dist_quat(C[None], megb.canonical(qs)).max()) < 1e-14
    # an enclosing ball: at least half the largest pairwise distance
    diam = max(so3.dist_quat(q[None], megb.canonical(qs)).max() for q in megb.canonical(qs)[:100])
    assert D >= 0.5 * diam - 1e-12


def test_mean_output_rule_two_samples_closed_form():
    # two samples a, b: C_0 = a, C_1 = b, C_2 = their geodesic midpoint; the three are symmetric about
    # the midpoint, so the mean of the last three is the midpoint and the radius half the distance
    a = so3.quat_exp(np.array([0.3, -0.1, 0.2]))
    b = so3.quat_exp(np.array([-0.2, 0.25, 0.05]))
    qs = megb.canonical(np.stack([a, b]))
    C, D, _ = megb.megb_rotation_mean(qs, 2, 3)
    mid = megb.canonical(so3.slerp(qs[0], qs[1], 0.5))
    th = so3.dist_quat(qs[0][None], qs[1][None])[0]
    assert np.abs(C - mid).max() < 1e-13 and abs(D - 0.5 * th) < 1e-13
    ts = np.array([[0.1, 0.2, 0.3], [-0.5, 0.4, 1.0]])
    c, d, _ = megb.megb_translation_mean(ts, 2, 3)
    assert np.abs(c - ts.mean(0)).max() < 1e-15 and abs(d - 0.5 * np.linalg.norm(ts[1] - ts[0])) < 1e-15
    # more iterates requested than exist: all of C_0 .. C_K
    c2, _, _ = megb.megb_translation_mean(ts, 2, 10)
    assert np.abs(c2 - ts.mean(0)).max() < 1e-15
