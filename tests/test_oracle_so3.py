"""Pins of the oracle's rotation helpers against closed forms and library routines."""
import numpy as np
import scipy.linalg
import scipy.spatial.transform as sst

from oracle import so3

rng = np.random.default_rng(0)


def rand_rot(n):
    return sst.Rotation.random(n, random_state=1).as_matrix()


def test_exp_matches_matrix_exponential():
    for v in rng.normal(size=(20, 3)) * rng.uniform(0, 3, (20, 1)):
        assert np.allclose(so3.exp_so3(v), scipy.linalg.expm(so3.hat(v)), atol=1e-13)


def test_exp_log_round_trip_including_edges():
    axes = rng.normal(size=(6, 3))
    axes /= np.linalg.norm(axes, axis=1, keepdims=True)
    for th in [0.0, 1e-12, 1e-7, 1e-3, 1.0, 3.0, np.pi - 1e-6, np.pi - 1e-9]:
        for u in axes:
            v = th * u
            R = so3.exp_so3(v)
            back = so3.log_so3(R)
            # near pi the axis sign is ambiguous only at exactly pi
            assert np.allclose(so3.exp_so3(back), R, atol=1e-12)
            assert abs(np.linalg.norm(back) - th) < 1e-9


def test_quaternion_conventions_match_scipy():
    R = rand_rot(50)
    q = so3.quat_from_R(R)
    assert np.all(q[:, 0] >= 0)
    xyzw = sst.Rotation.from_matrix(R).as_quat()
    wxyz = np.concatenate([xyzw[:, 3:], xyzw[:, :3]], 1)
    wxyz *= np.sign(wxyz[:, :1])
    assert np.allclose(q, wxyz, atol=1e-12)
    assert np.allclose(so3.R_from_quat(q), R, atol=1e-12)
    # product of quaternions is composition of rotations
    p = so3.quat_from_R(R[::-1])
    assert np.allclose(so3.R_from_quat(so3.quat_mul(p, q)), R[::-1] @ R, atol=1e-12)


def test_two_distance_formulas_agree():
    A, B = rand_rot(100), rand_rot(100)[::-1]
    d1 = so3.dist_so3(A, B)
    d2 = so3.dist_quat(so3.quat_from_R(A), so3.quat_from_R(B))
    assert np.allclose(d1, d2, atol=1e-7)  # arccos form loses digits near 0 and pi
    # geodesic distance equals the angle of A^T B
    d3 = np.linalg.norm(so3.log_so3(np.swapaxes(A, 1, 2) @ B), axis=1)
    assert np.allclose(d2, d3, atol=1e-12)


def test_projection_onto_so3():
    R = rand_rot(10)
    assert np.allclose(so3.proj_so3(R), R, atol=1e-13)
    assert np.allclose(so3.proj_so3(3.7 * R), R, atol=1e-13)
    M = R[0] + 0.3 * rng.normal(size=(3, 3))
    P = so3.proj_so3(M)
    assert abs(np.linalg.det(P) - 1) < 1e-12
    assert np.allclose(P.T @ P, np.eye(3), atol=1e-12)
    # nearest rotation maximises tr(P^T M) over SO(3)
    best = np.trace(P.T @ M)
    for Q in rand_rot(2000):
        assert np.trace(Q.T @ M) <= best + 1e-12
    for v in rng.normal(size=(200, 3)) * 1e-3:
        assert np.trace((so3.exp_so3(v) @ P).T @ M) <= best + 1e-12


def test_slerp_is_geodesic_interpolation():
    qa = so3.quat_from_R(rand_rot(20))
    qb = so3.quat_from_R(rand_rot(20)[::-1])
    dab = so3.dist_quat(qa, qb)
    for tau in [0.0, 0.1, 0.5, 0.9, 1.0]:
        x = so3.slerp(qa, qb, tau)
        assert np.allclose(so3.dist_quat(qa, x), tau * dab, atol=1e-12)
        assert np.allclose(so3.dist_quat(x, qb), (1 - tau) * dab, atol=1e-12)
