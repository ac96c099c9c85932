"""Pins of the oracle's RANSAG for 3D-3D (CPU only)."""
import numpy as np

from oracle import purse as op
from oracle import ransag, so3
from paper_2403_09990_gb300 import synthetic as syn

rng = np.random.default_rng(21)


def test_arun_recovers_noise_free_pose():
    for _ in range(20):
        R = so3.exp_so3(rng.normal(size=3) * 2)
        t = rng.normal(size=3)
        A = rng.normal(size=(3, 3))
        B = A @ R.T + t
        Rh, th = ransag.arun(A, B)
        assert np.allclose(Rh, R, atol=1e-10) and np.allclose(th, t, atol=1e-10)
        assert abs(np.linalg.det(Rh) - 1) < 1e-12


def test_arun_is_least_squares_optimal():
    A = rng.normal(size=(3, 3)) * 0.1
    B = A @ so3.exp_so3(rng.normal(size=3)).T + rng.normal(size=3) + rng.normal(size=(3, 3)) * 0.01
    R, t = ransag.arun(A, B)

    def cost(Rx, tx):
        return ((B - A @ Rx.T - tx) ** 2).sum()

    c0 = cost(R, t)
    for v in rng.normal(size=(500, 6)) * 1e-3:
        Rx = so3.exp_so3(v[:3]) @ R
        # best translation for Rx is the centroid difference
        tx = B.mean(0) - Rx @ A.mean(0)
        assert cost(Rx, tx) >= c0 - 1e-15
        assert cost(R, t + v[3:]) >= c0 - 1e-15


def test_ransag_seeds_are_in_the_purse():
    p = syn.purse_3d3d(8, 0)
    seeds, acc = ransag.ransag_3d3d(p, 0, 20000, 256)
    assert len(seeds) > 0
    assert np.all(np.diff(acc) > 0)
    R = seeds[:, :9].reshape(-1, 3, 3)
    assert np.allclose(R @ np.swapaxes(R, 1, 2), np.eye(3), atol=1e-12)
    assert np.all(op.in_purse(p, R, seeds[:, 9:]))
    # trial acceptance is reproducible trial by trial
    Rt, tt, ok, idx = ransag.ransag_trials(p, 0, acc[:5])
    assert ok.all() and np.allclose(Rt.reshape(-1, 9), seeds[:5, :9])
