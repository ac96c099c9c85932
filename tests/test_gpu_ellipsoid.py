"""Noise bounded in the general norm of eq. 4 (purse_set_noise) on the GPU against the oracle:
RANSAG seeds (ellipsoid draws and acceptance in that norm), the fused and the plain samplers
replayed by the oracle, eq. 11 distances, and the closed-form translation ball of the octahedral
PURSE with one noise matrix."""
import numpy as np
import pytest
import torch

from oracle import closure, megb as om, p3p, purse as op, ransag, so3
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn
from tests import parity
from tests.gpu_helpers import params_from, sample, to_dev
from tests.test_gpu_plain import sample_plain

pytestmark = pytest.mark.gpu


def test_ransag_3d3d_ellipsoidal_matches_oracle():
    p = syn.purse_3d3d_ellipsoidal(8, 4)
    seeds = torch.full((128, 12), np.nan, dtype=torch.float64, device="cuda")
    with P.Purse(p) as h:
        got = P.purse_ransag(h.h, 11, 100000, 128, seeds)
    ref, _ = ransag.ransag_3d3d(p, 11, 100000, 128)
    assert got == len(ref) > 0
    assert np.abs(seeds.cpu().numpy()[:got] - ref).max() <= 1e-9


def test_ransag_2d3d_ellipsoidal_matches_oracle():
    p = syn.purse_2d3d_ellipsoidal(6, 4)
    seeds = torch.full((64, 12), np.nan, dtype=torch.float64, device="cuda")
    with P.Purse(p) as h:
        got = P.purse_ransag(h.h, 11, 4000, 64, seeds)
    ref, _ = p3p.ransag_2d3d(p, 11, 4000, 64)
    assert got == len(ref) > 0
    d = np.abs(seeds.cpu().numpy()[:got] - ref).max(axis=1)
    assert np.median(d) <= 1e-10 and d.max() <= 1e-6


@pytest.mark.parametrize("kind,precision,sampler", [(0, 1, 0), (0, 0, 0), (0, 0, 1), (1, 0, 0), (1, 1, 1)])
def test_ellipsoidal_walks_replay(kind, precision, sampler):
    if kind == 0:
        p = syn.purse_3d3d_ellipsoidal(8, 2)
        prm = closure.preset_3d3d(v0=0.02, rot_perturb=0.2) if sampler else closure.preset_3d3d()
    else:
        p = syn.purse_2d3d_ellipsoidal(16, 2)
        prm = closure.preset_2d3d()
    seeds = p.seed_pose()[None]
    n = 161
    with P.Purse(p) as h:
        q, t, tr = sample_plain(h.h, prm, sampler, precision, 55, seeds, n)
    R, tt, rep = parity.replay_walks(p, seeds, prm, 55, np.arange(n), tr, precision, sampler)
    assert rep.ok(), rep.inconsistent[:10]
    assert not rep.robust_mismatch, rep.robust_mismatch[:10]
    tol = 1e-10 if precision else 1e-5
    assert parity.rot_angle(q, so3.quat_from_R(R)).max() <= tol
    assert np.abs(t - tt).max() <= tol
    assert np.all(parity.classify(p, so3.R_from_quat(q), t, precision) >= 0)
    print(f"ellipsoidal kind {kind} sampler {sampler} precision {precision}: robust {rep.robust.mean():.3f}")


FUSED = {
    "3d3d-R-fp64": (0, 8, 1, 0), "3d3d-R-fp32": (0, 8, 0, 0), "3d3d-t-fp32": (0, 8, 0, 1),
    "3d3d-t-fp64-n7": (0, 7, 1, 1), "2d3d-R-fp32": (1, 16, 0, 0), "2d3d-t-fp32": (1, 16, 0, 1),
    "2d3d-R-fp64": (1, 16, 1, 0), "2d3d-t-fp64-n9": (1, 9, 1, 1), "2d3d-R-fp32-n128": (1, 128, 0, 0),
}


@pytest.mark.parametrize("name", list(FUSED))
def test_ellipsoidal_fused_walks_replay(name):
    """The fused walk kernels with noise matrices (odd N: the padded half of the last ladder pair;
    N = 128: fewer warps per block for the larger tables), replayed by the oracle."""
    kind, n_kp, precision, sampler = FUSED[name]
    if kind == 0:
        p = syn.purse_3d3d_ellipsoidal(n_kp, 2)
        prm = closure.preset_3d3d(v0=0.02, rot_perturb=0.2) if sampler else closure.preset_3d3d()
    else:
        p = syn.purse_2d3d_ellipsoidal(n_kp, 2)
        prm = closure.preset_2d3d(n_iter=3 if n_kp > 32 else 5)
    seeds = p.seed_pose()[None]
    n = 257
    with P.Purse(p) as h:
        q, t, tr = sample(h.h, prm, sampler, precision, 66, seeds, n)
        evals = P.purse_last_evals(h.h)
    assert evals > n * prm.n_iter * prm.n_perturb * p.n
    R, tt, rep = parity.replay_walks(p, seeds, prm, 66, np.arange(n), tr, precision, sampler)
    assert rep.ok(), rep.inconsistent[:10]
    assert not rep.robust_mismatch, rep.robust_mismatch[:10]
    tol = 1e-10 if precision else 1e-5
    assert parity.rot_angle(q, so3.quat_from_R(R)).max() <= tol
    assert np.abs(t - tt).max() <= tol
    assert np.all(parity.classify(p, so3.R_from_quat(q), t, precision) >= 0)
    moved = (tr[:, :, prm.n_keep] >= 0).any(axis=1).mean()
    assert moved > 0.5
    print(f"fused ellipsoidal {name}: robust {rep.robust.mean():.3f}, moved {moved:.3f}")


def test_ellipsoidal_distance_mode0():
    p = syn.purse_2d3d_ellipsoidal(16, 3)
    rng = np.random.default_rng(0)
    R = so3.exp_so3(rng.normal(size=(3000, 3)) * 0.02) @ p.R_gt
    t = p.t_gt + rng.normal(size=(3000, 3)) * 0.01
    poses = np.concatenate([R.reshape(-1, 9), t], axis=1).astype(np.float32)
    Rf, tf = poses[:, :9].astype(np.float64).reshape(-1, 3, 3), poses[:, 9:].astype(np.float64)
    ref = op.dist_to_boundary(p, Rf, tf)
    out = torch.empty(3000, dtype=torch.float32, device="cuda")
    with P.Purse(p) as h:
        P.purse_dist(h.h, 0, torch.as_tensor(poses).cuda(), 3000, out)
        with pytest.raises(P.PurseError):
            P.purse_dist(h.h, 1, torch.as_tensor(poses).cuda(), 3000, out)
        P.purse_sync(h.h)
    got = out.cpu().numpy().astype(np.float64)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    assert np.abs(got[fin] - ref[fin]).max() <= 2e-3   # pixels, FP32 projection of coordinates ~600 px


def test_ellipsoidal_octahedron_translation_ball_on_gpu():
    p = syn.purse_octahedron_ellipsoidal(seed=3)
    dstar = 0.01 / np.sqrt(np.linalg.eigvalsh(p.lam[0]).min())
    prm = closure.preset_3d3d(v0=0.02, rot_perturb=0.2, n_iter=8)
    S = 4096
    q = torch.empty((S, 4), dtype=torch.float64, device="cuda")
    t = torch.empty((S, 3), dtype=torch.float64, device="cuda")
    res = torch.empty(9, dtype=torch.float64, device="cuda")
    with P.Purse(p) as h:
        P.purse_sample_plain(h.h, params_from(prm, 1, 1), 5, to_dev(p.seed_pose()[None]), 1, S, q, t)
        P.megb_solve_exact(h.h, 1, q, S, t, S, res)
        P.purse_sync(h.h)
    d = float(res.cpu().numpy()[8])
    assert d <= dstar * (1 + 1e-9) and d >= 0.97 * dstar, (d, dstar)


def test_noise_matrix_rules_and_identity_matrices_reproduce_the_identity_norm():
    """Lambda_i = I through the noise-matrix kernels (walks and boundary snap) gives the samples and
    snap records of the identity norm: U = I multiplies by one and adds zero, exactly."""
    p = syn.purse_3d3d(8, 1)
    prm = closure.preset_3d3d(n_iter=4, v0=0.02, rot_perturb=0.002, trans_perturb=0.002, perturb_units=1)
    W = 512
    with P.Purse(p) as h:
        bad = np.repeat(np.diag([1.0, -1.0, 1.0])[None], 8, axis=0)
        with pytest.raises(P.PurseError):
            P.purse_set_noise(h.h, bad)
        sd = to_dev(p.seed_pose()[None])
        outs = {}
        for lam in (None, np.repeat(np.eye(3)[None], 8, axis=0)):
            P.purse_set_noise(h.h, lam)
            for sampler in (0, 1):
                q = torch.empty((W, 4), dtype=torch.float32, device="cuda")
                t = torch.empty((W, 3), dtype=torch.float32, device="cuda")
                snap = torch.full((W, 12), np.nan, dtype=torch.float32, device="cuda")
                P.purse_sample(h.h, params_from(prm, sampler, 0), 3, sd, 1, W, q, t, snap=snap)
                P.purse_sync(h.h)
                outs[(lam is None, sampler)] = (q.cpu().numpy(), t.cpu().numpy(), snap.cpu().numpy())
        for sampler in (0, 1):
            a, b = outs[(True, sampler)], outs[(False, sampler)]
            assert (a[2][:, 0] >= 0).mean() > 0.5
            for x, y in zip(a, b):
                assert np.array_equal(x, y), (sampler, np.abs(x - y).max())
