"""dist(R, t, dS) of eq. 11 for materialised FP32 poses (purse_dist) against the FP64 oracle:
FP32 on the CUDA cores (mode 0), the tcgen05 split-TF32 contraction (mode 1) and one TF32
pass (mode 2).

Error bound of a contraction output o_c = sum_k p_k B_kc, with mag_c = sum_k |p_k B_kc|
(the absolute sum of its terms, computed here from the PURSE definitions):
* split TF32: hi = rna(x) leaves |lo| <= 2^-11 |x|, rna(lo) errs by <= 2^-22 |x|, and the
  dropped lo.lo term is <= 2^-22 |a b|: <= 3 2^-22 per product, plus FP32 accumulation of
  at most 48 terms (<= 48 2^-24): below 2^-17 mag_c with room to spare;
* one TF32 pass: <= 2 2^-11 per product, below 2^-9 mag_c;
* FP32 per-pose formula: the same 2^-17 bound.
The margin error follows: 3D-3D |d| <= |de|; 2D-3D (|de| + |e| |dP_z| / P_z) / P_z.
"""
import numpy as np
import pytest
import torch

from oracle import purse as op, so3
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

REL = {0: 2.0 ** -17, 1: 2.0 ** -17, 2: 2.0 ** -9}


def make_poses(p, n_poses, seed, behind=0):
    """FP32 poses around the ground truth (rotations up to 0.05 rad, translations of a few
    noise radii), plus `behind` poses of a 2D-3D PURSE moved behind the camera."""
    rng = np.random.default_rng(seed)
    phi = rng.normal(size=(n_poses, 3)) * 0.02
    R = so3.exp_so3(phi) @ p.R_gt
    scale = 3 * p.radii.mean() if p.kind == 0 else 0.01
    t = p.t_gt + rng.normal(size=(n_poses, 3)) * scale
    if behind:
        t[:behind, 2] = -2.0
    poses = np.concatenate([R.reshape(-1, 9), t], axis=1).astype(np.float32)
    return poses


def term_magnitudes(p, R, t):
    """mag of the three contraction outputs of every (pose, constraint): (..., N, 3)."""
    A = np.abs(np.einsum('...cj,nj->...ncj', R, p.model)).sum(axis=-1)  # sum_j |R_cj a_j|
    X = A + np.abs(t)[..., None, :]
    if p.kind == 0:
        return X + np.abs(p.obs)
    fx, fy, cx, cy = p.K
    u, v = p.obs[:, 0], p.obs[:, 1]
    mx = fx * X[..., 0] + np.abs(cx - u) * X[..., 2]
    my = fy * X[..., 1] + np.abs(cy - v) * X[..., 2]
    return np.stack([mx, my, X[..., 2]], axis=-1)


def bound(p, R, t, mode):
    mag = term_magnitudes(p, R, t)
    de = REL[mode] * mag
    if p.kind == 0:
        b = np.sqrt((de ** 2).sum(axis=-1))
    else:
        X = op.transform(p.model, R, t)
        fx, fy, cx, cy = p.K
        Pz = X[..., 2]
        ex = fx * X[..., 0] + (cx - p.obs[:, 0]) * Pz
        ey = fy * X[..., 1] + (cy - p.obs[:, 1]) * Pz
        e = np.hypot(ex, ey)
        Pzs = np.where(Pz > 0, Pz, 1.0)
        b = (np.hypot(de[..., 0], de[..., 1]) + e * de[..., 2] / Pzs) / Pzs
    return b.max(axis=-1)   # the minimum over constraints moves by at most the largest error


def run_dist(h, mode, poses):
    dp = torch.as_tensor(poses).cuda()
    out = torch.full((poses.shape[0],), np.nan, dtype=torch.float32, device="cuda")
    P.purse_dist(h, mode, dp, poses.shape[0], out)
    P.purse_sync(h)
    return out.cpu().numpy().astype(np.float64)


CASES = [(0, 8, 1000), (0, 3, 129), (0, 17, 4097), (0, 100, 3000), (0, 256, 1500),
         (1, 16, 1000), (1, 5, 200), (1, 33, 5000), (1, 80, 2000), (1, 96, 1000), (1, 256, 1300)]


@pytest.mark.parametrize("kind,n,n_poses", CASES)
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_dist_modes_against_oracle(kind, n, n_poses, mode):
    p = syn.purse_3d3d(n, 4) if kind == 0 else syn.purse_2d3d(n, 4)
    poses = make_poses(p, n_poses, 11, behind=7 if kind == 1 else 0)
    R = poses[:, :9].astype(np.float64).reshape(-1, 3, 3)
    t = poses[:, 9:].astype(np.float64)
    ref = op.dist_to_boundary(p, R, t)
    with P.Purse(p) as h:
        got = run_dist(h.h, mode, poses)
    inf = np.isinf(ref)
    assert np.array_equal(np.isinf(got), inf) and np.all(got[inf] == ref[inf])
    err = np.abs(got[~inf] - ref[~inf])
    b = bound(p, R, t, mode)[~inf]
    assert np.all(err <= b), (err.max(), b[np.argmax(err - b)])
    print(f"kind {kind} n {n} mode {mode}: max err {err.max():.3e}, median bound use {np.median(err / b):.3f}")


def test_split_tf32_is_near_fp32_and_single_pass_is_not():
    """The three-pass split recovers about FP32 accuracy; one TF32 pass is far coarser."""
    p = syn.purse_2d3d(16, 0)
    poses = make_poses(p, 1 << 16, 3)
    R = poses[:, :9].astype(np.float64).reshape(-1, 3, 3)
    t = poses[:, 9:].astype(np.float64)
    ref = op.dist_to_boundary(p, R, t)
    with P.Purse(p) as h:
        e = [np.abs(run_dist(h.h, m, poses) - ref).max() for m in (0, 1, 2)]
    assert e[1] < 20 * e[0] and e[2] > 20 * e[1], e


def test_dist_large_launch_sampled():
    """4 M poses (many tiles per CTA of the persistent grid): sampled rows against the oracle."""
    p = syn.purse_2d3d(16, 0)
    n_poses = (1 << 22) + 77
    poses = make_poses(p, n_poses, 5)
    rng = np.random.default_rng(0)
    ids = np.concatenate([rng.choice(n_poses, 4000, replace=False), [0, n_poses - 1]])
    R = poses[ids, :9].astype(np.float64).reshape(-1, 3, 3)
    t = poses[ids, 9:].astype(np.float64)
    ref = op.dist_to_boundary(p, R, t)
    with P.Purse(p) as h:
        for mode in (0, 1):
            got = run_dist(h.h, mode, poses)[ids]
            assert np.all(np.abs(got - ref) <= bound(p, R, t, mode))


def test_dist_empty_and_bad_arguments():
    p = syn.purse_3d3d(8, 0)
    with P.Purse(p) as h:
        e = torch.empty((0, 12), dtype=torch.float32, device="cuda")
        d = torch.empty((0,), dtype=torch.float32, device="cuda")
        P.purse_dist(h.h, 1, e, 0, d)
        with pytest.raises(P.PurseError):
            P.purse_dist(h.h, 3, e, 0, d)
