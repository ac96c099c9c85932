"""Exact Step III balls on the GPU (megb_solve_exact) against the oracle's exact balls.

The minimum enclosing ball is unique, so the GPU's centre and radius must equal the
oracle's (Welzl in FP64 on the same values) up to rounding.  At full size the oracle
cannot run Welzl on millions of points; there the ball is checked through what fixes it:
every sample inside, and the exact ball of the samples near the boundary (the only ones
that can support it) equal to the GPU's."""
import numpy as np
import pytest
import torch

from oracle import megb as om, so3
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn
from tests.gpu_helpers import DT, to_dev

pytestmark = pytest.mark.gpu


def clouds(n, seed, rot_scale=(0.03, 0.08, 0.15), t_scale=(0.004, 0.01, 0.02)):
    rng = np.random.default_rng(seed)
    C0 = so3.quat_from_R(so3.exp_so3(rng.normal(size=3)))
    q = so3.quat_mul(so3.quat_exp(rng.normal(size=(n, 3)) * np.array(rot_scale)), C0[None])
    q = q * np.where(q[:, :1] < 0, -1.0, 1.0)          # stored with w >= 0, as the samplers do
    t = rng.normal(size=(n, 3)) * np.array(t_scale) + rng.normal(size=3)
    return q, t


def solve_exact(h, precision, q, t, ref=None):
    dq = to_dev(q, DT[precision]) if q is not None else None
    dt = to_dev(t, DT[precision]) if t is not None else None
    res = torch.full((9,), np.nan, dtype=torch.float64, device="cuda")
    P.megb_solve_exact(h, precision, dq, 0 if q is None else len(q), dt, 0 if t is None else len(t), res,
                       None if ref is None else to_dev(ref))
    P.purse_sync(h)
    return res.cpu().numpy()


@pytest.mark.parametrize("n,precision", [(1, 1), (2, 1), (5, 1), (300, 1), (5000, 1), (5000, 0), (20011, 0)])
def test_exact_balls_match_the_oracle(n, precision):
    q, t = clouds(n, n)
    if precision == 0:
        q, t = q.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64)
    p = syn.purse_3d3d(8, 0)
    with P.Purse(p) as h:
        res = solve_exact(h.h, precision, q, t)
    C, D = om.meb_exact_rotation(q, q[0])
    c, d = om.meb_exact_translation(t)
    assert abs(res[8] - d) <= 1e-9 * max(d, 1e-300) + 1e-15, (res[8], d)
    assert abs(res[7] - D) <= 1e-9 * max(D, 1e-300) + 1e-12, (res[7], D)
    if n > 1:
        assert np.abs(res[4:7] - c).max() <= 1e-6 * d + 1e-12
        assert so3.dist_quat(res[:4], C) <= 1e-6 * D + 1e-12
    # every sample inside; the translation ball is never larger than the descent ball
    assert np.linalg.norm(t - res[4:7], axis=1).max() <= res[8] * (1 + 1e-12) + 1e-15
    assert so3.dist_quat(res[None, :4], q).max() <= res[7] + 1e-12
    cg, dg, _ = om.megb_translation(t, 200)
    assert res[8] <= dg * (1 + 1e-12)


def test_exact_balls_of_boundary_samples_at_full_size():
    """2^20 samples of each sampler from the fused walks (2D-3D, N = 16, 5 iterations), FP32."""
    from oracle import closure
    from tests.gpu_helpers import params_from
    p = syn.purse_2d3d(16, 0)
    prm = closure.preset_2d3d(n_iter=5)
    n = 1 << 20
    seeds = to_dev(p.seed_pose()[None])
    q = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    t = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    q2 = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    t2 = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    res = torch.full((9,), np.nan, dtype=torch.float64, device="cuda")
    ggd = torch.full((9,), np.nan, dtype=torch.float64, device="cuda")
    with P.Purse(p) as h:
        P.purse_sample(h.h, params_from(prm, 0, 0), 3, seeds, 1, n, q, t)
        P.purse_sample(h.h, params_from(prm, 1, 0), 3, seeds, 1, n, q2, t2)
        P.megb_solve(h.h, 0, 200, q, n, t2, n, ggd)
        P.megb_solve_exact(h.h, 0, q, n, t2, n, res, ggd[:4].contiguous())
        P.purse_sync(h.h)
    r, g = res.cpu().numpy(), ggd.cpu().numpy()
    qn = q.cpu().numpy().astype(np.float64)
    tn = t2.cpu().numpy().astype(np.float64)
    # translations: all inside; the exact ball of the samples within 1e-3 of the boundary is the same ball
    dist = np.linalg.norm(tn - r[4:7], axis=1)
    assert dist.max() <= r[8] * (1 + 1e-12)
    near = tn[dist >= r[8] * (1 - 1e-3)]
    c, d = om.meb_exact_translation(near)
    assert abs(d - r[8]) <= 1e-9 * r[8] and np.abs(c - r[4:7]).max() <= 1e-6 * r[8]
    assert r[8] <= g[8] * (1 + 1e-12)
    # rotations: the same through the quaternion embedding, signs on the side of the descent centre
    s = np.where(qn @ g[:4] < 0, -1.0, 1.0)[:, None]
    c4 = r[:4] / np.linalg.norm(r[:4])
    chord = np.linalg.norm(qn * s - c4, axis=1)
    near_q = qn[chord >= chord.max() * (1 - 1e-3)]
    C, D = om.meb_exact_rotation(near_q, g[:4])
    assert so3.dist_quat(C, r[:4]) <= 1e-6 * r[7]
    assert so3.dist_quat(r[None, :4], qn).max() <= r[7] * (1 + 1e-12)
    print(f"exact D {r[7]:.6f} (descent {g[7]:.6f}), exact d {r[8]:.6f} (descent {g[8]:.6f}), "
          f"{len(near)} / {len(near_q)} samples near the boundaries")


def test_exact_empty_sets():
    q, t = clouds(50, 1)
    p = syn.purse_3d3d(8, 0)
    with P.Purse(p) as h:
        r1 = solve_exact(h.h, 1, None, t)
        r2 = solve_exact(h.h, 1, q, None)
    assert np.all(r1[[0, 1, 2, 3, 7]] == 0) and r1[8] > 0
    assert np.all(r2[[4, 5, 6, 8]] == 0) and r2[7] > 0
