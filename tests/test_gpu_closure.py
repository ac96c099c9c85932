"""End to end on the GPU (Alg. 1): Step I -> Step II -> Step III.

* 3D-3D in FP64 (N = 8, 2048 RANSAG seeds, 4096 samples, 200 GGD
  iterations): every stage against the oracle (seeds identical, walk trace
  replay, ball replay) and the invariants of Section II.
* The octahedral PURSE, whose balls have closed forms: the inner
  approximation of Prop. 1 from below, close to D* and d*.
"""
import numpy as np
import pytest
import torch

from oracle import closure, megb as om, ransag, so3
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn
from tests import parity
from tests.gpu_helpers import megb, sample
from tests.test_gpu_megb import check_rotation, check_translation

pytestmark = pytest.mark.gpu


def test_closure_3d3d_fp64_against_oracle():
    p = syn.purse_3d3d(8, 0)
    prm = closure.preset_3d3d()
    K = 200
    with P.Purse(p) as h:
        seeds = torch.empty((2048, 12), dtype=torch.float64, device="cuda")
        s0 = P.purse_ransag(h.h, 0, 1 << 20, 2048, seeds)
        seeds_np = seeds.cpu().numpy()[:s0]
        q, t, tr = sample(h.h, prm, 0, 1, 3, seeds_np, 4096)
        res, far = megb(h.h, 1, K, q, t)
    ref_seeds, _ = ransag.ransag_3d3d(p, 0, 1 << 20, 2048)
    assert s0 == len(ref_seeds) == 2048
    assert np.abs(seeds_np - ref_seeds).max() <= 1e-9
    R, tt, rep = parity.replay_walks(p, ref_seeds, prm, 3, np.arange(4096), tr, 1, 0)
    assert rep.ok() and not rep.robust_mismatch
    assert parity.rot_angle(q, so3.quat_from_R(R)).max() <= 1e-10
    assert np.abs(t - tt).max() <= 1e-10
    C, D = check_rotation(q, res, far[:K], 1)
    c, d = check_translation(t, res, far[K:], 1)
    # Section II invariants: every sample in S, inside its ball
    assert np.all(parity.classify(p, so3.R_from_quat(q), t, 1) >= 0)
    assert np.all(om.rotation_distances(C, om.canonical(q)) <= D + 1e-12)
    assert np.all(np.linalg.norm(t - c, axis=1) <= d + 1e-12)
    # the walks push the samples out: the ball of the boundary samples exceeds that of the seeds
    q0 = so3.quat_from_R(ref_seeds[:, :9].reshape(-1, 3, 3))
    assert D > om.megb_rotation(q0, K)[1]


def test_octahedral_closed_form_on_gpu():
    L, r = 0.1, 0.01
    p = syn.purse_octahedron(L, r, 0)
    Dstar, dstar = 2 * np.arcsin(r * np.sqrt(6) / (4 * L)), r
    K = 200
    with P.Purse(p) as h:
        q, t, _ = sample(h.h, closure.preset_3d3d(), 0, 0, 1, p.seed_pose()[None], 4096, trace=False)
        res, _ = megb(h.h, 0, K, q, None)
        qt, tt, _ = sample(h.h, closure.preset_3d3d(v0=0.02, rot_perturb=0.2), 1, 0, 1, p.seed_pose()[None], 4096,
                           trace=False)
        res_t, _ = megb(h.h, 0, K, None, tt)
    assert 0.9 * Dstar <= res[7] <= Dstar * (1 + 1 / np.sqrt(K))
    assert 0.9 * dstar <= res_t[8] <= dstar * (1 + 1 / np.sqrt(K))
    assert parity.rot_angle(res[:4], so3.quat_from_R(p.R_gt)) < 0.2 * Dstar
