"""Pose-regression PURSE (Example 3) on the GPU against the oracle: convex-combination seeds,
the fused and the plain per-operation samplers replayed by the oracle, and the closed-form
balls of a nested PURSE through the GPU's own seeds, walks and exact balls."""
import numpy as np
import pytest
import torch

from oracle import closure, purse as op, ransag, so3
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn
from tests import parity
from tests.gpu_helpers import params_from, sample, to_dev
from tests.test_gpu_plain import sample_plain

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,trials,max_seeds", [(10, 3000, 200), (3, 500, 500), (40, 70000, 100000)])
def test_convex_seeds_match_oracle(n, trials, max_seeds):
    p = syn.purse_reg(n, 4)
    seeds = torch.full((max_seeds, 12), np.nan, dtype=torch.float64, device="cuda")
    with P.Purse(p) as h:
        try:
            got = P.purse_ransag(h.h, 21, trials, max_seeds, seeds)
        except P.PurseError as e:
            assert e.status == 3
            got = 0
    ref, acc = ransag.convex_seeds(p, 21, trials, max_seeds)
    assert got == len(ref)
    if got:
        assert np.abs(seeds.cpu().numpy()[:got] - ref).max() <= 1e-12


@pytest.mark.parametrize("precision", [1, 0])
def test_regression_walks_replay(precision):
    p = syn.purse_reg(10, 4)
    prm = closure.preset_reg()
    seeds, _ = ransag.convex_seeds(p, 21, 3000, 40)
    n = 161
    with P.Purse(p) as h:
        q, t, tr = sample_plain(h.h, prm, 0, precision, 77, seeds, n)
        evals = P.purse_last_evals(h.h)
    assert evals == n * prm.n_iter * (prm.n_perturb + prm.n_steps * prm.n_keep) * 2 * p.n
    R, tt, rep = parity.replay_walks(p, seeds, prm, 77, np.arange(n), tr, precision, 0)
    assert rep.ok(), rep.inconsistent[:10]
    assert not rep.robust_mismatch, rep.robust_mismatch[:10]
    tol = 1e-10 if precision else 1e-5
    assert parity.rot_angle(q, so3.quat_from_R(R)).max() <= tol
    assert np.abs(t - tt).max() <= tol
    assert np.all(parity.classify(p, so3.R_from_quat(q), t, precision) >= 0)
    assert (tr[:, :, prm.n_keep] >= 0).any(axis=1).mean() > 0.5
    print(f"regression precision {precision}: robust fraction {rep.robust.mean():.3f}")


FUSED = {
    "R-fp32": (10, 0, 0, {}), "R-fp64": (10, 1, 0, {}), "R-fp32-n3": (3, 0, 0, {}),
    "R-fp64-n40-keep7-np100-nt9": (40, 1, 0, dict(n_keep=7, n_perturb=100, n_steps=9)),
    "t-fp32": (10, 0, 1, dict(rot_perturb=0.2, v0=0.02)), "t-fp64": (10, 1, 1, dict(rot_perturb=0.2, v0=0.02)),
    "R-fp32-np256-keep32-nt32": (10, 0, 0, dict(n_perturb=256, n_keep=32, n_steps=32)),
}


@pytest.mark.parametrize("name", list(FUSED))
def test_regression_fused_walks_replay(name):
    """The fused pose-regression walks (one part of each hypothesis per perturbation, separable
    ladder) replayed by the oracle, and their evaluation count."""
    n_hyp, precision, sampler, kw = FUSED[name]
    p = syn.purse_reg(n_hyp, 4)
    prm = closure.preset_reg(**kw)
    seeds, _ = ransag.convex_seeds(p, 21, 20000, 40)
    n = 257
    with P.Purse(p) as h:
        q, t, tr = sample(h.h, prm, sampler, precision, 78, seeds, n)
        evals = P.purse_last_evals(h.h)
    # per iteration N_P moving parts and N_T + N_P* ladder factors of N hypotheses; the part the
    # perturbations do not move once in the first iteration and after every move
    assert evals == (n * prm.n_iter * (prm.n_perturb + prm.n_steps + prm.n_keep) + fixed_count(tr, prm)) * p.n
    R, tt, rep = parity.replay_walks(p, seeds, prm, 78, np.arange(n), tr, precision, sampler)
    assert rep.ok(), rep.inconsistent[:10]
    assert not rep.robust_mismatch, rep.robust_mismatch[:10]
    tol = 1e-10 if precision else 1e-5
    assert parity.rot_angle(q, so3.quat_from_R(R)).max() <= tol
    assert np.abs(t - tt).max() <= tol
    assert np.all(parity.classify(p, so3.R_from_quat(q), t, precision) >= 0)
    moved = (tr[:, :, prm.n_keep] >= 0).any(axis=1).mean()
    assert moved > 0.5
    print(f"fused regression {name}: robust {rep.robust.mean():.3f}, moved {moved:.3f}")


def fixed_count(tr, prm):
    """Iterations that evaluate the unmoved part: the first and every one after a move."""
    mv = tr[:, :, prm.n_keep] >= 0
    return int(tr.shape[0] + mv[:, :-1].sum())


def test_nested_regression_closed_form_on_gpu():
    """Seeds, walks and the exact balls all on the GPU: the rotation ball approaches the known
    angle 2 asin(beta / (2 sqrt 2)) from below, the translation ball stays within its radius."""
    p = syn.purse_reg_nested(10, 0, beta_rot=0.04, beta_t=0.006)
    Dstar = 2 * np.arcsin(0.04 / (2 * np.sqrt(2)))
    prm = closure.preset_reg()
    S = 200 * prm.n_walk
    seeds = torch.empty((200, 12), dtype=torch.float64, device="cuda")
    q = torch.empty((S, 4), dtype=torch.float32, device="cuda")
    t = torch.empty((S, 3), dtype=torch.float32, device="cuda")
    res = torch.empty(9, dtype=torch.float64, device="cuda")
    with P.Purse(p) as h:
        s0 = P.purse_ransag(h.h, 3, 20000, 200, seeds)
        P.purse_sample_plain(h.h, params_from(prm, 0, 0), 5, seeds, s0, S, q, t)
        P.megb_solve_exact(h.h, 0, q, S, t, S, res)
        P.purse_sync(h.h)
    r = res.cpu().numpy()
    qn, tn = q.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64)
    assert np.all(parity.classify(p, so3.R_from_quat(qn), tn, 0) >= 0)
    assert r[7] <= Dstar * (1 + 1e-5) and r[7] >= 0.97 * Dstar, (r[7], Dstar)
    assert r[8] <= 0.006 * (1 + 1e-5)
    print(f"nested regression: D {r[7]:.6f} / D* {Dstar:.6f}, d {r[8]:.6f} / d* 0.006")


def test_regression_rejections():
    p = syn.purse_reg(10, 0)
    with P.Purse(p) as h:
        sd = to_dev(p.seed_pose()[None])
        q = torch.empty((8, 4), dtype=torch.float32, device="cuda")
        t = torch.empty((8, 3), dtype=torch.float32, device="cuda")
        snap = torch.empty((8, 12), dtype=torch.float32, device="cuda")
        with pytest.raises(P.PurseError) as e:   # no boundary snap for regression PURSEs
            P.purse_sample(h.h, params_from(closure.preset_reg(), 0, 0), 1, sd, 1, 8, q, t, snap=snap)
        assert e.value.status == 1
        P.purse_sample(h.h, params_from(closure.preset_reg(), 0, 0), 1, sd, 1, 8, q, t)
        poses = torch.zeros((4, 12), dtype=torch.float32, device="cuda")
        d = torch.empty(4, dtype=torch.float32, device="cuda")
        with pytest.raises(P.PurseError):
            P.purse_dist(h.h, 1, poses, 4, d)
        P.purse_dist(h.h, 0, poses, 4, d)   # mode 0 serves regression PURSEs
        P.purse_sync(h.h)
