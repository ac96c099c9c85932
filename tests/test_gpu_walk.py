"""Fused walk kernel (Alg. 2-5) against the oracle: decision-trace replay.

For every walk the oracle recomputes each iteration in FP64 from the same
Philox draws, checks that the GPU's ranked perturbation list and its (m0, k0)
choice are consistent with the FP64 values outside the rounding band, then
follows the GPU's decisions; final poses must agree within 1e-5 rad and
1e-5 m (FP32) or 1e-10 (FP64).  Walks whose oracle decisions are all outside
the band must have exactly the GPU's trace.
"""
import numpy as np
import pytest

from oracle import closure, purse as op, ransag, so3
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn
from tests import parity
from tests.gpu_helpers import sample

pytestmark = pytest.mark.gpu

TOL = {0: (1e-5, 1e-5), 1: (1e-10, 1e-10)}


def seeds_3d3d(p, n):
    s, _ = ransag.ransag_3d3d(p, 0, 200000, n)
    return s


def seeds_2d3d_multi(p, n):
    # interior poses from a short oracle walk (all inside the PURSE) as a multi-seed S0
    prm = closure.preset_2d3d(n_iter=2)
    R, t = closure.sample_rotation_boundary(p, p.seed_pose()[None], prm, 99, np.arange(n))
    return np.concatenate([R.reshape(-1, 9), t], axis=1)


CASES = {
    "3d3d-R-fp64": dict(kind=0, sampler=0, precision=1, prm=dict(), seeds="ransag"),
    "3d3d-R-fp32": dict(kind=0, sampler=0, precision=0, prm=dict(), seeds="ransag"),
    "2d3d-R-fp32": dict(kind=1, sampler=0, precision=0, prm=dict(), seeds="gt"),
    "2d3d-t-fp32": dict(kind=1, sampler=1, precision=0, prm=dict(), seeds="gt"),
    "2d3d-t-fp32-pca": dict(kind=1, sampler=1, precision=0, prm=dict(), seeds="multi"),
    "2d3d-R-fp64": dict(kind=1, sampler=0, precision=1, prm=dict(), seeds="multi"),
    "3d3d-t-fp32": dict(kind=0, sampler=1, precision=0, prm=dict(v0=0.02, rot_perturb=0.2), seeds="ransag"),
    "2d3d-R-fp32-keep7-np100-nt9": dict(kind=1, sampler=0, precision=0,
                                        prm=dict(n_keep=7, n_perturb=100, n_steps=9), seeds="gt"),
    "3d3d-R-fp32-keep32-np256-nt32-raw": dict(kind=0, sampler=0, precision=0,
                                              prm=dict(n_keep=32, n_perturb=256, n_steps=32, perturb_units=1,
                                                       trans_perturb=0.002), seeds="ransag"),
    # large constraint tables: fewer warps per block fit the shared memory (N > 32 keeps table order)
    "2d3d-R-fp64-n256": dict(kind=1, sampler=0, precision=1, prm=dict(n_iter=3), seeds="gt", n=256),
    "2d3d-t-fp32-n128": dict(kind=1, sampler=1, precision=0, prm=dict(n_iter=3), seeds="gt", n=128),
    "3d3d-R-fp32-n64": dict(kind=0, sampler=0, precision=0, prm=dict(n_iter=3), seeds="gt", n=64),
    # degenerate settings: the fewest constraints, one perturbation kept of one, a single rung, gamma = 1
    "3d3d-R-fp64-n3-np1-keep1-nt1": dict(kind=0, sampler=0, precision=1, seeds="gt", n=3,
                                         prm=dict(n_perturb=1, n_keep=1, n_steps=1)),
    "2d3d-t-fp32-n3-np2-keep2-nt2-gamma1": dict(kind=1, sampler=1, precision=0, seeds="gt", n=3,
                                                prm=dict(n_perturb=2, n_keep=2, n_steps=2, gamma=1.0)),
    "2d3d-R-fp32-np33-keep1": dict(kind=1, sampler=0, precision=0, seeds="gt", prm=dict(n_perturb=33, n_keep=1)),
}


def make_case(c):
    if c["kind"] == 0:
        p = syn.purse_3d3d(c.get("n", 8), 0)
        prm = closure.preset_3d3d(**c["prm"])
        seeds = p.seed_pose()[None] if c["seeds"] == "gt" else seeds_3d3d(p, 32)
    else:
        p = syn.purse_2d3d(c.get("n", 16), 0)
        prm = closure.preset_2d3d(**c["prm"])
        seeds = p.seed_pose()[None] if c["seeds"] == "gt" else seeds_2d3d_multi(p, 8)
    return p, prm, seeds


@pytest.mark.parametrize("name", list(CASES))
def test_walk_replay(name):
    c = CASES[name]
    p, prm, seeds = make_case(c)
    n = 257  # several warps and blocks plus a ragged tail
    seed = 1234
    with P.Purse(p) as h:
        q, t, tr = sample(h.h, prm, c["sampler"], c["precision"], seed, seeds, n)
    assert tr.min() >= -1
    R, tt, rep = parity.replay_walks(p, seeds, prm, seed, np.arange(n), tr, c["precision"], c["sampler"])
    assert rep.ok(), f"inconsistent decisions: {rep.inconsistent[:10]}"
    assert not rep.robust_mismatch, rep.robust_mismatch[:10]
    atol_r, atol_t = TOL[c["precision"]]
    ang = parity.rot_angle(q, so3.quat_from_R(R))
    assert ang.max() <= atol_r, ang.max()
    assert np.abs(t - tt).max() <= atol_t, np.abs(t - tt).max()
    # every sample is a pose of the PURSE (up to the rounding band)
    cls = parity.classify(p, so3.R_from_quat(q), t, c["precision"])
    assert np.all(cls >= 0)
    # the walks move: most end away from their seed
    moved = (tr[:, :, prm.n_keep] >= 0).any(axis=1).mean()
    if prm.n_steps >= 3:  # with one or two rungs the full step may never fit
        assert moved > 0.5
    print(f"{name}: robust fraction {rep.robust.mean():.3f}, moved {moved:.3f}")


def test_walk_zero_iterations_returns_seeds():
    p = syn.purse_2d3d(16, 1)
    prm = closure.preset_2d3d(n_iter=0)
    with P.Purse(p) as h:
        q, t, _ = sample(h.h, prm, 0, 0, 5, p.seed_pose()[None], 33, trace=False)
    assert parity.rot_angle(q, so3.quat_from_R(p.R_gt)[None]).max() < 1e-6
    assert np.abs(t - p.t_gt).max() < 1e-6


def test_empty_sample_count_is_a_no_op():
    p = syn.purse_3d3d(8, 1)
    with P.Purse(p) as h:
        q, t, _ = sample(h.h, closure.preset_3d3d(), 0, 0, 5, p.seed_pose()[None], 0, trace=False)
    assert q.shape == (0, 4)


def test_full_size_launch_sampled_parity():
    """The 2D-3D workload at full size (2^20 walks, 100 iterations, both samplers):
    64 sampled walks replayed by the oracle, membership on 4096 sampled outputs."""
    p = syn.purse_2d3d(16, 0)
    prm = closure.preset_2d3d(n_iter=100)
    n = 1 << 20
    rng = np.random.default_rng(0)
    ids = np.sort(rng.choice(n, 64, replace=False))
    ids[-1] = n - 1
    with P.Purse(p) as h:
        for sampler in (0, 1):
            q, t, tr = sample(h.h, prm, sampler, 0, 77, p.seed_pose()[None], n, trace_rows=ids)
            R, tt, rep = parity.replay_walks(p, p.seed_pose()[None], prm, 77, ids, tr, 0, sampler)
            assert rep.ok(), rep.inconsistent[:10]
            ang = parity.rot_angle(q[ids], so3.quat_from_R(R))
            assert ang.max() <= 1e-5 and np.abs(t[ids] - tt).max() <= 1e-5
            pick = rng.choice(n, 4096, replace=False)
            assert np.all(parity.classify(p, so3.R_from_quat(q[pick]), t[pick], 0) >= 0)
            evals = P.purse_last_evals(h.h)
            assert evals >= n * prm.n_iter * prm.n_perturb * p.n
