"""Autotuner on the GPU: every tuning call picks one of its candidates and times it beside the
default shape, and no shape changes a result (walks: one warp per walk; balls: the lowest-index
maximum whatever the grid; distances: one pose each), so forcing different cached shapes gives
bit-identical outputs."""
import numpy as np
import pytest
import torch

from oracle import closure
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn
from tests.gpu_helpers import params_from, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _clean_cache():
    P.purse_tune_cache_clear()
    yield
    P.purse_tune_cache_clear()


def _walk(h, prm, sampler, seeds, W):
    q = torch.empty((W, 4), dtype=torch.float32, device="cuda")
    t = torch.empty((W, 3), dtype=torch.float32, device="cuda")
    P.purse_sample(h.h, params_from(prm, sampler, 0), 9, seeds, 1, W, q, t, None)
    P.purse_sync(h.h)
    return q, t


@pytest.mark.parametrize("kind,sampler", [(1, 1), (0, 0)])
def test_walk_shapes_give_identical_samples_and_tuning_picks_one(kind, sampler):
    p = syn.purse_2d3d(16, 0) if kind == 1 else syn.purse_3d3d(8, 0)
    prm = closure.preset_2d3d(n_iter=4) if kind == 1 else closure.preset_3d3d(n_iter=4)
    W = 20000
    seeds = to_dev(p.seed_pose()[None])
    with P.Purse(p) as h:
        outs = []
        for warps in (8, 4, 2):
            P.purse_tune_cache_put(P.TUNE_WALK, kind, p.n, W, sampler, None, warps)
            outs.append(_walk(h, prm, sampler, seeds, W))
        for q, t in outs[1:]:
            assert torch.equal(q, outs[0][0]) and torch.equal(t, outs[0][1])
        P.purse_tune_cache_clear()
        q = torch.empty((W, 4), dtype=torch.float32, device="cuda")
        t = torch.empty((W, 3), dtype=torch.float32, device="cuda")
        r = P.purse_tune_walk(h.h, params_from(prm, sampler, 0), 9, seeds, 1, W, q, t)
        assert r["config"] in (8, 4, 2) and r["n_tried"] == 3 and r["default_config"] == 8
        assert 0 < r["ms"] <= r["default_ms"] * 1.0001
        assert P.purse_tune_cache_get(P.TUNE_WALK, kind, p.n, W, sampler)["config"] == r["config"]
        q2, t2 = _walk(h, prm, sampler, seeds, W)
        assert torch.equal(q2, outs[0][0]) and torch.equal(t2, outs[0][1])


@pytest.mark.parametrize("precision,n", [(0, 300000), (1, 40000)])
def test_ball_shapes_give_identical_balls(precision, n):
    rng = np.random.default_rng(3)
    dt = torch.float32 if precision == 0 else torch.float64
    q = rng.normal(size=(n, 4)) * np.array([1.0, 0.05, 0.05, 0.05]) + np.array([1.0, 0, 0, 0])
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    qd = torch.as_tensor(q, dtype=dt).cuda()
    td = torch.as_tensor(rng.normal(size=(n, 3)) * 0.01, dtype=dt).cuda()
    p = syn.purse_3d3d(8, 0)
    with P.Purse(p) as h:
        res = []
        cands = (1, 2, 4, 8, 16, 32, 64) if precision == 0 else (1, 2, 4, 8)
        for spt in cands:
            P.purse_tune_cache_put(P.TUNE_MEGB, 0, p.n, n, precision, None, spt)
            out = torch.empty(9, dtype=torch.float64, device="cuda")
            far = torch.empty(400, dtype=torch.int32, device="cuda")
            P.megb_solve(h.h, precision, 200, qd, n, td, n, out, far)
            P.purse_sync(h.h)
            res.append((out.cpu().numpy(), far.cpu().numpy()))
        for o, f in res[1:]:
            assert np.array_equal(o, res[0][0]) and np.array_equal(f, res[0][1])
        P.purse_tune_cache_clear()
        out = torch.empty(9, dtype=torch.float64, device="cuda")
        r = P.purse_tune_megb(h.h, precision, 200, qd, n, td, n, out)
        assert r["config"] in cands and r["n_tried"] == len(cands)
        assert np.array_equal(out.cpu().numpy(), res[0][0])


def test_tensor_core_shapes_give_identical_distances():
    p = syn.purse_2d3d(16, 0)
    rng = np.random.default_rng(5)
    n = 1 << 18
    R = np.broadcast_to(p.R_gt, (n, 3, 3)).reshape(n, 9)
    t = p.t_gt + rng.normal(size=(n, 3)) * np.array([0.004, 0.004, 0.03])
    poses = torch.as_tensor(np.concatenate([R, t], axis=1), dtype=torch.float32).cuda().contiguous()
    with P.Purse(p) as h:
        outs = []
        for cta in (2, 1):
            P.purse_tune_cache_put(P.TUNE_DIST, 1, p.n, n, 3, None, cta)
            d = torch.empty(n, dtype=torch.float32, device="cuda")
            P.purse_dist(h.h, 1, poses, n, d)
            P.purse_sync(h.h)
            outs.append(d)
        for d in outs[1:]:
            assert torch.equal(d, outs[0])
        P.purse_tune_cache_clear()
        d = torch.empty(n, dtype=torch.float32, device="cuda")
        r = P.purse_tune_dist(h.h, 1, poses, n, d)
        assert r["config"] in (2, 1) and torch.equal(d, outs[0])
