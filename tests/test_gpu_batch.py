"""Batched solves (one graph: statistics, one persistent walk launch, one block per ball)
against the single-PURSE path: PURSE p of a batch solved with key seed + p must give exactly the
samples, farthest-sample sequences and balls of purse_sample / megb_solve with that key."""
import numpy as np
import pytest
import torch

from oracle import closure, so3
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn
from tests import parity
from tests.gpu_helpers import params_from

pytestmark = pytest.mark.gpu


def presets(n_iter=5):
    p3 = closure.preset_3d3d(n_iter=n_iter)
    p2 = closure.preset_2d3d(n_iter=n_iter)
    return p3, p2


def single(purse, prm, sampler, seed, S):
    with P.Purse(purse) as h:
        seeds = torch.as_tensor(purse.seed_pose()[None], dtype=torch.float64, device="cuda")
        q = torch.empty((S, 4), device="cuda")
        t = torch.empty((S, 3), device="cuda")
        P.purse_sample(h.h, params_from(prm, sampler, 0), seed, seeds, 1, S, q, t)
        P.purse_sync(h.h)
        return q, t


@pytest.mark.parametrize("n_purses,S,K,tune", [(24, 256, 50, False), (7, 333, 20, True)])
def test_batch_equals_single_path(n_purses, S, K, tune):
    purses = syn.purse_batch(n_purses, seed=3, n_lo=4, n_hi=64)
    p3, p2 = presets()
    seed = 1000
    seeds = torch.as_tensor(syn.seed_array(purses), dtype=torch.float64, device="cuda")
    res = torch.full((n_purses, 9), np.nan, dtype=torch.float64, device="cuda")
    b = P.purse_batch_create(purses)
    try:
        pp3, pp2 = params_from(p3, 0, 0), params_from(p2, 0, 0)
        if tune:
            chunk, warps, ms = P.purse_batch_tune(b, pp3, pp2, seed, seeds, S)
            assert chunk in (1, 4, 16, 64) and warps in (4, 8) and ms > 0
        P.purse_batch_solve(b, pp3, pp2, seed, seeds, S, K, res)
        P.purse_batch_solve(b, pp3, pp2, seed, seeds, S, K, res)  # graph replay
        evals = P.purse_batch_sync(b)
        assert evals > 0
        far = torch.empty((n_purses, 2 * K), dtype=torch.int32, device="cuda")
        P.purse_batch_copy_farthest(b, far)
        for p, pu in enumerate(purses):
            bq, bt = torch.empty((S, 4), device="cuda"), torch.empty((S, 3), device="cuda")
            bq2, bt2 = torch.empty((S, 4), device="cuda"), torch.empty((S, 3), device="cuda")
            P.purse_batch_copy_samples(b, p, bq, bt, bq2, bt2)
            torch.cuda.synchronize()
            prm = p3 if pu.kind == 0 else p2
            q, t = single(pu, prm, 0, seed + p, S)
            assert torch.equal(q, bq) and torch.equal(t, bt), p
            if pu.kind == 1:
                q2, t2 = single(pu, prm, 1, seed + p, S)
                assert torch.equal(t2, bt2), p
                tball = t2
            else:
                tball = t
            r1 = torch.empty(9, dtype=torch.float64, device="cuda")
            f1 = torch.empty(2 * K, dtype=torch.int32, device="cuda")
            with P.Purse(pu) as h:
                P.megb_solve(h.h, 0, K, q, S, tball, S, r1, f1)
                P.purse_sync(h.h)
            assert torch.equal(f1, far[p]), p
            assert torch.allclose(r1, res[p], rtol=1e-12, atol=1e-15), (p, r1, res[p])
            # samples inside their PURSE (FP32 rounding band)
            qn, tn = q.cpu().numpy().astype(np.float64), tball.cpu().numpy().astype(np.float64)
            if pu.kind == 0:
                assert np.all(parity.classify(pu, so3.R_from_quat(qn), tn, 0) >= 0)
    finally:
        P.purse_batch_destroy(b)


def test_batch_argument_errors():
    purses = syn.purse_batch(3, seed=1)
    b = P.purse_batch_create(purses)
    try:
        p3, p2 = presets()
        seeds = torch.as_tensor(syn.seed_array(purses), dtype=torch.float64, device="cuda")
        res = torch.empty((3, 9), dtype=torch.float64, device="cuda")
        with pytest.raises(P.PurseError):
            P.purse_batch_solve(b, params_from(p3, 0, 0), params_from(p2, 0, 0), 0, seeds, 20000, 10, res)
        with pytest.raises(P.PurseError):
            P.purse_batch_solve(b, params_from(p3, 0, 1), params_from(p2, 0, 0), 0, seeds, 100, 10, res)
        with pytest.raises(P.PurseError):
            P.purse_batch_copy_samples(b, 5)
    finally:
        P.purse_batch_destroy(b)
