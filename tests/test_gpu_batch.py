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
from tests.gpu_helpers import params_from, sample

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


def test_batch_gradients_equal_single_path():
    """Gradients enabled: snap records, balls and purse_batch_backward equal the single-PURSE
    purse_sample (snap) / megb_solve / megb_backward with key seed + p; 3D-3D PURSEs with v0 > 0
    take their translation ball from dS_t walks."""
    n_purses, S, K, seed = 12, 192, 40, 77
    purses = syn.purse_batch(n_purses, seed=5, n_lo=4, n_hi=40)
    p3 = closure.preset_3d3d(n_iter=3, v0=0.02, rot_perturb=0.025, trans_perturb=0.00125, perturb_units=1)
    p2 = closure.preset_2d3d(n_iter=3, rot_perturb=0.002, trans_perturb=0.002, perturb_units=1)
    seeds = torch.as_tensor(syn.seed_array(purses), dtype=torch.float64, device="cuda")
    res = torch.full((n_purses, 9), np.nan, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(0)
    g = torch.as_tensor(rng.normal(size=(n_purses, 9)), device="cuda")
    total = sum(pu.n for pu in purses)
    gy = torch.full((total, 3), np.nan, dtype=torch.float64, device="cuda")
    gr = torch.full((total,), np.nan, dtype=torch.float64, device="cuda")
    b = P.purse_batch_create(purses)
    try:
        pp3, pp2 = params_from(p3, 0, 0), params_from(p2, 0, 0)
        with pytest.raises(P.PurseError):
            P.purse_batch_backward(b, res, g, gy, gr)  # no solve with gradients yet
        P.purse_batch_set_grad(b, 1)
        P.purse_batch_solve(b, pp3, pp2, seed, seeds, S, K, res)
        P.purse_batch_backward(b, res, g, gy, gr)
        P.purse_batch_sync(b)
        far = torch.empty((n_purses, 2 * K), dtype=torch.int32, device="cuda")
        P.purse_batch_copy_farthest(b, far)
        o = 0
        for p, pu in enumerate(purses):
            prm = p3 if pu.kind == 0 else p2
            bsr = torch.empty((S, 12), device="cuda")
            bst = torch.empty((S, 12), device="cuda")
            P.purse_batch_copy_snap(b, p, bsr, bst)
            with P.Purse(pu) as h:
                sd = torch.as_tensor(pu.seed_pose()[None], dtype=torch.float64, device="cuda")
                out = []
                for sampler in (0, 1):
                    q = torch.empty((S, 4), device="cuda")
                    t = torch.empty((S, 3), device="cuda")
                    sn = torch.empty((S, 12), device="cuda")
                    P.purse_sample(h.h, params_from(prm, sampler, 0), seed + p, sd, 1, S, q, t, None, snap=sn)
                    out.append((q, t, sn))
                r1 = torch.empty(9, dtype=torch.float64, device="cuda")
                f1 = torch.empty(2 * K, dtype=torch.int32, device="cuda")
                P.megb_solve(h.h, 0, K, out[0][0], S, out[1][1], S, r1, f1)
                dim = 3 if pu.kind == 0 else 2
                y1 = torch.empty((pu.n, dim), dtype=torch.float64, device="cuda")
                rr1 = torch.empty(pu.n, dtype=torch.float64, device="cuda")
                P.megb_backward(h.h, 0, K, out[0][0], out[0][2], S, out[1][1], out[1][2], S, f1, r1, g[p].contiguous(),
                                y1, rr1)
                P.purse_sync(h.h)
            torch.cuda.synchronize()
            assert torch.equal(out[0][2], bsr) and torch.equal(out[1][2], bst), p
            assert torch.equal(f1, far[p]), p
            assert torch.allclose(r1, res[p], rtol=1e-12, atol=1e-15), p
            gyb, grb = gy[o:o + pu.n], gr[o:o + pu.n]
            assert torch.allclose(y1, gyb[:, :dim], rtol=1e-10, atol=1e-12 * float(y1.abs().max())), p
            assert torch.allclose(rr1, grb, rtol=1e-10, atol=1e-12 * float(rr1.abs().max())), p
            if dim == 2:
                assert torch.all(gyb[:, 2] == 0)
            assert float(rr1.abs().max()) > 0
            o += pu.n
    finally:
        P.purse_batch_destroy(b)


def test_batch_full_size_sampled():
    """The batched workload at full size and in the bench's launch configuration (4096 PURSEs of
    4096 samples, autotuned launch, graph replay): eight sampled PURSEs equal the single-PURSE path
    bit for bit, sixteen sampled walks of two of them are replayed by the oracle, every result is
    finite and every ball radius is positive."""
    n_purses, S, K = 4096, 4096, 200
    purses = syn.purse_batch(n_purses, seed=7)
    p3, p2 = presets()
    seeds = torch.as_tensor(syn.seed_array(purses), dtype=torch.float64, device="cuda")
    res = torch.full((n_purses, 9), np.nan, dtype=torch.float64, device="cuda")
    pp3, pp2 = params_from(p3, 0, 0), params_from(p2, 0, 0)
    b = P.purse_batch_create(purses)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(n_purses, 8, replace=False))
    try:
        P.purse_batch_tune(b, pp3, pp2, 1, seeds, 1024)
        P.purse_batch_solve(b, pp3, pp2, 55, seeds, S, K, res)
        P.purse_batch_sync(b)
        r = res.cpu().numpy()
        assert np.all(np.isfinite(r)) and np.all(r[:, 7] > 0) and np.all(r[:, 8] > 0)
        for n, p in enumerate(pick):
            pu = purses[p]
            bq, bt = torch.empty((S, 4), device="cuda"), torch.empty((S, 3), device="cuda")
            bq2, bt2 = torch.empty((S, 4), device="cuda"), torch.empty((S, 3), device="cuda")
            P.purse_batch_copy_samples(b, int(p), bq, bt, bq2, bt2)
            torch.cuda.synchronize()
            prm = p3 if pu.kind == 0 else p2
            q, t = single(pu, prm, 0, 55 + int(p), S)
            assert torch.equal(q, bq) and torch.equal(t, bt), p
            if n < 2:  # oracle replay of sampled walks of this PURSE (the batch draws with key seed + p)
                ids = np.sort(rng.choice(S, 8, replace=False))
                with P.Purse(pu) as h:
                    _, _, tr = sample(h.h, prm, 0, 0, 55 + int(p), pu.seed_pose()[None], S, trace_rows=ids)
                R, tt, rep = parity.replay_walks(pu, pu.seed_pose()[None], prm, 55 + int(p), ids, tr, 0, 0)
                assert rep.ok(), rep.inconsistent[:5]
                qn = q.cpu().numpy()[ids].astype(np.float64)
                assert parity.rot_angle(qn, so3.quat_from_R(R)).max() <= 1e-5
    finally:
        P.purse_batch_destroy(b)


def test_batch_noise_matrices_equal_single_path():
    """purse_batch_set_noise (eq. 4 over a batch): PURSE p gives exactly the samples, snap records,
    farthest sequences, balls and gradients of purse_sample / megb_solve / megb_backward on a handle
    given the same matrices by purse_set_noise; one PURSE without matrices keeps the identity norm."""
    rng = np.random.default_rng(3)
    purses = []
    for p in range(9):
        n = int(rng.integers(4, 40))
        purses.append(syn.purse_3d3d_ellipsoidal(n, 100 + p) if p % 2 == 0 else syn.purse_2d3d_ellipsoidal(n, 100 + p))
    purses.append(syn.purse_2d3d(12, 5))
    n_purses, S, K, seed = len(purses), 160, 30, 91
    p3 = closure.preset_3d3d(n_iter=3, v0=0.02, rot_perturb=0.025, trans_perturb=0.00125, perturb_units=1)
    p2 = closure.preset_2d3d(n_iter=3, rot_perturb=0.002, trans_perturb=0.002, perturb_units=1)
    seeds = torch.as_tensor(syn.seed_array(purses), dtype=torch.float64, device="cuda")
    res = torch.full((n_purses, 9), np.nan, dtype=torch.float64, device="cuda")
    g = torch.as_tensor(rng.normal(size=(n_purses, 9)), device="cuda")
    total = sum(pu.n for pu in purses)
    gy = torch.full((total, 3), np.nan, dtype=torch.float64, device="cuda")
    gr = torch.full((total,), np.nan, dtype=torch.float64, device="cuda")
    b = P.purse_batch_create(purses)
    try:
        bad = [syn.purse_3d3d_ellipsoidal(p.n, 1) if p.kind == 0 else p for p in purses]
        bad[0].lam = -bad[0].lam  # not positive definite
        with pytest.raises(P.PurseError):
            P.purse_batch_set_noise(b, bad)
        P.purse_batch_set_noise(b, purses)
        pp3, pp2 = params_from(p3, 0, 0), params_from(p2, 0, 0)
        P.purse_batch_set_grad(b, 1)
        P.purse_batch_solve(b, pp3, pp2, seed, seeds, S, K, res)
        P.purse_batch_backward(b, res, g, gy, gr)
        P.purse_batch_sync(b)
        far = torch.empty((n_purses, 2 * K), dtype=torch.int32, device="cuda")
        P.purse_batch_copy_farthest(b, far)
        o = 0
        for p, pu in enumerate(purses):
            prm = p3 if pu.kind == 0 else p2
            bq, bt = torch.empty((S, 4), device="cuda"), torch.empty((S, 3), device="cuda")
            bq2, bt2 = torch.empty((S, 4), device="cuda"), torch.empty((S, 3), device="cuda")
            P.purse_batch_copy_samples(b, p, bq, bt, bq2, bt2)
            bsr, bst = torch.empty((S, 12), device="cuda"), torch.empty((S, 12), device="cuda")
            P.purse_batch_copy_snap(b, p, bsr, bst)
            with P.Purse(pu) as h:
                sd = torch.as_tensor(pu.seed_pose()[None], dtype=torch.float64, device="cuda")
                out = []
                for sampler in (0, 1):
                    q = torch.empty((S, 4), device="cuda")
                    t = torch.empty((S, 3), device="cuda")
                    sn = torch.empty((S, 12), device="cuda")
                    P.purse_sample(h.h, params_from(prm, sampler, 0), seed + p, sd, 1, S, q, t, None, snap=sn)
                    out.append((q, t, sn))
                r1 = torch.empty(9, dtype=torch.float64, device="cuda")
                f1 = torch.empty(2 * K, dtype=torch.int32, device="cuda")
                P.megb_solve(h.h, 0, K, out[0][0], S, out[1][1], S, r1, f1)
                dim = 3 if pu.kind == 0 else 2
                y1 = torch.empty((pu.n, dim), dtype=torch.float64, device="cuda")
                rr1 = torch.empty(pu.n, dtype=torch.float64, device="cuda")
                P.megb_backward(h.h, 0, K, out[0][0], out[0][2], S, out[1][1], out[1][2], S, f1, r1, g[p].contiguous(),
                                y1, rr1)
                P.purse_sync(h.h)
            torch.cuda.synchronize()
            assert torch.equal(out[0][0], bq) and torch.equal(out[0][1], bt), p
            assert torch.equal(out[1][0], bq2) and torch.equal(out[1][1], bt2), p
            assert torch.equal(out[0][2], bsr) and torch.equal(out[1][2], bst), p
            assert torch.equal(f1, far[p]), p
            assert torch.allclose(r1, res[p], rtol=1e-12, atol=1e-15), p
            gyb, grb = gy[o:o + pu.n], gr[o:o + pu.n]
            assert torch.allclose(y1, gyb[:, :dim], rtol=1e-10, atol=1e-12 * float(y1.abs().max())), p
            assert torch.allclose(rr1, grb, rtol=1e-10, atol=1e-12 * float(rr1.abs().max())), p
            o += pu.n
        # back to the identity norm: the next solve captures a new graph and runs
        P.purse_batch_set_noise(b, None)
        P.purse_batch_solve(b, pp3, pp2, seed, seeds, S, K, res)
        P.purse_batch_sync(b)
        assert torch.all(torch.isfinite(res))
    finally:
        P.purse_batch_destroy(b)


def test_batch_regression_equals_single_path():
    """purse_batch_create_regression (Example 3 over a batch): PURSE p gives exactly the samples of
    both samplers, the farthest sequences and the balls of purse_sample / megb_solve on a regression
    handle with key seed + p; snap, gradients and noise matrices are refused."""
    rng = np.random.default_rng(4)
    purses = [syn.purse_reg(int(n), 200 + p) for p, n in enumerate([1, 3, 10, 29, 7, 16, 40])]
    purses.append(syn.purse_reg_nested(10, 3))
    n_purses, S, K, seed = len(purses), 300, 40, 123
    prm = closure.preset_reg(n_iter=4, rot_perturb=0.2, v0=0.02)
    seeds = torch.as_tensor(syn.seed_array(purses), dtype=torch.float64, device="cuda")
    res = torch.full((n_purses, 9), np.nan, dtype=torch.float64, device="cuda")
    b = P.purse_batch_create_regression(purses)
    try:
        pp = params_from(prm, 0, 0)
        with pytest.raises(P.PurseError):
            P.purse_batch_set_grad(b, 1)
        with pytest.raises(P.PurseError):
            P.purse_batch_set_noise(b, None)
        P.purse_batch_solve(b, pp, pp, seed, seeds, S, K, res)
        evals = P.purse_batch_sync(b)
        assert evals > 0
        far = torch.empty((n_purses, 2 * K), dtype=torch.int32, device="cuda")
        P.purse_batch_copy_farthest(b, far)
        for p, pu in enumerate(purses):
            bq, bt = torch.empty((S, 4), device="cuda"), torch.empty((S, 3), device="cuda")
            bq2, bt2 = torch.empty((S, 4), device="cuda"), torch.empty((S, 3), device="cuda")
            P.purse_batch_copy_samples(b, p, bq, bt, bq2, bt2)
            torch.cuda.synchronize()
            q, t = single(pu, prm, 0, seed + p, S)
            q2, t2 = single(pu, prm, 1, seed + p, S)
            assert torch.equal(q, bq) and torch.equal(t, bt), p
            assert torch.equal(q2, bq2) and torch.equal(t2, bt2), p
            r1 = torch.empty(9, dtype=torch.float64, device="cuda")
            f1 = torch.empty(2 * K, dtype=torch.int32, device="cuda")
            with P.Purse(pu) as h:
                P.megb_solve(h.h, 0, K, q, S, t2, S, r1, f1)
                P.purse_sync(h.h)
            assert torch.equal(f1, far[p]), p
            assert torch.allclose(r1, res[p], rtol=1e-12, atol=1e-15), (p, r1, res[p])
            for qq, tt in ((q, t), (q2, t2)):  # every sample of both samplers inside its PURSE
                qn, tn = qq.cpu().numpy().astype(np.float64), tt.cpu().numpy().astype(np.float64)
                assert np.all(parity.classify(pu, so3.R_from_quat(qn), tn, 0) >= 0), p
    finally:
        P.purse_batch_destroy(b)
