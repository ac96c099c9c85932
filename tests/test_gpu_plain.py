"""Plain per-operation samplers (Alg. 3 / Alg. 5 in the paper's parallel form) against the
oracle: the same decision-trace replay as the fused walk kernel, the executed evaluation
count of the tensor formulation, and agreement with the fused kernel where neither took a
decision inside the rounding band."""
import numpy as np
import pytest
import torch

from oracle import closure, so3
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn
from tests import parity
from tests.gpu_helpers import DT, params_from, sample, to_dev
from tests.test_gpu_walk import make_case

pytestmark = pytest.mark.gpu

TOL = {0: (1e-5, 1e-5), 1: (1e-10, 1e-10)}


def sample_plain(handle, prm, sampler, precision, seed, seeds_np, n_samples):
    seeds = to_dev(seeds_np.reshape(-1, 12))
    q = torch.empty((n_samples, 4), dtype=DT[precision], device="cuda")
    t = torch.empty((n_samples, 3), dtype=DT[precision], device="cuda")
    tr = torch.full((n_samples, prm.n_iter, prm.n_keep + 2), -7, dtype=torch.int16, device="cuda")
    P.purse_sample_plain(handle, params_from(prm, sampler, precision), seed, seeds, seeds.shape[0], n_samples, q, t,
                         tr)
    P.purse_sync(handle)
    return (q.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64),
            tr.cpu().numpy().astype(np.int64))


CASES = {
    "3d3d-R-fp64": dict(kind=0, sampler=0, precision=1, prm=dict(), seeds="ransag"),
    "3d3d-R-fp32": dict(kind=0, sampler=0, precision=0, prm=dict(), seeds="ransag"),
    "2d3d-R-fp32": dict(kind=1, sampler=0, precision=0, prm=dict(), seeds="gt"),
    "2d3d-t-fp32": dict(kind=1, sampler=1, precision=0, prm=dict(), seeds="gt"),
    "2d3d-t-fp64-pca": dict(kind=1, sampler=1, precision=1, prm=dict(), seeds="multi"),
    "3d3d-t-fp32": dict(kind=0, sampler=1, precision=0, prm=dict(v0=0.02, rot_perturb=0.2), seeds="ransag"),
    "2d3d-R-fp32-keep7-np100-nt9": dict(kind=1, sampler=0, precision=0,
                                        prm=dict(n_keep=7, n_perturb=100, n_steps=9), seeds="gt"),
    "3d3d-R-fp32-keep32-np256-nt32-raw": dict(kind=0, sampler=0, precision=0,
                                              prm=dict(n_keep=32, n_perturb=256, n_steps=32, perturb_units=1,
                                                       trans_perturb=0.002), seeds="ransag"),
    "2d3d-t-fp32-n128": dict(kind=1, sampler=1, precision=0, prm=dict(n_iter=3), seeds="gt", n=128),
}


@pytest.mark.parametrize("name", list(CASES))
def test_plain_replay(name):
    c = CASES[name]
    p, prm, seeds = make_case(c)
    n = 161  # several warps and blocks plus a ragged tail
    seed = 4321
    with P.Purse(p) as h:
        q, t, tr = sample_plain(h.h, prm, c["sampler"], c["precision"], seed, seeds, n)
        evals = P.purse_last_evals(h.h)
    assert evals == n * prm.n_iter * (prm.n_perturb + prm.n_steps * prm.n_keep) * p.n
    assert tr.min() >= -1
    R, tt, rep = parity.replay_walks(p, seeds, prm, seed, np.arange(n), tr, c["precision"], c["sampler"])
    assert rep.ok(), f"inconsistent decisions: {rep.inconsistent[:10]}"
    assert not rep.robust_mismatch, rep.robust_mismatch[:10]
    atol_r, atol_t = TOL[c["precision"]]
    ang = parity.rot_angle(q, so3.quat_from_R(R))
    assert ang.max() <= atol_r, ang.max()
    assert np.abs(t - tt).max() <= atol_t, np.abs(t - tt).max()
    assert np.all(parity.classify(p, so3.R_from_quat(q), t, c["precision"]) >= 0)
    moved = (tr[:, :, prm.n_keep] >= 0).any(axis=1).mean()
    assert moved > 0.5
    print(f"{name}: robust fraction {rep.robust.mean():.3f}, moved {moved:.3f}")


@pytest.mark.parametrize("kind,sampler", [(0, 0), (1, 0), (1, 1)])
def test_plain_matches_fused_in_fp64(kind, sampler):
    """FP64: both paths replay the oracle; walks whose decisions are all outside the band
    have identical traces and poses in the two paths."""
    p = syn.purse_3d3d(8, 2) if kind == 0 else syn.purse_2d3d(16, 2)
    prm = closure.preset_3d3d(n_iter=4) if kind == 0 else closure.preset_2d3d(n_iter=4)
    seeds = p.seed_pose()[None]
    n = 300
    with P.Purse(p) as h:
        qf, tf, trf = sample(h.h, prm, sampler, 1, 99, seeds, n)
        qp, tp, trp = sample_plain(h.h, prm, sampler, 1, 99, seeds, n)
    same = (trf == trp).all(axis=(1, 2))
    assert same.mean() > 0.95, same.mean()
    assert parity.rot_angle(qf[same], qp[same]).max() < 1e-12
    assert np.abs(tf[same] - tp[same]).max() < 1e-12


def test_plain_several_chunks_sampled_parity_and_empty():
    """300000 walks span three chunks of intermediates (2^31 bytes each: FP32, N_P = 150,
    N_P* = 10, N_T = 15 take 15266 bytes per walk, so 140671 walks per chunk); walks on both
    sides of the two chunk boundaries and a random sample are replayed by the oracle.  Zero
    walks is a no-op."""
    p = syn.purse_2d3d(16, 3)
    prm = closure.preset_2d3d(n_iter=2)
    n = 300000
    per_walk = 4 * (12 * 150 + 150 + 12 * 15 * 10 + 3) + 4 * 10 + 15 * 10 + 64
    chunk = (2 << 30) // per_walk
    rng = np.random.default_rng(1)
    edges = [chunk - 1, chunk, 2 * chunk - 1, 2 * chunk]
    ids = np.unique(np.concatenate([rng.choice(n, 40, replace=False), [0, n - 1], edges]))
    seeds = p.seed_pose()[None]
    with P.Purse(p) as h:
        q, t, tr = sample_plain(h.h, prm, 0, 0, 5, seeds, n)
        q0 = torch.empty((0, 4), dtype=torch.float32, device="cuda")
        t0 = torch.empty((0, 3), dtype=torch.float32, device="cuda")
        P.purse_sample_plain(h.h, params_from(prm, 0, 0), 5, to_dev(seeds), 1, 0, q0, t0)
        P.purse_sync(h.h)
    R, tt, rep = parity.replay_walks(p, seeds, prm, 5, ids, tr[ids], 0, 0)
    assert rep.ok(), rep.inconsistent[:10]
    assert parity.rot_angle(q[ids], so3.quat_from_R(R)).max() <= 1e-5
    assert np.abs(t[ids] - tt).max() <= 1e-5
