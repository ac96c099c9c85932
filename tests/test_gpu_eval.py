"""purse_eval (eq. 2/3, eq. 11, SE(3) gradient) against the oracle, element by element."""
import numpy as np
import pytest
import torch

from oracle import purse as op
from oracle import so3
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn
from tests.gpu_helpers import DT, to_dev
from tests.parity import constraint_bands

pytestmark = pytest.mark.gpu


def poses_near(p, n, seed, behind=0):
    rng = np.random.default_rng(seed)
    R = so3.exp_so3(rng.normal(size=(n, 3)) * 0.02) @ p.R_gt
    scale = np.array([0.004, 0.004, 0.04]) if p.kind == 1 else np.full(3, 0.01)
    t = p.t_gt + rng.normal(size=(n, 3)) * scale
    if behind:
        t[:behind, 2] = -t[:behind, 2]
    return R, t


@pytest.mark.parametrize("kind,n,precision", [(0, 8, 1), (0, 8, 0), (1, 16, 0), (1, 16, 1), (0, 3, 0),
                                              (1, 256, 0), (0, 64, 0)])
def test_eval_matches_oracle(kind, n, precision):
    p = syn.purse_3d3d(n, 3) if kind == 0 else syn.purse_2d3d(n, 3)
    npose = 1000 + 37  # several blocks and a ragged tail
    R, t = poses_near(p, npose, 5, behind=5 if kind == 1 else 0)
    poses = np.concatenate([R.reshape(-1, 9), t], axis=1)
    with P.Purse(p) as h:
        d_poses = to_dev(poses, DT[precision])
        margin = torch.empty((npose, n), dtype=DT[precision], device="cuda")
        active = torch.empty(npose, dtype=torch.int32, device="cuda")
        grad = torch.empty((npose, 6), dtype=DT[precision], device="cuda")
        P.purse_eval(h.h, precision, d_poses, npose, margin, active, grad)
        P.purse_sync(h.h)
        # zero poses is a no-op
        P.purse_eval(h.h, precision, d_poses, 0, margin, active, grad)
    m_gpu = margin.cpu().numpy().astype(np.float64)
    a_gpu = active.cpu().numpy()
    g_gpu = grad.cpu().numpy().astype(np.float64)
    Rq = poses[:, :9].reshape(-1, 3, 3)
    if precision == 0:  # the oracle evaluates the FP32-rounded poses the GPU saw
        Rq = Rq.astype(np.float32).astype(np.float64)
        tq = poses[:, 9:].astype(np.float32).astype(np.float64)
    else:
        tq = poses[:, 9:]
    m_ref = op.margins(p, Rq, tq)
    finite = np.isfinite(m_ref)
    assert np.array_equal(finite, np.isfinite(m_gpu))
    assert np.all(m_gpu[~finite] == -np.inf)
    band = constraint_bands(p, Rq, tq, precision)
    assert np.all(np.abs(m_gpu[finite] - m_ref[finite]) <= band[finite])
    # active constraint: unique where the two smallest margins are separated by more than the bands
    srt = np.sort(np.where(finite, m_ref, -1e300), axis=1)
    clear = (srt[:, 1] - srt[:, 0]) > 2 * band.max(axis=1)
    a_ref = np.argmin(np.where(finite, m_ref, -1e300), axis=1)
    assert np.array_equal(a_gpu[clear], a_ref[clear])
    assert clear.mean() > 0.9
    # gradient of the active constraint's residual norm
    G = op.margin_gradient(p, Rq, tq)
    rows = np.arange(npose)
    ok = clear & np.isfinite(m_ref[rows, a_ref])
    g_ref = G[rows, a_ref][ok]
    # Bound from the arithmetic: the gradient is (R a_j x w, w) with w the unit residual direction
    # (2D-3D: pulled back through the projection and K).  The residual g_j is a difference of
    # terms of size mag_j, so its rounding error is within the band's 8 eps mag_j, and the unit
    # direction moves by at most twice that over |g_j|; the remaining products add a few eps.
    eps = 2.0 ** -23 if precision == 0 else 2.0 ** -52
    a_ok = a_ref[ok]
    r_act = p.radii[a_ok]
    e_norm = r_act - m_ref[rows, a_ref][ok]                     # |g_j| of the active constraint
    rounding = band[rows, a_ref][ok] - 1e-6 * r_act             # 8 eps mag_j
    rel = 2.0 * rounding / e_norm + 64 * eps
    scale = np.abs(g_ref).max(axis=1)
    err = np.abs(g_gpu[ok] - g_ref).max(axis=1)
    assert np.all(err <= rel * scale), (err / scale / rel).max()
