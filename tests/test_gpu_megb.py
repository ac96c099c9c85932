"""GGD ball kernels against the oracle: the GPU's farthest-sample sequence is
checked against FP64 distances (within the rounding band) and replayed; the
centres, D-hat and d-hat must agree with FP64."""
import numpy as np
import pytest

from oracle import megb as om
from oracle import so3
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn
from tests import parity
from tests.gpu_helpers import megb
from tests.parity import EPS, check_rotation, check_translation, rot_keys  # noqa: F401

pytestmark = pytest.mark.gpu


def cluster(n, seed, spread=(0.02, 0.05, 0.1)):
    rng = np.random.default_rng(seed)
    C0 = so3.quat_from_R(so3.exp_so3(rng.normal(size=3)))
    q = so3.quat_mul(so3.quat_exp(rng.normal(size=(n, 3)) * np.array(spread)), C0[None])
    t = rng.normal(size=(n, 3)) * np.array([0.003, 0.003, 0.03]) + rng.normal(size=3)
    return q, t


@pytest.mark.parametrize("n,K,precision", [(1, 5, 0), (2, 7, 0), (1000, 200, 0), (4096, 200, 1), (4096, 200, 0),
                                           (1 << 18, 200, 0), (77777, 50, 1)])
def test_megb_replay(n, K, precision):
    q, t = cluster(n, n)
    dt = np.float32 if precision == 0 else np.float64
    q32, t32 = q.astype(dt), t.astype(dt)
    with P.Purse(syn.purse_3d3d(8, 0)) as h:
        res, far = megb(h.h, precision, K, q32, t32)
    assert far.min() >= 0 and far.max() < n
    q64, t64 = q32.astype(np.float64), t32.astype(np.float64)
    C, D = check_rotation(q64, res, far[:K], precision)
    c, d = check_translation(t64, res, far[K:], precision)
    if n == 1:
        assert res[7] <= 1e-12 and res[8] <= 1e-12
    # containment and diameter bounds on a subsample
    sub = np.random.default_rng(0).choice(n, min(n, 2000), replace=False)
    dq = om.rotation_distances(res[:4], om.canonical(q64[sub]))
    assert np.all(dq <= res[7] + 1e-12)
    dmax = max(so3.dist_quat(om.canonical(q64[s])[None], om.canonical(q64[sub])).max() for s in sub[:200])
    assert res[7] >= dmax / 2 - 1e-12


def test_megb_one_ball_only():
    q, t = cluster(500, 3)
    with P.Purse(syn.purse_3d3d(8, 0)) as h:
        res, far = megb(h.h, 0, 20, q.astype(np.float32), None)
        assert res[8] == 0 and np.all(res[4:7] == 0) and res[7] > 0
        res2, _ = megb(h.h, 0, 20, None, t.astype(np.float32))
        assert res2[7] == 0 and res2[8] > 0


def test_megb_closed_form_geodesic():
    # rotations about one axis: the ball is the middle of the arc with radius half its length
    rng = np.random.default_rng(1)
    C0 = so3.quat_from_R(so3.exp_so3(rng.normal(size=3)))
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    ang = rng.uniform(-0.3, 0.5, 3000)
    q = so3.quat_mul(so3.quat_exp(ang[:, None] * u), C0[None])
    K = 400
    with P.Purse(syn.purse_3d3d(8, 0)) as h:
        res, _ = megb(h.h, 1, K, q, None)
    half = 0.5 * (ang.max() - ang.min())
    assert half * (1 - 1e-12) <= res[7] <= half * (1 + 1 / np.sqrt(K))


@pytest.mark.parametrize("precision", [0, 1])
def test_rotation_ball_with_radius_near_pi(precision):
    """Samples up to 3.1 rad from a centre in every direction: the keys sin^2(theta/2) flatten near pi
    (FP32 resolves about 3e-6 rad there) and the final angle comes from the FP64 log map."""
    rng = np.random.default_rng(11)
    n, K = 20000, 100
    C0 = so3.quat_from_R(so3.exp_so3(rng.normal(size=3)))
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    th = 3.1 * rng.random(n) ** (1 / 3)
    q = so3.quat_mul(so3.quat_exp(u * th[:, None]), C0[None])
    if precision == 0:
        q = q.astype(np.float32).astype(np.float64)  # the samples the FP32 kernels see
    with P.Purse(syn.purse_3d3d(8, 0)) as h:
        res, f = megb(h.h, precision, K, q, None)
    _, D = check_rotation(q, res, f[:K], precision)
    assert D > 3.0


def megb_mean(handle, precision, K, n_last, q_np, t_np):
    import torch
    from tests.gpu_helpers import DT, to_dev
    q, t = to_dev(q_np, DT[precision]), to_dev(t_np, DT[precision])
    res = torch.full((9,), np.nan, dtype=torch.float64, device="cuda")
    far = torch.full((2 * K,), -1, dtype=torch.int32, device="cuda")
    P.megb_solve_mean(handle, precision, K, n_last, q, q_np.shape[0], t, t_np.shape[0], res, far)
    P.purse_sync(handle)
    return res.cpu().numpy(), far.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("n,K,n_last,precision", [(4096, 200, 10, 1), (4096, 200, 10, 0), (1 << 18, 200, 10, 0),
                                                  (1000, 5, 10, 0), (3001, 50, 1, 0), (20000, 37, 12, 1)])
def test_megb_mean_output_rule(n, K, n_last, precision):
    """Alg. 6's output rule: the same farthest samples as megb_solve, then the centres from the last
    n_last iterates, against the oracle replaying the GPU's (band-checked) farthest sequence."""
    q, t = cluster(n, n + 1)
    dt = np.float32 if precision == 0 else np.float64
    q32, t32 = q.astype(dt), t.astype(dt)
    with P.Purse(syn.purse_3d3d(8, 0)) as h:
        res, far = megb(h.h, precision, K, q32, t32)
        resm, farm = megb_mean(h.h, precision, K, n_last, q32, t32)
        # megb_backward differentiates megb_solve's plain output only
        with pytest.raises(P.PurseError):
            P.megb_backward(h.h, precision, K, None, None, 0, None, None, 0, None, None, None, None, None)
    assert np.array_equal(far, farm)
    q64, t64 = q32.astype(np.float64), t32.astype(np.float64)
    check_rotation(q64, res, far[:K], precision)
    check_translation(t64, res, far[K:], precision)
    if n_last == 1:
        assert np.array_equal(res, resm)
    C, D, _ = om.megb_rotation_mean(q64, K, n_last, f=far[:K])
    c, d, _ = om.megb_translation_mean(t64, K, n_last, f=far[K:])
    assert so3.dist_quat(resm[:4][None], C[None])[0] <= 1e-9
    assert resm[0] >= 0 and abs(np.linalg.norm(resm[:4]) - 1) < 1e-12
    assert np.abs(resm[4:7] - c).max() <= 1e-9 * (1 + np.abs(c).max())
    assert abs(resm[7] - D) <= 1e-5 * D + 1e-12 and abs(resm[8] - d) <= 1e-5 * d + 1e-12
    if n_last > 1 and K >= n_last:
        assert so3.dist_quat(resm[:4][None], res[:4][None])[0] > 0  # a different centre than C_K
