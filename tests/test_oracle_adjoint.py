"""Pins of the oracle's reverse-mode derivative (CPU only): the SO(3)
Jacobians against finite differences of Exp/Log, both ball adjoints against
central differences of the ball replays with the farthest-sample sequence
held, and the whole pipeline (walks, snap, balls) against central
differences in the observations y_i and radii r_i with the walks re-run at
+-h (a coordinate counts only where the walks and farthest sequences are
unchanged at both ends)."""
import numpy as np
import pytest

from oracle import adjoint, closure
from oracle.megb import canonical, megb_rotation_replay, megb_translation_replay, rotation_distances
from oracle.so3 import exp_so3, log_so3, quat_exp, quat_mul
from paper_2403_09990_gb300 import synthetic as syn


@pytest.mark.parametrize("th", [1e-8, 1e-3, 0.7, 2.0, 3.1])
def test_left_jacobian_and_inverse_match_finite_differences(th):
    rng = np.random.default_rng(int(th * 1e3) + 1)
    u = rng.normal(size=3)
    phi = th * u / np.linalg.norm(u)
    Jl, Jli = adjoint.jac_left(phi), adjoint.jac_left_inv(phi)
    e = 1e-6
    for i in range(3):
        d = np.zeros(3)
        d[i] = e
        # Exp(phi + e) Exp(phi)^T = Exp(J_l(phi) e)
        col = (log_so3(exp_so3(phi + d) @ exp_so3(phi).T) - log_so3(exp_so3(phi - d) @ exp_so3(phi).T)) / (2 * e)
        assert np.allclose(col, Jl[:, i], atol=1e-7)
        # Log(Exp(a) Exp(phi)) = phi + J_l(phi)^-1 a
        col = (log_so3(exp_so3(d) @ exp_so3(phi)) - log_so3(exp_so3(-d) @ exp_so3(phi))) / (2 * e)
        assert np.allclose(col, Jli[:, i], atol=2e-6 * (1 + abs(Jli).max()))
    assert np.allclose(adjoint.jac_right(phi), adjoint.jac_left(-phi))


def _cluster(n, seed):
    rng = np.random.default_rng(seed)
    C0 = quat_exp(rng.normal(size=3))
    q = quat_mul(quat_exp(rng.normal(size=(n, 3)) * np.array([0.05, 0.1, 0.3])), C0[None])
    t = rng.normal(size=(n, 3)) * np.array([0.01, 0.01, 0.05])
    return canonical(q), t


def _rot_loss(qs, f, fstar, gq, gD):
    C = megb_rotation_replay(qs, f)[-1]
    return float(gq @ C + gD * rotation_distances(C, qs[fstar:fstar + 1])[0])


@pytest.mark.parametrize("K", [1, 2, 17, 60])
def test_rotation_adjoint_matches_central_differences(K):
    qs, _ = _cluster(40, K)
    from oracle.megb import megb_rotation
    _, _, f = megb_rotation(qs, K)
    rng = np.random.default_rng(7)
    gq, gD = rng.normal(size=4), 1.3
    g, fstar = adjoint.rotation_adjoint(qs, f, gq, gD)
    h = 1e-6
    for s in sorted(set([0, fstar, 5, 11] + [int(x) for x in f[:6]])):
        for i in range(3):
            d = np.zeros(3)
            d[i] = h
            qp, qm = qs.copy(), qs.copy()
            qp[s] = canonical(quat_mul(quat_exp(d), qs[s]))
            qm[s] = canonical(quat_mul(quat_exp(-d), qs[s]))
            fd = (_rot_loss(qp, f, fstar, gq, gD) - _rot_loss(qm, f, fstar, gq, gD)) / (2 * h)
            assert abs(fd - g[s, i]) <= 1e-6 * (1 + abs(fd)), (s, i, fd, g[s, i])


@pytest.mark.parametrize("K", [1, 3, 50])
def test_translation_adjoint_matches_central_differences(K):
    _, ts = _cluster(30, 100 + K)
    from oracle.megb import megb_translation
    _, _, f = megb_translation(ts, K)
    gc, gd = np.array([0.3, -1.0, 0.5]), 0.8
    g, fstar = adjoint.translation_adjoint(ts, f, gc, gd)

    def loss(x):
        c = megb_translation_replay(x, f)[-1]
        return float(gc @ c + gd * np.linalg.norm(x[fstar] - c))

    h = 1e-6
    for s in range(len(ts)):
        for i in range(3):
            xp, xm = ts.copy(), ts.copy()
            xp[s, i] += h
            xm[s, i] -= h
            fd = (loss(xp) - loss(xm)) / (2 * h)
            assert abs(fd - g[s, i]) <= 1e-7 * (1 + abs(fd))


def _pipeline_case(kind, lam=False):
    if kind == 0:
        p = syn.purse_3d3d_ellipsoidal(8, 3) if lam else syn.purse_3d3d(8, 3)
        pr = closure.preset_3d3d(n_iter=3, rot_perturb=0.002, trans_perturb=0.002, perturb_units=1)
        pt = closure.preset_3d3d(n_iter=3, v0=0.02, rot_perturb=0.002, trans_perturb=0.002, perturb_units=1)
    else:
        p = syn.purse_2d3d_ellipsoidal(10, 3) if lam else syn.purse_2d3d(10, 3)
        pr = closure.preset_2d3d(n_iter=3, rot_perturb=0.002, trans_perturb=0.002, perturb_units=1)
        pt = pr
    return p, p.seed_pose()[None], pr, pt


@pytest.mark.parametrize("kind,lam", [(0, False), (1, False), (0, True), (1, True)])
def test_pipeline_gradient_matches_central_differences(kind, lam):
    p, seeds, pr, pt = _pipeline_case(kind, lam)
    W, K, seed = 48, 40, 11
    fw = adjoint.closure_balls(p, seeds, pr, pt, seed, W, K)
    g_res = np.array([0.2, -0.4, 0.1, 0.3, 0.5, -0.2, 0.7, 1.0, 1.0])
    gy, gr = adjoint.closure_backward(p, fw, g_res)

    def loss(q):
        fq = adjoint.closure_balls(q, seeds, pr, pt, seed, W, K)
        same = all(np.array_equal(fq[k][a], fw[k][a]) for k in ("rot", "tr") for a in ("R", "t", "jstar"))
        same = same and np.array_equal(fq["f_rot"], fw["f_rot"]) and np.array_equal(fq["f_tr"], fw["f_tr"])
        v = np.concatenate([fq["C"], fq["c"], [fq["D"], fq["d"]]])
        return float(g_res @ v), same

    h = 1e-6
    active = sorted(set(fw["rot"]["jstar"][fw["rot"]["jstar"] >= 0]) | set(fw["tr"]["jstar"][fw["tr"]["jstar"] >= 0]))
    checked = 0
    for j in active:
        for c in range(p.obs.shape[1] + 1):
            vals = []
            for sgn in (1, -1):
                obs, radii = p.obs.copy(), p.radii.copy()
                if c < p.obs.shape[1]:
                    obs[j, c] += sgn * h
                else:
                    radii[j] += sgn * h
                vals.append(loss(syn.Purse(p.kind, p.model, obs, radii, p.K, lam=p.lam)))
            if not (vals[0][1] and vals[1][1]):
                continue
            fd = (vals[0][0] - vals[1][0]) / (2 * h)
            ref = gy[j, c] if c < p.obs.shape[1] else gr[j]
            assert abs(fd - ref) <= 1e-7 + 1e-5 * abs(ref), (j, c, fd, ref)
            checked += 1
    assert checked >= 4
    assert np.abs(gr).max() > 0 and np.abs(gy).max() > 0
