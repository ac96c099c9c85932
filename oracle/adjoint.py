"""Reverse-mode derivative of the enclosing balls through the boundary snap
(FP64, oracle side; test infrastructure only).

Conventions.  Rotations are perturbed on the left, R -> Exp(delta) R (world
frame), for samples and centres alike; the SO(3) Jacobians are
  J_l(phi)      = I + (1 - cos th)/th^2 [phi]x + (th - sin th)/th^3 [phi]x^2,
  J_l(phi)^-1   = I - [phi]x / 2 + (1/th^2 - cot(th/2) / (2 th)) [phi]x^2,
  J_r(phi)      = J_l(-phi),
so that Exp(phi + e) = Exp(J_l(phi) e) Exp(phi) and
Log(Exp(a) Exp(phi)) = phi + J_l(phi)^-1 a to first order.

Rotation ball (Section II, geodesic gradient descent with step 1/k):
  phi_k = Log(C_{k-1}^T R_{f_k}),  C_k = C_{k-1} Exp(phi_k / k),
linearised in the centre perturbation eps_k and the sample perturbations
delta_s:
  eps_k = (I - A_k) eps_{k-1} + A_k delta_{f_k},
  A_k   = (1/k) C_k J_r(phi_k / k) J_l(phi_k)^-1 C_{k-1}^T,
and eps_0 = delta_{s=0} (C_0 is the first sample).  The radius is the
geodesic distance D = |psi|, psi = Log(C_K^T R_{f*}) with f* the farthest
sample from C_K; since J_l(psi)^-T psi = psi,
  dD = (C_K u)^T (delta_{f*} - eps_K),  u = psi / |psi|,
the direction of the gradient of the squared distance given in the
appendix on geodesic gradient descent.  The reverse sweep takes
lambda_K = dL/d eps_K, then for k = K..1: g[f_k] += A_k^T lambda_k,
lambda_{k-1} = lambda_k - A_k^T lambda_k.

Translation ball (Badoiu-Clarkson): c_k = c_{k-1} + (t_{f_k} - c_{k-1}) / k,
d = |t_{f*} - c_K|; reverse: mu_K = dL/dc_K, g[f_k] += mu_k / k,
mu_{k-1} = (1 - 1/k) mu_k.

Snap (reading: each final sample moved along its last move direction to
the boundary, see oracle.snap): at the snapped sample h_j*(x(tau*)) = r_j*,
so d tau* = (d r_j* - (dh/dy) . d y_j*) / h'(tau*) and the sample moves by
direction * d tau* (a left rotation perturbation for the rotation ray, a
translation for the translation ray).  A sample whose ray does not move the
coordinate its ball uses (a rotation-ray sample in the translation ball)
contributes nothing.

The centre quaternion gradient dL/dq_C (4 values, q_C with w >= 0) maps to
the left tangent as g_C = (w g_v - g_w v + v x g_v) / 2, from
dq = (0, eps) (x) q / 2.

Parity: pinned in tests/test_oracle_adjoint.py (the Jacobians against finite
differences of Exp/Log; both ball adjoints against central differences of
the ball replays; the whole pipeline -- walks, snap, balls -- against
central differences in y and r with the walks re-run at +-h).
"""
from __future__ import annotations

import numpy as np

from . import closure, snap
from .megb import canonical, megb_rotation, megb_translation
from .so3 import R_from_quat, exp_so3, hat, log_so3, quat_from_R


def jac_left(phi):
    phi = np.asarray(phi, dtype=np.float64)
    th = float(np.linalg.norm(phi))
    V = hat(phi)
    if th < 1e-5:
        a, b = 0.5 - th * th / 24.0, 1.0 / 6.0 - th * th / 120.0
    else:
        a, b = (1.0 - np.cos(th)) / th ** 2, (th - np.sin(th)) / th ** 3
    return np.eye(3) + a * V + b * (V @ V)


def jac_left_inv(phi):
    phi = np.asarray(phi, dtype=np.float64)
    th = float(np.linalg.norm(phi))
    V = hat(phi)
    if th < 1e-5:
        c = 1.0 / 12.0 + th * th / 720.0
    else:
        c = 1.0 / th ** 2 - 1.0 / (2.0 * th * np.tan(0.5 * th))
    return np.eye(3) - 0.5 * V + c * (V @ V)


def jac_right(phi):
    return jac_left(-np.asarray(phi, dtype=np.float64))


def quat_grad_to_tangent(q, gq):
    """dL/d(eps) for q -> Exp(eps) q, from dL/dq."""
    w, v = q[0], np.asarray(q[1:])
    gw, gv = gq[0], np.asarray(gq[1:])
    return 0.5 * (w * gv - gw * v + np.cross(v, gv))


def rotation_adjoint(qs, f, gq, gD):
    """Gradient of L = gq . C_K + gD D with respect to left perturbations of every sample (S, 3)."""
    qs = canonical(qs)
    Rs = R_from_quat(qs)
    C = [Rs[0]]
    phis = []
    for k, fk in enumerate(f, start=1):
        phi = log_so3(C[-1].T @ Rs[int(fk)])
        phis.append(phi)
        C.append(C[-1] @ exp_so3(phi / k))
    CK = C[-1]
    g = np.zeros((len(qs), 3))
    dist = np.linalg.norm(log_so3(np.einsum('ji,sjk->sik', CK, Rs)), axis=1)
    fstar = int(np.argmax(dist))
    psi = log_so3(CK.T @ Rs[fstar])
    lam = quat_grad_to_tangent(canonical(quat_from_R(CK)), np.asarray(gq, dtype=np.float64))
    if np.linalg.norm(psi) > 0:
        w = CK @ (psi / np.linalg.norm(psi))
        g[fstar] += gD * w
        lam = lam - gD * w
    for k in range(len(f), 0, -1):
        A = C[k] @ jac_right(phis[k - 1] / k) @ jac_left_inv(phis[k - 1]) @ C[k - 1].T / k
        v = A.T @ lam
        g[int(f[k - 1])] += v
        lam = lam - v
    g[0] += lam
    return g, fstar


def translation_adjoint(ts, f, gc, gd):
    """Gradient of L = gc . c_K + gd d with respect to every sample translation (S, 3)."""
    ts = np.asarray(ts, dtype=np.float64)
    c = ts[0].copy()
    for k, fk in enumerate(f, start=1):
        c = c + (ts[int(fk)] - c) / k
    g = np.zeros_like(ts)
    dist = np.linalg.norm(ts - c, axis=1)
    fstar = int(np.argmax(dist))
    mu = np.asarray(gc, dtype=np.float64).copy()
    if dist[fstar] > 0:
        e = (ts[fstar] - c) / dist[fstar]
        g[fstar] += gd * e
        mu = mu - gd * e
    for k in range(len(f), 0, -1):
        g[int(f[k - 1])] += mu / k
        mu = mu * (1.0 - 1.0 / k)
    g[0] += mu
    return g, fstar


def snap_scatter(purse, g, jstar, ray_is_rotation, ball_is_rotation, direction, dh_dtau, dh_dy):
    """Push sample gradients g (S, 3) through the snap onto (grad_obs (N, dim), grad_radii (N,))."""
    dim = purse.obs.shape[1]
    gy = np.zeros((len(purse.radii), dim))
    gr = np.zeros(len(purse.radii))
    if ray_is_rotation != ball_is_rotation:
        return gy, gr
    for s in np.nonzero((jstar >= 0) & np.any(g != 0, axis=1))[0]:
        gt = float(g[s] @ direction[s]) / dh_dtau[s]
        gr[jstar[s]] += gt
        gy[jstar[s]] -= gt * dh_dy[s][:dim]
    return gy, gr


def closure_balls(purse, seeds, prm_rot, prm_tr, seed, n_walks, K, rot_sampler=0, tr_sampler=1):
    """Forward pipeline with snap: walks (Alg. 3 / Alg. 5), snap, GGD balls.

    The rotation ball takes the rotations of sampler rot_sampler, the translation
    ball the translations of sampler tr_sampler (0: dS_R, 1: dS_t).  Returns a
    dict with the pre-snap samples, snap records, balls and farthest sequences."""
    w = np.arange(n_walks)
    out = {}
    for key, sampler, prm in (("rot", rot_sampler, prm_rot), ("tr", tr_sampler, prm_tr)):
        st = closure.center_stats(purse, seeds, prm)
        R0, t0 = closure.start_walks(seeds, w)
        if sampler == 0:
            R, t = closure.sample_rotation_boundary(purse, seeds, prm, seed, w, st)
            d = closure.init_angular_velocity(R0, st.Rbar, prm.omega0, seed, w)
        else:
            R, t = closure.sample_translation_boundary(purse, seeds, prm, seed, w, st)
            d = closure.init_center_velocity(t0, st.tbar, prm.v0, st.S, seed, w)
        rot = sampler == 0
        Rs, ts, tau, j = snap.snap(purse, R, t, d, closure.step_ladder(prm), rotation=rot)
        dh_dtau, dh_dy = snap.ray_derivatives(purse, Rs, ts, d, j, rotation=rot)
        out[key] = dict(R=R, t=t, Rs=Rs, ts=ts, dir=d, jstar=j, ray_rot=rot, dh_dtau=dh_dtau, dh_dy=dh_dy)
    qs = canonical(quat_from_R(out["rot"]["Rs"]))
    C, D, f_rot = megb_rotation(qs, K)
    c, dd, f_tr = megb_translation(out["tr"]["ts"], K)
    out.update(q=qs, C=C, D=D, f_rot=f_rot, c=c, d=dd, f_tr=f_tr)
    return out


def closure_backward(purse, fw, g_result):
    """(grad_obs, grad_radii) of L = g_result . (C (4), c (3), D, d) for a closure_balls result."""
    g_result = np.asarray(g_result, dtype=np.float64)
    g_rot, _ = rotation_adjoint(fw["q"], fw["f_rot"], g_result[:4], g_result[7])
    g_tr, _ = translation_adjoint(fw["tr"]["ts"], fw["f_tr"], g_result[4:7], g_result[8])
    gy = np.zeros(purse.obs.shape)
    gr = np.zeros(len(purse.radii))
    for key, g, ball_rot in (("rot", g_rot, True), ("tr", g_tr, False)):
        r = fw[key]
        y, rr = snap_scatter(purse, g, r["jstar"], r["ray_rot"], ball_rot, r["dir"], r["dh_dtau"], r["dh_dy"])
        gy += y
        gr += rr
    return gy, gr
