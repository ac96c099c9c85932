"""Pins of the oracle's boundary snap (CPU only): the snapped samples lie on the
PURSE boundary, the active constraint is the one at zero margin, and central
finite differences of the snapped ray parameter match the implicit-function
derivatives d tau*/d r = 1/h'(tau*), d tau*/d y = -(dh/dy)/h'(tau*)."""
import numpy as np
import pytest

from oracle import closure, purse as op, snap
from paper_2403_09990_gb300 import synthetic as syn


def walked(kind, sampler, n=24, lam=False):
    if kind == 0:
        p = syn.purse_3d3d_ellipsoidal(8, 2) if lam else syn.purse_3d3d(8, 2)
        prm = closure.preset_3d3d(n_iter=3, v0=0.02, rot_perturb=0.002, trans_perturb=0.001, perturb_units=1)
    else:
        p = syn.purse_2d3d_ellipsoidal(16, 2) if lam else syn.purse_2d3d(16, 2)
        prm = closure.preset_2d3d(n_iter=3, rot_perturb=0.002, trans_perturb=0.001, perturb_units=1)
    seeds = p.seed_pose()[None]
    st = closure.center_stats(p, seeds, prm)
    w = np.arange(n)
    R0, t0 = closure.start_walks(seeds, w)
    if sampler == 0:
        R, t = closure.sample_rotation_boundary(p, seeds, prm, 5, w)
        d = closure.init_angular_velocity(R0, st.Rbar, prm.omega0, 5, w)
    else:
        R, t = closure.sample_translation_boundary(p, seeds, prm, 5, w)
        d = closure.init_center_velocity(t0, st.tbar, prm.v0, st.S, 5, w)
    return p, prm, R, t, d


CASES = [(k, s, lam) for lam in (False, True) for k in (0, 1) for s in (0, 1)]


@pytest.mark.parametrize("kind,sampler,lam", CASES)
def test_snapped_samples_are_on_the_boundary(kind, sampler, lam):
    p, prm, R, t, d = walked(kind, sampler, lam=lam)
    Rs, ts, tau, j = snap.snap(p, R, t, d, closure.step_ladder(prm), rotation=sampler == 0)
    assert (j >= 0).mean() > 0.8
    assert np.all(op.in_purse(p, Rs, ts))
    m = op.margins(p, Rs, ts)
    ok = j >= 0
    mj = m[np.arange(len(j)), np.maximum(j, 0)]
    assert np.all(np.abs(mj[ok]) <= 1e-9 * p.radii.max())
    assert np.all(m.min(axis=1)[ok] == mj[ok])


@pytest.mark.parametrize("kind,sampler,lam", CASES)
def test_snap_derivatives_match_finite_differences(kind, sampler, lam):
    p, prm, R, t, d = walked(kind, sampler, n=8, lam=lam)
    ladder = closure.step_ladder(prm)
    rot = sampler == 0
    Rs, ts, tau, j = snap.snap(p, R, t, d, ladder, rotation=rot)
    dh_dtau, dh_dy = snap.ray_derivatives(p, Rs, ts, d, j, rotation=rot)
    h = 1e-7
    checked = 0
    for w in np.nonzero(j >= 0)[0]:
        jj = int(j[w])
        taus = []
        for sgn in (1, -1):
            pr = syn.Purse(p.kind, p.model, p.obs, p.radii.copy(), p.K, lam=p.lam)
            pr.radii[jj] += sgn * h
            _, _, tw, jw = snap.snap(pr, R[w:w + 1], t[w:w + 1], d[w:w + 1], ladder, rotation=rot)
            taus.append(tw[0] if jw[0] == jj else np.nan)
        fd_r = (taus[0] - taus[1]) / (2 * h)
        if np.isfinite(fd_r):
            assert abs(fd_r - 1 / dh_dtau[w]) <= 1e-4 * abs(1 / dh_dtau[w]), (w, fd_r, 1 / dh_dtau[w])
            checked += 1
        c = 0
        taus = []
        for sgn in (1, -1):
            obs = p.obs.copy()
            obs[jj, c] += sgn * h
            pr = syn.Purse(p.kind, p.model, obs, p.radii, p.K, lam=p.lam)
            _, _, tw, jw = snap.snap(pr, R[w:w + 1], t[w:w + 1], d[w:w + 1], ladder, rotation=rot)
            taus.append(tw[0] if jw[0] == jj else np.nan)
        fd_y = (taus[0] - taus[1]) / (2 * h)
        if np.isfinite(fd_y):
            ref = -dh_dy[w, c] / dh_dtau[w]
            assert abs(fd_y - ref) <= 1e-4 * abs(1 / dh_dtau[w]), (w, fd_y, ref)
    assert checked >= 4
