"""Parity helpers: error bands and the replay of GPU decision traces.

A walk is a chain of discrete decisions (top-k ranks, the first feasible rung
of the ladder) taken on floating-point values; the GPU takes them in FP32 (or
FP64), the oracle in FP64.  The protocol:

* band: a decision whose deciding margin lies within the rounding band of the
  GPU arithmetic is ambiguous; either outcome is accepted.  The band of a
  constraint is 1e-6 r_i + 8 eps (|R a_i| + |t| + |b_i|) for 3D-3D and
  1e-6 r_i + 8 eps (|P_x| + |u_i P_z| + |P_y| + |v_i P_z|) / P_z for 2D-3D,
  eps the unit roundoff of the GPU arithmetic type.
* replay: the oracle recomputes every iteration in FP64, checks that each
  decision of the GPU trace is consistent with its own values outside the
  band, then follows the GPU's decision; the final poses must agree to the
  stated tolerances.
* free run: walks whose every decision is outside the band in the oracle's
  own free run must have exactly the GPU's trace.
"""
from __future__ import annotations

import numpy as np

from oracle import closure, philox
from oracle import megb as megb_o
from oracle import so3 as so3_o
from oracle import purse as op
from oracle.purse import KIND_2D3D, KIND_REG

EPS = {0: 2.0 ** -23, 1: 2.0 ** -52}


def constraint_bands(purse, R, t, precision):
    """(..., N) band of each constraint's margin at poses (R, t) ((..., 2N) for pose regression:
    1e-6 beta + 8 eps times the norms of the two matrices, or of the two translations)."""
    eps = EPS[precision]
    if purse.kind == KIND_REG:
        R = np.asarray(R, dtype=np.float64)
        t = np.asarray(t, dtype=np.float64)
        bR = 1e-6 * purse.radii_rot + 8.0 * eps * (np.sqrt((R ** 2).sum(axis=(-2, -1)))[..., None]
                                                   + np.sqrt((purse.rot_hyp ** 2).sum(axis=(-2, -1))))
        bt = 1e-6 * purse.radii + 8.0 * eps * (np.linalg.norm(t, axis=-1)[..., None]
                                               + np.linalg.norm(purse.obs, axis=-1))
        lead = np.broadcast_shapes(bR.shape[:-1], bt.shape[:-1])
        return np.concatenate([np.broadcast_to(bR, lead + bR.shape[-1:]),
                               np.broadcast_to(bt, lead + bt.shape[-1:])], axis=-1)
    X = op.transform(purse.model, R, t)
    lam = getattr(purse, "lam", None)
    # with noise matrices (eq. 4) a residual error grows by at most sqrt(lambda_max(Lambda_i))
    lscale = 1.0 if lam is None else np.sqrt(np.linalg.eigvalsh(lam)[:, -1])
    if purse.kind == KIND_2D3D:
        fx, fy, cx, cy = purse.K
        Px = fx * X[..., 0] + cx * X[..., 2]
        Py = fy * X[..., 1] + cy * X[..., 2]
        Pz = X[..., 2]
        u, v = purse.obs[:, 0], purse.obs[:, 1]
        Pzs = np.where(Pz > 0, Pz, 1.0)
        mag = (np.abs(Px) + np.abs(u * Pz) + np.abs(Py) + np.abs(v * Pz)) / Pzs
    else:
        RA = X - np.asarray(t)[..., None, :]
        mag = (np.linalg.norm(RA, axis=-1) + np.linalg.norm(np.asarray(t), axis=-1)[..., None]
               + np.linalg.norm(purse.obs, axis=-1))
    return 1e-6 * purse.radii + 8.0 * eps * mag * lscale


def classify(purse, R, t, precision):
    """+1 decided feasible, -1 decided infeasible, 0 ambiguous (within the band)."""
    m = op.margins(purse, R, t)
    b = constraint_bands(purse, R, t, precision)
    infeas = (m < -b).any(axis=-1)
    feas = (m > b).all(axis=-1)
    return np.where(infeas, -1, np.where(feas, 1, 0))


class ReplayReport:
    def __init__(self):
        self.inconsistent = []   # (walk, iteration, what)
        self.robust = None       # walks whose oracle free-run decisions are all outside the band
        self.robust_mismatch = []  # (walk, iteration): robust decision where the GPU trace differs

    def ok(self):
        return not self.inconsistent


def _check_topk(d, band_d, J, K):
    """GPU's ranked list J consistent with the oracle's distances d (within band)."""
    W = d.shape[0]
    bad = np.zeros(W, bool)
    rows = np.arange(W)[:, None]
    dj = d[rows, J]                                         # (W, K)
    bj = band_d[rows, J]
    # ranks descending (ties allowed inside the band)
    bad |= (dj[:, 1:] > dj[:, :-1] + bj[:, 1:] + bj[:, :-1]).any(axis=1)
    # everything left out is not above the last kept one (beyond the band)
    mask = np.ones_like(d, dtype=bool)
    mask[rows, J] = False
    last = dj[:, -1] + bj[:, -1]
    bad |= ((d - band_d > last[:, None]) & mask).any(axis=1)
    # distinct, in range
    bad |= np.array([len(set(r)) != K for r in J])
    return bad


def _check_ladder(cls, m0, k0):
    """cls (W, K, T) in {-1, 0, 1}; GPU chose (m0, k0) (-1 = none)."""
    W, K, T = cls.shape
    bad = np.zeros(W, bool)
    for w in range(W):
        c = cls[w]
        if m0[w] < 0:
            bad[w] = (c == 1).any()
            continue
        m, k = m0[w], k0[w]
        if m >= T or k >= K or k < 0:
            bad[w] = True
            continue
        if (c[:, :m] == 1).any():
            bad[w] = True
        if (c[:k, m] == 1).any():
            bad[w] = True
        if c[k, m] == -1:
            bad[w] = True
    return bad


def replay_walks(purse, seeds, prm, seed, walk_ids, trace, precision, sampler):
    """Follow the GPU trace with FP64 arithmetic; returns (R, t, report)."""
    walk_ids = np.asarray(walk_ids, dtype=np.int64)
    K, NT = prm.n_keep, prm.n_steps
    stats = closure.center_stats(purse, seeds, prm)
    R, t = closure.start_walks(seeds, walk_ids)
    if sampler == 0:
        vel = closure.init_angular_velocity(R, stats.Rbar, prm.omega0, seed, walk_ids)
    else:
        vel = closure.init_center_velocity(t, stats.tbar, prm.v0, stats.S, seed, walk_ids)
    rep = ReplayReport()
    robust = np.ones(len(walk_ids), bool)
    W = len(walk_ids)
    rows = np.arange(W)
    for i in range(prm.n_iter):
        if sampler == 0:
            c = closure.rotation_walk_candidates(purse, R, t, vel, i, walk_ids, seed, prm, stats)
            # the perturbed poses: (R*, t_j)
            pr, pt = np.broadcast_to(R[:, None], c.tc.shape[:2] + (3, 3)), c.tc
        else:
            c = closure.translation_walk_candidates(purse, R, t, vel, i, walk_ids, seed, prm, stats)
            pr, pt = c.Rc, np.broadcast_to(t[:, None], c.Rc.shape[:2] + (3,))
        band_d = constraint_bands(purse, pr, pt, precision).max(axis=-1)
        J = trace[:, i, :K].astype(np.int64)
        m0 = trace[:, i, K].astype(np.int64)
        k0 = trace[:, i, K + 1].astype(np.int64)
        bad_topk = _check_topk(c.d, band_d, np.clip(J, 0, prm.n_perturb - 1), K)
        bad_topk |= (J < 0).any(axis=1) | (J >= prm.n_perturb).any(axis=1)
        Jc = np.clip(J, 0, prm.n_perturb - 1)
        # ladder candidates of the GPU's ranked list
        if sampler == 0:
            Rk = np.broadcast_to(c.Rc[:, None], (W, K, NT, 3, 3))
            tk = np.broadcast_to(c.tc[rows[:, None], Jc][:, :, None], (W, K, NT, 3))
        else:
            Rk = np.broadcast_to(c.Rc[rows[:, None], Jc][:, :, None], (W, K, NT, 3, 3))
            tk = np.broadcast_to(c.tc[:, None], (W, K, NT, 3))
        cls = classify(purse, Rk, tk, precision)
        bad_ladder = _check_ladder(cls, m0, k0)
        for w in np.nonzero(bad_topk | bad_ladder)[0]:
            if bad_topk[w]:
                dj = c.d[w, Jc[w]]
                why = ("topk", [round(float(x), 6) for x in dj], float(band_d[w].max()),
                       [int(x) for x in c.J[w]], [int(x) for x in J[w]])
            else:
                mm = op.margins(purse, Rk[w], tk[w]).min(axis=-1)
                why = ("ladder", int(m0[w]), int(k0[w]), np.array2string(cls[w], max_line_width=200),
                       float(np.abs(mm[np.isfinite(mm)]).min()) if np.isfinite(mm).any() else None)
            rep.inconsistent.append((int(walk_ids[w]), i, why))
        # robustness of the oracle's own decisions (free-run protocol)
        Jo = c.J
        do = c.d[rows[:, None], Jo]
        bo = band_d[rows[:, None], Jo]
        gaps = do[:, :-1] - do[:, 1:]
        rest = c.d.copy()
        rest[rows[:, None], Jo] = -np.inf
        gap_last = do[:, -1] - rest.max(axis=1)
        robust &= (gaps > bo[:, :-1] + bo[:, 1:]).all(axis=1) & (gap_last > 2 * bo[:, -1])
        mo, ko = closure.find_farthest(c.I)
        if sampler == 0:
            Ro = np.broadcast_to(c.Rc[:, None], (W, K, NT, 3, 3))
            to = np.broadcast_to(c.tc[rows[:, None], Jo][:, :, None], (W, K, NT, 3))
        else:
            Ro = np.broadcast_to(c.Rc[rows[:, None], Jo][:, :, None], (W, K, NT, 3, 3))
            to = np.broadcast_to(c.tc[:, None], (W, K, NT, 3))
        clo = classify(purse, Ro, to, precision)
        decided = np.ones(W, bool)
        for w in range(W):
            # every candidate scanned up to and including the decision must be decided
            upto = NT if mo[w] < 0 else mo[w] + 1
            decided[w] = (clo[w, :, :upto] != 0).all()
        robust &= decided
        same = (J == Jo).all(axis=1) & (m0 == mo) & (k0 == ko)
        for w in np.nonzero(robust & ~same)[0]:
            rep.robust_mismatch.append((int(walk_ids[w]), i))
        # follow the GPU
        mv = m0 >= 0
        w_idx = rows[mv]
        R, t = R.copy(), t.copy()
        if sampler == 0:
            R[mv] = c.Rc[w_idx, m0[mv]]
            t[mv] = c.tc[w_idx, Jc[w_idx, k0[mv]]]
        else:
            R[mv] = c.Rc[w_idx, Jc[w_idx, k0[mv]]]
            t[mv] = c.tc[w_idx, m0[mv]]
    rep.robust = robust
    return R, t, rep


def free_run_trace(purse, seeds, prm, seed, walk_ids, sampler):
    """The oracle's own decisions: (W, N_I, K + 2) like the GPU trace."""
    walk_ids = np.asarray(walk_ids, dtype=np.int64)
    stats = closure.center_stats(purse, seeds, prm)
    R, t = closure.start_walks(seeds, walk_ids)
    if sampler == 0:
        vel = closure.init_angular_velocity(R, stats.Rbar, prm.omega0, seed, walk_ids)
    else:
        vel = closure.init_center_velocity(t, stats.tbar, prm.v0, stats.S, seed, walk_ids)
    K = prm.n_keep
    tr = np.zeros((len(walk_ids), prm.n_iter, K + 2), np.int64)
    for i in range(prm.n_iter):
        if sampler == 0:
            c = closure.rotation_walk_candidates(purse, R, t, vel, i, walk_ids, seed, prm, stats)
        else:
            c = closure.translation_walk_candidates(purse, R, t, vel, i, walk_ids, seed, prm, stats)
        m0, k0 = closure.find_farthest(c.I)
        tr[:, i, :K] = c.J
        tr[:, i, K] = m0
        tr[:, i, K + 1] = k0
        if sampler == 0:
            R, t = closure.apply_rotation_step(R, t, c, m0, k0)
        else:
            R, t = closure.apply_translation_step(R, t, c, m0, k0)
    return tr, R, t


def rot_angle(qa, qb):
    """Geodesic angle between unit quaternions (sign-invariant)."""
    qa = np.asarray(qa, np.float64)
    qb = np.asarray(qb, np.float64)
    qa = qa / np.linalg.norm(qa, axis=-1, keepdims=True)
    qb = qb / np.linalg.norm(qb, axis=-1, keepdims=True)
    s = np.where((qa * qb).sum(-1) < 0, -1.0, 1.0)
    # chord |qa - s qb| = 2 sin(phi / 2) with phi the angle of the 4-vectors; rotation angle = 2 phi
    chord = np.linalg.norm(qa - s[..., None] * qb, axis=-1)
    return 4.0 * np.arcsin(np.clip(chord / 2.0, 0.0, 1.0))


def lattice_points(seed, phase, j, i, w, unit=False):
    pts, used = philox.ball_points(seed, phase, j, i, w, unit=unit)
    return pts, used


def rot_keys(C, qs):
    d = so3_o.quat_mul(so3_o.quat_conj(C)[None], qs)
    return (d[:, 1:] ** 2).sum(1)


def check_rotation(q64, res, f, precision):
    """GGD protocol for the rotation ball: every farthest choice f_k of the GPU is within the
    rounding band of the FP64 maximum key from the replayed centre C_{k-1}; the replayed centre
    and its radius match the GPU's result.  Returns (C, D)."""
    K = len(f)
    qs = megb_o.canonical(q64)
    Cs = megb_o.megb_rotation_replay(qs, f)
    for k in range(1, K + 1):
        keys = rot_keys(Cs[k - 1], qs)
        band = 64 * EPS[precision] * (np.sqrt(keys.max()) + EPS[precision])
        assert keys[f[k - 1]] >= keys.max() - band, (k, keys[f[k - 1]], keys.max())
    C = Cs[-1]
    assert rot_angle(res[:4], C) <= 1e-9
    D = megb_o.rotation_distances(C, qs).max()
    assert abs(res[7] - D) <= 1e-5 * D + 1e-12, (res[7], D)
    return C, D


def check_translation(t64, res, f, precision):
    """The same protocol for the translation ball (Badoiu-Clarkson steps).  Returns (c, d)."""
    K = len(f)
    cs = megb_o.megb_translation_replay(t64, f)
    scale = np.abs(t64).max()
    for k in range(1, K + 1):
        keys = ((t64 - cs[k - 1]) ** 2).sum(1)
        band = 16 * EPS[precision] * scale * (np.sqrt(keys.max()) + EPS[precision] * scale)
        assert keys[f[k - 1]] >= keys.max() - band
    c = cs[-1]
    assert np.abs(res[4:7] - c).max() <= 1e-12 * (1 + scale)
    d = np.sqrt(((t64 - c) ** 2).sum(1)).max()
    assert abs(res[8] - d) <= 1e-5 * d + 1e-12
    return c, d
