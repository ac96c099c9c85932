"""Step I of CLOSURE for 2D-3D in FP64 (oracle side): RANSAG with a P3P minimal solver.

Section IV, Step I (Example 1): each trial picks three distinct constraints,
takes one pixel inside each of their noise disks, solves the perspective-
three-point problem for the candidate poses, and keeps every candidate that
satisfies all constraints of eq. (2)/(5).  S0 is the accepted poses in trial
order (candidates of one trial in ascending order of the quartic root v
below), at most ``max_seeds`` of them.

P3P: the paper calls Gao et al.'s solver; every exact P3P solver returns the
same set of (up to four) poses, and this oracle uses Grunert's elimination as
reviewed by Haralick, Lee, Ottenberg and Nolle (IJCV 1994).  With unit
bearings f_i of the three pixels, world points P_i and camera-frame points
s_i f_i (s_i > 0), the law of cosines on the sides a = |P_2 - P_3|,
b = |P_1 - P_3|, c = |P_1 - P_2| with cos(alpha) = f_2.f_3,
cos(beta) = f_1.f_3, cos(gamma) = f_1.f_2 gives
    s_2^2 + s_3^2 - 2 s_2 s_3 cos(alpha) = a^2
    s_1^2 + s_3^2 - 2 s_1 s_3 cos(beta)  = b^2
    s_1^2 + s_2^2 - 2 s_1 s_2 cos(gamma) = c^2.
With s_2 = u s_1, s_3 = v s_1 and Q(v) = 1 + v^2 - 2 v cos(beta), dividing the
first and third equations by the second and subtracting them gives u = N(v)/D(v),
    N(v) = k Q(v) + v^2 - 1,  k = (c^2 - a^2) / b^2,  D(v) = 2 (v cos(alpha) - cos(gamma)),
and the third divided by the second becomes the quartic
    N(v)^2 - 2 cos(gamma) N(v) D(v) + (1 - (c^2 / b^2) Q(v)) D(v)^2 = 0.
Each real root v gives s_1 = b / sqrt(Q(v)) and s_3 = v s_1; u solves the
third equation over the second, u^2 - 2 cos(gamma) u + 1 - (c^2 / b^2) Q(v) = 0,
and of its two roots the ones that also satisfy the first equation over the
second (relative residual below 1e-8) are kept (one where D(v) != 0, where it
equals N(v) / D(v); possibly both where D(v) = 0).  s_2 = u s_1, and the pose
maps P_i onto s_i f_i (Arun's fit on three exact correspondences).
Roots: numpy's companion-matrix eigenvalues, the real ones (|imag| below
1e-7 of max(1, |v|)) polished by two Newton steps.

Random draws: trial tau uses the Philox streams (phase 5, j, 0, tau); j = 0
gives the index triple, j = 1..3 the disk points (oracle.philox.disk_points).

Parity: pinned in tests/test_oracle_p3p.py (exact recovery of noise-free
poses among the candidates, every candidate reprojecting onto its bearings
and preserving the triangle, the four-solution count on a configuration
that has four, every accepted seed inside the PURSE).

Test infrastructure: imported by tests/, __graft_entry__.smoke() and the
bench's CPU baseline only.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import polynomial as npoly

from . import philox
from .purse import in_purse
from .ransag import arun

IMAG_TOL = 1e-7


def bearings(K, z):
    """Unit viewing rays K^-1 (u, v, 1) of pixels z (..., 2)."""
    fx, fy, cx, cy = K
    z = np.asarray(z, dtype=np.float64)
    r = np.stack([(z[..., 0] - cx) / fx, (z[..., 1] - cy) / fy, np.ones(z.shape[:-1])], axis=-1)
    return r / np.linalg.norm(r, axis=-1, keepdims=True)


def quartic(P, f):
    """Coefficients (increasing powers of v) of Grunert's quartic and the pieces N, D, Q, b."""
    P = np.asarray(P, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    a = np.linalg.norm(P[1] - P[2])
    b = np.linalg.norm(P[0] - P[2])
    c = np.linalg.norm(P[0] - P[1])
    ca, cb, cg = f[1] @ f[2], f[0] @ f[2], f[0] @ f[1]
    k = (c * c - a * a) / (b * b)
    Q = np.array([1.0, -2.0 * cb, 1.0])
    N = k * Q + np.array([-1.0, 0.0, 1.0])
    D = np.array([-2.0 * cg, 2.0 * ca])
    rest = npoly.polysub([1.0], (c * c) / (b * b) * Q)
    A = npoly.polyadd(npoly.polysub(npoly.polymul(N, N), 2.0 * cg * npoly.polymul(N, D)),
                      npoly.polymul(rest, npoly.polymul(D, D)))
    return A, N, D, Q, b


def real_roots(A):
    """Real roots of the polynomial A (increasing powers), ascending, Newton-polished."""
    A = np.trim_zeros(np.asarray(A, dtype=np.float64), 'b')
    if len(A) < 2:
        return np.zeros(0)
    r = npoly.polyroots(A)
    v = np.sort(r[np.abs(r.imag) <= IMAG_TOL * np.maximum(1.0, np.abs(r))].real)
    dA = npoly.polyder(A)
    for _ in range(2):
        d = npoly.polyval(v, dA)
        step = np.where(d != 0, npoly.polyval(v, A) / np.where(d != 0, d, 1.0), 0.0)
        v = v - step
    return v


def p3p(P, f):
    """Candidate poses (R, t) with s_i f_i = R P_i + t, s_i > 0: a list of up to four."""
    P = np.asarray(P, dtype=np.float64)
    A, N, D, Q, b = quartic(P, f)
    out = []
    f = np.asarray(f, dtype=np.float64)
    a2 = np.sum((P[1] - P[2]) ** 2)
    c2 = np.sum((P[0] - P[1]) ** 2)
    ca, cg = f[1] @ f[2], f[0] @ f[1]
    for v in real_roots(A):
        Qv = npoly.polyval(v, Q)
        if not Qv > 0:
            continue
        # u from the third equation over the second (a quadratic), kept where the first one
        # holds too; this also covers D(v) = 0, where u = N(v) / D(v) is undefined
        disc = cg * cg - 1.0 + (c2 / (b * b)) * Qv
        if disc < -1e-12:
            continue
        r = np.sqrt(max(disc, 0.0))
        for u in ((cg - r, cg + r) if r > 0 else (cg,)):
            if abs(u * u + v * v - 2.0 * u * v * ca - (a2 / (b * b)) * Qv) > 1e-8 * (1.0 + u * u + v * v):
                continue
            s1 = b / np.sqrt(Qv)
            s = np.array([s1, u * s1, v * s1])
            if not np.all(s > 0):
                continue
            R, t = arun(P, s[:, None] * f)
            out.append((R, t))
    return out


def ransag_trial_candidates(purse, seed: int, trials):
    """For every trial index in ``trials``: the list of (R, t, accepted) of its P3P candidates,
    in solver order."""
    tau = np.asarray(trials, dtype=np.int64)
    words = philox.stream_words(seed, philox.PHASE_RANSAG, 0, 0, tau, 3)
    idx = philox.distinct_triple(words, purse.n)                                       # (T, 3)
    pts = np.stack([philox.disk_points(seed, philox.PHASE_RANSAG, c + 1, 0, tau)[0]
                    for c in range(3)], axis=1)                                         # (T, 3, 2)
    lam = getattr(purse, "lam", None)
    if lam is not None:  # a point of the noise ellipse {e : e^T Lambda e <= r^2}: e = r U^-1 u
        U = np.swapaxes(np.linalg.cholesky(lam[idx]), -1, -2)
        pts = np.linalg.solve(U, pts[..., None])[..., 0]
    z = purse.obs[idx] + purse.radii[idx][..., None] * pts
    f = bearings(purse.K, z)
    out = []
    for n in range(len(tau)):
        out.append([(R, t, bool(in_purse(purse, R, t))) for R, t in p3p(purse.model[idx[n]], f[n])])
    return out


def ransag_2d3d(purse, seed: int, n_trials: int, max_seeds: int, chunk: int = 1 << 12):
    """S0 as an (n, 12) array (R row-major, t) and (trial, candidate) of each accepted seed."""
    seeds, acc = [], []
    for start in range(0, n_trials, chunk):
        tau = np.arange(start, min(n_trials, start + chunk))
        for n, cands in enumerate(ransag_trial_candidates(purse, seed, tau)):
            for k, (R, t, ok) in enumerate(cands):
                if ok and len(seeds) < max_seeds:
                    seeds.append(np.concatenate([R.reshape(9), t]))
                    acc.append((int(tau[n]), k))
        if len(seeds) == max_seeds:
            break
    return np.array(seeds).reshape(-1, 12), np.array(acc, dtype=np.int64).reshape(-1, 2)
