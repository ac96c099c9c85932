"""Step III in FP64 (oracle side): minimum enclosing geodesic balls of samples.

* megb_rotation: geodesic gradient descent on SO(3) (Section II, "Geodesic
  Gradient Descent"; step rule of Alg. 6): start at the first sample, at
  iteration k = 1..K take the sample farthest from the current centre (the
  maximiser that generates the subdifferential, Theorem 5) and move to
  SLERP(C_{k-1}, R_hat, 1/k).  The radius is the largest geodesic distance
  from the final centre to any sample.  Rotations are unit quaternions with
  w >= 0; distances are 2 atan2(|vec(c* q)|, |c . q|), the geodesic distance
  of Section II.
* megb_translation: the Euclidean version (Badoiu-Clarkson,
  c_k = c_{k-1} + (t_far - c_{k-1}) / k).
* megb_rotation_mean / megb_translation_mean: the same descents with the output
  rule of Alg. 6 (the appendix's SDP-based descent): the centre is the
  projection onto SO(3) of the sum of the last iterates (ten in the paper),
  the translation centre the mean of the last iterates.
* welzl_meb / meb_bruteforce: exact minimum enclosing ball in R^d.
* meb_exact_translation / meb_exact_rotation: Step III as the paper states it
  (Section IV, Step III): the exact minimum enclosing ball of the translation
  samples in R^3, and of the rotation samples embedded as unit quaternions in
  R^4 (signs aligned to a reference rotation, the quaternion of each rotation
  on the reference's side), its centre projected back to the unit sphere and
  the radius taken as the largest geodesic distance from that centre.
Ties in the farthest point go to the lowest sample index.

Parity: pinned in tests/test_oracle_megb.py (rectangle corners, points on one
geodesic, Badoiu-Clarkson bound against the exact ball, octahedral
configurations with a known centre, containment and diameter bounds).
"""
from __future__ import annotations

import itertools

import numpy as np

from .so3 import R_from_quat, dist_quat, proj_so3, quat_from_R, slerp


def canonical(q):
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    return q * np.where(q[..., :1] < 0, -1.0, 1.0)


def rotation_distances(C, qs):
    return dist_quat(np.asarray(C)[None, :], qs)


def megb_rotation(qs, K: int):
    """(centre quaternion, radius D-hat, farthest-sample sequence f_1..f_K)."""
    qs = canonical(qs)
    C = qs[0].copy()
    f = np.empty(K, dtype=np.int64)
    for k in range(1, K + 1):
        fk = int(np.argmax(rotation_distances(C, qs)))
        f[k - 1] = fk
        C = slerp(C, qs[fk], 1.0 / k)
    D = float(rotation_distances(C, qs).max())
    return C, D, f


def megb_rotation_replay(qs, f):
    """Centres C_0..C_K when the farthest samples are the given sequence f."""
    qs = canonical(qs)
    Cs = [qs[0].copy()]
    for k, fk in enumerate(f, start=1):
        Cs.append(slerp(Cs[-1], qs[int(fk)], 1.0 / k))
    return np.array(Cs)


def megb_translation(ts, K: int):
    """(centre, radius d-hat, farthest-sample sequence f_1..f_K)."""
    ts = np.asarray(ts, dtype=np.float64)
    c = ts[0].copy()
    f = np.empty(K, dtype=np.int64)
    for k in range(1, K + 1):
        fk = int(np.argmax(((ts - c) ** 2).sum(axis=1)))
        f[k - 1] = fk
        c = c + (ts[fk] - c) / k
    d = float(np.sqrt(((ts - c) ** 2).sum(axis=1)).max())
    return c, d, f


def megb_rotation_mean(qs, K: int, n_last: int, f=None):
    """GGD on SO(3) with the output rule of Alg. 6: K iterations as in megb_rotation, then the
    centre R* = proj_SO3(sum of the rotation matrices of the last n_last iterates
    C_{K-n_last+1} .. C_K; fewer when K + 1 < n_last, C_0 included), and D-hat the largest geodesic
    distance from R*.  Returns (R* as a quaternion with w >= 0, D-hat, farthest sequence).
    f: a farthest sequence to replay instead of the free run's (tests replay the GPU's)."""
    if f is None:
        _, _, f = megb_rotation(qs, K)
    Cs = megb_rotation_replay(qs, f)
    M = sum(R_from_quat(c) for c in Cs[max(0, K - n_last + 1):])
    C = canonical(quat_from_R(proj_so3(M)))
    D = float(rotation_distances(C, canonical(qs)).max())
    return C, D, f


def megb_translation_mean(ts, K: int, n_last: int, f=None):
    """Badoiu-Clarkson with the same output rule in R^3 (projection = identity): the mean of the
    last n_last centres c_{K-n_last+1} .. c_K (c_0 included when K + 1 < n_last), and d-hat the
    largest distance from it.  Returns (centre, d-hat, farthest sequence); f as in megb_rotation_mean."""
    if f is None:
        _, _, f = megb_translation(ts, K)
    cs = megb_translation_replay(ts, f)
    c = cs[max(0, K - n_last + 1):].mean(axis=0)
    ts = np.asarray(ts, dtype=np.float64)
    return c, float(np.sqrt(((ts - c) ** 2).sum(axis=1)).max()), f


def megb_translation_replay(ts, f):
    ts = np.asarray(ts, dtype=np.float64)
    cs = [ts[0].copy()]
    for k, fk in enumerate(f, start=1):
        cs.append(cs[-1] + (ts[int(fk)] - cs[-1]) / k)
    return np.array(cs)


def _circumball(P):
    """Smallest ball with every row of P on its boundary (centre in their affine hull)."""
    p0 = P[0]
    if P.shape[0] == 1:
        return p0.copy(), 0.0
    D = P[1:] - p0
    G = 2.0 * D @ D.T
    rhs = (D * D).sum(axis=1)
    lam = np.linalg.lstsq(G, rhs, rcond=None)[0]
    c = p0 + lam @ D
    return c, float(np.linalg.norm(P - c, axis=1).max())


def meb_bruteforce(P, tol=1e-12):
    """Exact minimum enclosing ball by trying every support set of size <= d + 1."""
    P = np.asarray(P, dtype=np.float64)
    n, dim = P.shape
    best = None
    for s in range(1, min(n, dim + 1) + 1):
        for sub in itertools.combinations(range(n), s):
            c, r = _circumball(P[list(sub)])
            if np.all(np.linalg.norm(P - c, axis=1) <= r * (1 + tol) + tol):
                if best is None or r < best[1]:
                    best = (c, r)
    return best


def welzl_meb(P):
    """Exact minimum enclosing ball (Welzl's recursion, iterative move-to-front form)."""
    P = np.asarray(P, dtype=np.float64)
    dim = P.shape[1]

    def ball(R):
        if not R:
            return np.zeros(dim), -1.0
        return _circumball(P[R])

    def inside(c, r, p):
        return r >= 0 and np.linalg.norm(P[p] - c) <= r * (1 + 1e-12) + 1e-15

    def mtf(idx, R):
        c, r = ball(R)
        if len(R) == dim + 1:
            return c, r
        for k in range(len(idx)):
            p = idx[k]
            if not inside(c, r, p):
                c, r = mtf(idx[:k], R + [p])
        return c, r

    order = list(np.random.default_rng(0).permutation(P.shape[0]))
    return mtf(order, [])


def meb_exact_translation(ts):
    """(centre, radius) of the exact minimum enclosing ball of the translations in R^3."""
    ts = np.asarray(ts, dtype=np.float64)
    c, _ = welzl_meb(ts)
    return c, float(np.linalg.norm(ts - c, axis=1).max())


def meb_exact_rotation(qs, ref):
    """(centre quaternion with w >= 0, geodesic radius) from the exact minimum enclosing ball of the
    unit quaternions in R^4, each taken with the sign that puts it on the side of ``ref``."""
    qs = np.asarray(qs, dtype=np.float64)
    s = np.where(qs @ np.asarray(ref, dtype=np.float64) < 0, -1.0, 1.0)
    c4, _ = welzl_meb(qs * s[:, None])
    C = canonical(c4)
    return C, float(rotation_distances(C, qs).max())
