"""Pins of the oracle's P3P solver and RANSAG for 2D-3D (CPU only).

The solver is checked against things it does not compute itself: poses projected
exactly must come back, every candidate must satisfy the three law-of-cosines
equations it eliminates, and the candidate set must equal the positive solutions
that a multistart Newton search finds on the original three equations."""
import numpy as np

from oracle import p3p, philox, so3
from oracle import purse as op
from paper_2403_09990_gb300 import synthetic as syn

rng = np.random.default_rng(31)


def random_view():
    """A pose with three world points 0.5..3 m in front of the camera and their bearings."""
    R = so3.exp_so3(rng.normal(size=3) * 2)
    t = np.array([0.0, 0.0, 2.0]) + rng.normal(size=3) * 0.3
    Xc = rng.normal(size=(3, 3)) * 0.4 + np.array([0.0, 0.0, 2.0])     # camera frame
    P = (Xc - t) @ R                                                      # world: R^T (Xc - t)
    f = Xc / np.linalg.norm(Xc, axis=1, keepdims=True)
    return R, t, P, f


def law_of_cosines_residual(P, f, s):
    s1, s2, s3 = s
    a = np.linalg.norm(P[1] - P[2])
    b = np.linalg.norm(P[0] - P[2])
    c = np.linalg.norm(P[0] - P[1])
    ca, cb, cg = f[1] @ f[2], f[0] @ f[2], f[0] @ f[1]
    return np.array([s2 * s2 + s3 * s3 - 2 * s2 * s3 * ca - a * a,
                     s1 * s1 + s3 * s3 - 2 * s1 * s3 * cb - b * b,
                     s1 * s1 + s2 * s2 - 2 * s1 * s2 * cg - c * c])


def multistart_depths(P, f, n=12):
    """Positive solutions of the three equations by Newton from an n^3 grid of starts."""
    scale = 3 * max(np.linalg.norm(P[i] - P[j]) for i in range(3) for j in range(3)) + 4.0
    g = np.linspace(0.05, scale, n)
    S = np.stack(np.meshgrid(g, g, g, indexing='ij'), -1).reshape(-1, 3)
    a2 = np.linalg.norm(P[1] - P[2]) ** 2
    b2 = np.linalg.norm(P[0] - P[2]) ** 2
    c2 = np.linalg.norm(P[0] - P[1]) ** 2
    ca, cb, cg = f[1] @ f[2], f[0] @ f[2], f[0] @ f[1]
    for _ in range(60):
        s1, s2, s3 = S.T
        F = np.stack([s2 * s2 + s3 * s3 - 2 * s2 * s3 * ca - a2,
                      s1 * s1 + s3 * s3 - 2 * s1 * s3 * cb - b2,
                      s1 * s1 + s2 * s2 - 2 * s1 * s2 * cg - c2], -1)
        J = np.zeros((len(S), 3, 3))
        J[:, 0, 1], J[:, 0, 2] = 2 * s2 - 2 * s3 * ca, 2 * s3 - 2 * s2 * ca
        J[:, 1, 0], J[:, 1, 2] = 2 * s1 - 2 * s3 * cb, 2 * s3 - 2 * s1 * cb
        J[:, 2, 0], J[:, 2, 1] = 2 * s1 - 2 * s2 * cg, 2 * s2 - 2 * s1 * cg
        ok = np.abs(np.linalg.det(J)) > 1e-14
        S[ok] = S[ok] - np.linalg.solve(J[ok], F[ok][..., None])[..., 0]
    res = np.abs(np.stack([law_of_cosines_residual(P, f, s) for s in S])).max(axis=1)
    good = S[(res < 1e-10) & (S > 1e-9).all(axis=1)]
    sols = []
    for s in good:
        if all(np.abs(s - q).max() > 1e-6 for q in sols):
            sols.append(s)
    return sorted(sols, key=lambda s: s[2] / s[0])


def depths_of(P, R, t, f):
    X = P @ R.T + t
    return np.einsum('ij,ij->i', X, f), X


def test_noise_free_pose_is_among_the_candidates():
    # near a double root of the quartic the problem itself loses half the digits, so the
    # bound is on the median and on the worst of 200 random views
    errs = []
    for _ in range(200):
        R, t, P, f = random_view()
        cands = p3p.p3p(P, f)
        assert 1 <= len(cands) <= 4
        errs.append(min(np.abs(Rc - R).max() + np.abs(tc - t).max() for Rc, tc in cands))
    assert np.median(errs) < 1e-11 and max(errs) < 1e-6, (np.median(errs), max(errs))


def test_every_candidate_reprojects_and_solves_the_eliminated_equations():
    for _ in range(40):
        _, _, P, f = random_view()
        for R, t in p3p.p3p(P, f):
            s, X = depths_of(P, R, t, f)
            assert np.all(s > 0)
            assert np.abs(X - s[:, None] * f).max() < 1e-9          # on the viewing rays
            assert np.abs(law_of_cosines_residual(P, f, s)).max() < 1e-9
            assert abs(np.linalg.det(R) - 1) < 1e-12


def test_candidate_set_equals_the_multistart_solutions():
    counts = []
    for _ in range(25):
        _, _, P, f = random_view()
        got = [depths_of(P, R, t, f)[0] for R, t in p3p.p3p(P, f)]
        ref = multistart_depths(P, f)
        assert len(got) == len(ref), (len(got), len(ref))
        for s in ref:
            assert min(np.abs(g - s).max() for g in got) < 1e-7
        counts.append(len(got))
    assert max(counts) >= 2


def test_four_solution_views():
    # generic views with four positive solutions (found by the multistart search on the
    # original equations) give four candidates with the same depths
    g = np.random.default_rng(5)
    found = 0
    for _ in range(300):
        X = g.normal(size=(3, 3)) * 0.4 + np.array([0.0, 0.0, 2.0])
        f = X / np.linalg.norm(X, axis=1, keepdims=True)
        ref = multistart_depths(X, f, n=10)
        if len(ref) != 4:
            continue
        got = [depths_of(X, R, t, f)[0] for R, t in p3p.p3p(X, f)]
        assert len(got) == 4
        for s in ref:
            assert min(np.abs(q - s).max() for q in got) < 1e-7
        found += 1
        if found == 3:
            break
    assert found == 3


def test_disk_points_are_uniform_in_the_unit_disk():
    pts, used = philox.disk_points(0, philox.PHASE_RANSAG, 1, 0, np.arange(40000))
    r2 = (pts ** 2).sum(-1)
    assert r2.max() <= 1.0
    assert abs(r2.mean() - 0.5) < 0.01                      # E|x|^2 = 1/2 for the uniform disk
    assert abs((used == 1).mean() - np.pi / 4) < 0.01       # lattice acceptance ~ pi / 4
    q = (pts[:, 0] > 0).astype(int) + 2 * (pts[:, 1] > 0)
    assert np.all(np.abs(np.bincount(q, minlength=4) / len(q) - 0.25) < 0.01)


def test_ransag_2d3d_seeds_are_in_the_purse():
    p = syn.purse_2d3d(8, 0)
    seeds, acc = p3p.ransag_2d3d(p, 0, 3000, 64)
    assert len(seeds) > 0
    assert np.all(np.diff(acc[:, 0]) >= 0)
    R = seeds[:, :9].reshape(-1, 3, 3)
    assert np.allclose(R @ np.swapaxes(R, 1, 2), np.eye(3), atol=1e-12)
    assert np.all(op.in_purse(p, R, seeds[:, 9:]))
    # the accepted poses cluster around the ground truth
    ang = np.array([so3.dist_so3(p.R_gt, r) for r in R])
    assert np.median(ang) < 0.2
