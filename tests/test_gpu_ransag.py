"""GPU RANSAG (Step I) against the oracle: same accepted trials and candidates, same poses.

3D-3D (Arun/Horn fit) and 2D-3D (P3P).  For 2D-3D the comparison skips the trials whose
outcome is fragile in FP64 -- a quartic with a near-double root (two real roots, or a complex
pair, within 1e-6), or a candidate within 1e-9 r of the PURSE boundary -- since either side may
then legitimately decide otherwise; such trials are rare and counted, and every other accepted
seed (at least 90 % of them) is compared.  The
P3P poses agree to rounding in the bulk and to 1e-6 where the view is ill-conditioned."""
import numpy as np
import pytest
import torch

from oracle import purse as op
from oracle import p3p, ransag
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,max_seeds,trials", [(8, 256, 200000), (8, 5000, 70000), (50, 64, 300000), (3, 100, 5000)])
def test_ransag_matches_oracle(n, max_seeds, trials):
    p = syn.purse_3d3d(n, 4)
    seeds = torch.full((max_seeds, 12), np.nan, dtype=torch.float64, device="cuda")
    with P.Purse(p) as h:
        try:
            got = P.purse_ransag(h.h, 11, trials, max_seeds, seeds)
        except P.PurseError as e:
            assert e.status == 3
            got = 0
    ref, acc = ransag.ransag_3d3d(p, 11, trials, max_seeds)
    assert got == len(ref)
    g = seeds.cpu().numpy()[:got]
    if got:
        assert np.abs(g - ref).max() <= 1e-9
        assert np.all(op.in_purse(p, g[:, :9].reshape(-1, 3, 3), g[:, 9:]))


def test_ransag_empty_purse_reports_empty():
    p = syn.purse_3d3d(8, 0)
    rng = np.random.default_rng(0)
    bad = syn.Purse(0, p.model, rng.uniform(-5, 5, (8, 3)), np.full(8, 1e-4))
    seeds = torch.empty((10, 12), dtype=torch.float64, device="cuda")
    with P.Purse(bad) as h:
        with pytest.raises(P.PurseError) as e:
            P.purse_ransag(h.h, 0, 3000, 10, seeds)
    assert e.value.status == 3


def fragile_trials(p, seed, n_trials):
    """Trial indices whose P3P outcome is decided within FP64 rounding."""
    from numpy.polynomial import polynomial as npoly
    from oracle import philox
    tau = np.arange(n_trials)
    words = philox.stream_words(seed, philox.PHASE_RANSAG, 0, 0, tau, 3)
    idx = philox.distinct_triple(words, p.n)
    pts = np.stack([philox.disk_points(seed, philox.PHASE_RANSAG, c + 1, 0, tau)[0] for c in range(3)], axis=1)
    f = p3p.bearings(p.K, p.obs[idx] + p.radii[idx][..., None] * pts)
    out = []
    for k in range(n_trials):
        A = p3p.quartic(p.model[idx[k]], f[k])[0]
        r = npoly.polyroots(np.trim_zeros(A, 'b'))
        close = any(abs(r[i] - r[j]) < 1e-6 * max(1.0, abs(r[i])) for i in range(len(r)) for j in range(i))
        edge = any(abs(op.dist_to_boundary(p, R, t)) < 1e-9 * p.radii.min() for R, t in p3p.p3p(p.model[idx[k]], f[k]))
        if close or edge:
            out.append(k)
    return out


@pytest.mark.parametrize("n,max_seeds,trials", [(8, 64, 4000), (4, 3000, 2500), (6, 5000, 70000), (16, 4, 40000)])
def test_ransag_2d3d_matches_oracle(n, max_seeds, trials):
    p = syn.purse_2d3d(n, 4)
    seeds = torch.full((max_seeds, 12), np.nan, dtype=torch.float64, device="cuda")
    with P.Purse(p) as h:
        try:
            got = P.purse_ransag(h.h, 11, trials, max_seeds, seeds)
        except P.PurseError as e:
            assert e.status == 3
            got = 0
    ref, acc = p3p.ransag_2d3d(p, 11, trials, max_seeds)
    g = seeds.cpu().numpy()[:got]
    if got:
        assert np.all(op.in_purse(p, g[:, :9].reshape(-1, 3, 3), g[:, 9:]))
    last = int(acc[-1, 0]) + 1 if len(acc) and len(ref) == max_seeds else trials
    frag = fragile_trials(p, 11, last)
    if not frag:
        assert got == len(ref)
    pairs = align_seeds(g, ref, acc, frag)
    # every accepted seed of a trial decided outside the FP64 band is compared; the fragile
    # trials are rare, so at least 90 % of the oracle's seeds are
    robust = int(sum(1 for k in range(len(ref)) if acc[k, 0] not in set(frag)))
    assert len(pairs) >= min(robust, max(1, int(0.9 * len(ref)))) if len(ref) else len(pairs) == 0, \
        (len(pairs), robust, len(ref))
    d = np.zeros(0)
    if pairs:
        gi, ri = np.array(pairs).T
        # P3P loses digits near degenerate views (the pose moves like 1/A'(v) at a root v of the
        # quartic), so identical FP64 arithmetic on the two sides agrees to rounding in the bulk and
        # to 1e-6 at worst; a different candidate would differ by the noise radius scale (> 1e-3)
        d = np.abs(g[gi] - ref[ri]).max(axis=1)
        assert np.median(d) <= 1e-10 and d.max() <= 1e-6, (np.median(d), d.max())
    print(f"n {n}: {got} seeds from {trials} trials, {len(frag)} fragile trials, {len(pairs)} of "
          f"{len(ref)} seeds compared, max |pose difference| {d.max() if len(d) else 0:.2e}")


def align_seeds(g, ref, acc, frag):
    """(GPU index, oracle index) pairs of the seeds of the trials decided outside the FP64 band.

    Both sides list seeds in (trial, ascending root) order.  The oracle's seeds of fragile trials
    are skipped; on the GPU side up to four candidates per fragile trial passed since the last
    compared seed may be skipped (a fragile trial may yield other candidates there).  Any other
    difference in the sequence fails."""
    frag = np.asarray(sorted(frag), dtype=np.int64)
    fset = set(frag.tolist())
    pairs = []
    i, last_trial = 0, -1
    for j in range(len(ref)):
        tr = int(acc[j, 0])
        if tr in fset:
            continue
        if i >= len(g):
            break
        skips = 4 * int(((frag > last_trial) & (frag < tr)).sum())
        k = i
        while k < len(g) and k - i <= skips and np.abs(g[k] - ref[j]).max() > 1e-6:
            k += 1
        assert k < len(g) and k - i <= skips, f"GPU seed sequence differs at oracle seed {j} (trial {tr})"
        pairs.append((k, j))
        i, last_trial = k + 1, tr
    return pairs
