"""GPU RANSAG (Step I, 3D-3D) against the oracle: same accepted trials, same poses."""
import numpy as np
import pytest
import torch

from oracle import purse as op
from oracle import ransag
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


def test_ransag_rejects_2d3d():
    p = syn.purse_2d3d(16, 0)
    seeds = torch.empty((10, 12), dtype=torch.float64, device="cuda")
    with P.Purse(p) as h:
        with pytest.raises(P.PurseError) as e:
            P.purse_ransag(h.h, 0, 100, 10, seeds)
    assert e.value.status == 1
