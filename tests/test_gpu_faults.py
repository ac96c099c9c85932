"""Failure detection on the GPU without a GPU fault.

* ``stall``: after staging its constraint table (the bulk copy has landed), the walk kernel waits
  on a second mbarrier that nothing arrives at, with a poll limit of 2^10 tries; the wait runs
  out, the kernel flags a timeout in the handle's status word and returns.  purse_sync reports
  PURSE_ERR_TIMEOUT, the context stays usable, and the next call on the same handle gives the
  same samples as a call on a fresh handle.
* ``empty_seed`` / ``alloc`` / ``launch``: refused on the host in the middle of a pipeline; the
  handle keeps working once the fault is lifted, and a refused launch queues no work.
* megb_solve_noalloc allocates nothing, so PURSE_FAULT=alloc does not stop it.
"""
import numpy as np
import pytest
import torch

from oracle import closure
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn
from tests.gpu_helpers import params_from, to_dev

pytestmark = pytest.mark.gpu

TIMEOUT, EMPTY, CUDA, NOMEM = 4, 3, 2, 5


def _sample(h, prm, sampler, seeds, W, precision=0):
    dt = torch.float32 if precision == 0 else torch.float64
    q = torch.full((W, 4), np.nan, dtype=dt, device="cuda")
    t = torch.full((W, 3), np.nan, dtype=dt, device="cuda")
    P.purse_sample(h, params_from(prm, sampler, precision), 5, seeds, seeds.shape[0], W, q, t, None)
    return q, t


@pytest.mark.parametrize("kind,sampler", [(0, 0), (1, 1)])
def test_stalled_wait_reports_timeout_and_the_handle_recovers(monkeypatch, kind, sampler):
    p = syn.purse_3d3d(8, 0) if kind == 0 else syn.purse_2d3d(16, 0)
    prm = closure.preset_3d3d(n_iter=4) if kind == 0 else closure.preset_2d3d(n_iter=4)
    seeds = to_dev(p.seed_pose()[None])
    W = 3000
    with P.Purse(p) as ref:
        q0, t0 = _sample(ref.h, prm, sampler, seeds, W)
        P.purse_sync(ref.h)
    with P.Purse(p) as h:
        monkeypatch.setenv("PURSE_FAULT", "stall")
        _sample(h.h, prm, sampler, seeds, W)
        with pytest.raises(P.PurseError) as e:
            P.purse_sync(h.h)
        assert e.value.status == TIMEOUT
        assert "bounded device wait" in str(e.value)
        monkeypatch.delenv("PURSE_FAULT")
        P.purse_sync(h.h)  # the status word was cleared by the previous sync
        q1, t1 = _sample(h.h, prm, sampler, seeds, W)
        P.purse_sync(h.h)
    assert torch.equal(q0, q1) and torch.equal(t0, t1)
    assert torch.isfinite(q1).all() and torch.isfinite(t1).all()


def test_empty_seed_fault_and_recovery(monkeypatch):
    p = syn.purse_3d3d(8, 0)
    prm = closure.preset_3d3d(n_iter=2)
    seeds = torch.empty((16, 12), dtype=torch.float64, device="cuda")
    with P.Purse(p) as h:
        monkeypatch.setenv("PURSE_FAULT", "empty_seed")
        with pytest.raises(P.PurseError) as e:
            P.purse_ransag(h.h, 0, 20000, 16, seeds)
        assert e.value.status == EMPTY and "PURSE_FAULT=empty_seed" in str(e.value)
        one = to_dev(p.seed_pose()[None])
        with pytest.raises(P.PurseError) as e:
            _sample(h.h, prm, 0, one, 64)
        assert e.value.status == EMPTY
        monkeypatch.delenv("PURSE_FAULT")
        n = P.purse_ransag(h.h, 0, 20000, 16, seeds)
        assert n >= 1
        q, t = _sample(h.h, prm, 0, seeds[:n], 64)
        P.purse_sync(h.h)
        assert torch.isfinite(q).all() and torch.isfinite(t).all()


def test_alloc_and_launch_faults_mid_pipeline(monkeypatch):
    p = syn.purse_3d3d(8, 1)
    prm = closure.preset_3d3d(n_iter=2)
    seeds = to_dev(p.seed_pose()[None])
    W = 4096
    with P.Purse(p) as h:
        q, t = _sample(h.h, prm, 0, seeds, W)
        P.purse_sync(h.h)
        res = torch.full((9,), np.nan, dtype=torch.float64, device="cuda")
        # a refused launch queues nothing: the result buffer is untouched
        monkeypatch.setenv("PURSE_FAULT", "launch")
        with pytest.raises(P.PurseError) as e:
            P.megb_solve(h.h, 0, 100, q, W, t, W, res)
        assert e.value.status == CUDA
        torch.cuda.synchronize()
        assert torch.isnan(res).all()
        # a refused allocation: megb_solve with more iterations needs more scratch than the handle has
        monkeypatch.setenv("PURSE_FAULT", "alloc")
        with pytest.raises(P.PurseError) as e:
            P.megb_solve(h.h, 0, 200000, q, W, t, W, res)
        assert e.value.status == NOMEM
        # the allocation-free solver is not affected
        got = torch.full((9,), np.nan, dtype=torch.float64, device="cuda")
        P.megb_solve_noalloc(0, 100, q, W, t, W, got)
        monkeypatch.delenv("PURSE_FAULT")
        P.megb_solve(h.h, 0, 100, q, W, t, W, res)
        P.purse_sync(h.h)
        r, g = res.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(r)) and abs(g[7] - r[7]) <= 1e-5 * r[7] and abs(g[8] - r[8]) <= 1e-5 * r[8]
