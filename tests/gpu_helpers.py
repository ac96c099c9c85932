"""Calls through the C ABI for the GPU tests (device buffers from torch)."""
from __future__ import annotations

import numpy as np
import torch

from paper_2403_09990_gb300 import purse as P

DT = {0: torch.float32, 1: torch.float64}


def to_dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def params_from(prm, sampler, precision):
    """purse_params from an oracle.closure.Params."""
    return P.make_params(n_iter=prm.n_iter, n_perturb=prm.n_perturb, n_keep=prm.n_keep, n_steps=prm.n_steps,
                         omega0=prm.omega0, v0=prm.v0, gamma=prm.gamma, rot_perturb=prm.rot_perturb,
                         trans_perturb=prm.trans_perturb, perturb_units=prm.perturb_units, sampler=sampler,
                         precision=precision)


def sample(handle, prm, sampler, precision, seed, seeds_np, n_samples, trace=True, trace_rows=None):
    """Run purse_sample; returns (q, t, trace) as numpy arrays (trace only of trace_rows if given)."""
    seeds = to_dev(seeds_np.reshape(-1, 12))
    q = torch.empty((n_samples, 4), dtype=DT[precision], device="cuda")
    t = torch.empty((n_samples, 3), dtype=DT[precision], device="cuda")
    tr = torch.full((n_samples, prm.n_iter, prm.n_keep + 2), -7, dtype=torch.int16, device="cuda") if trace else None
    P.purse_sample(handle, params_from(prm, sampler, precision), seed, seeds, seeds.shape[0], n_samples, q, t, tr)
    P.purse_sync(handle)
    if trace and trace_rows is not None:
        tr = tr[torch.as_tensor(trace_rows, device="cuda")]
    return (q.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64),
            tr.cpu().numpy().astype(np.int64) if trace else None)


def megb(handle, precision, K, q_np, t_np):
    q = to_dev(q_np, DT[precision]) if q_np is not None else None
    t = to_dev(t_np, DT[precision]) if t_np is not None else None
    nq = 0 if q_np is None else q_np.shape[0]
    nt = 0 if t_np is None else t_np.shape[0]
    res = torch.full((9,), np.nan, dtype=torch.float64, device="cuda")
    far = torch.full((2 * K,), -1, dtype=torch.int32, device="cuda")
    P.megb_solve(handle, precision, K, q, nq, t, nt, res, far)
    P.purse_sync(handle)
    return res.cpu().numpy(), far.cpu().numpy().astype(np.int64)
