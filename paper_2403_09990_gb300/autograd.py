"""torch.autograd.Function over the C ABI: the enclosing balls of a PURSE as a
differentiable function of its observations y_i and radii r_i.

Forward: purse_create from the given arrays, purse_sample with boundary snap
(dS_R walks for the rotation ball; the translation ball takes the
translations of the sampler ``tr_sampler``: 0 reuses the dS_R walks, 1 runs
the dS_t walks of Alg. 5), megb_solve.  Backward: megb_backward.  This
module only marshals arguments; every step runs in the CUDA library.

The seed poses are constants of the function (pass fixed poses, e.g. a
ground-truth or externally estimated pose): with seeds drawn from y (RANSAG)
the walks would start at poses that move with y, which the snap does not
differentiate.  With ``tr_sampler = 0`` the translation samples do not move
along a rotation ray, so d-hat has zero gradient.
"""
from __future__ import annotations

import numpy as np
import torch

from . import purse as P


class _Handle:
    """Owns a PURSE handle until the autograd graph that saved it is freed."""

    def __init__(self, kind, model, obs, radii, K):
        self.h = P.purse_create(kind, model, obs, radii, K)

    def __del__(self):
        if getattr(self, "h", None):
            try:
                P.purse_destroy(self.h)
            except Exception:
                pass
            self.h = None


def _with(p, sampler, precision):
    q = P.purse_params.from_buffer_copy(p)
    q.sampler, q.precision = sampler, precision
    return q


class ClosureBalls(torch.autograd.Function):
    """result (9 doubles, cuda) = (C quaternion (w >= 0), c, D-hat, d-hat)."""

    @staticmethod
    def forward(ctx, obs, radii, model, kind, intrinsics, p_rot, p_tr, tr_sampler, seed, seeds, n_samples, n_iters,
                precision):
        dev = torch.device("cuda", torch.cuda.current_device())
        dt = torch.float32 if precision == 0 else torch.float64
        model = model.detach().cpu().numpy() if torch.is_tensor(model) else np.asarray(model)
        h = _Handle(int(kind), model, obs.detach().cpu().numpy(), radii.detach().cpu().numpy(), intrinsics)
        p_rot = _with(p_rot, 0, precision)
        p_tr = _with(p_tr, 1, precision)
        seeds_d = torch.as_tensor(np.ascontiguousarray(seeds, dtype=np.float64).reshape(-1, 12), device=dev)
        s0 = seeds_d.shape[0]
        qR = torch.empty((n_samples, 4), dtype=dt, device=dev)
        tR = torch.empty((n_samples, 3), dtype=dt, device=dev)
        snR = torch.empty((n_samples, 12), dtype=dt, device=dev)
        P.purse_sample(h.h, p_rot, seed, seeds_d, s0, n_samples, qR, tR, None, snap=snR)
        if tr_sampler == 1:
            qT = torch.empty((n_samples, 4), dtype=dt, device=dev)
            tT = torch.empty((n_samples, 3), dtype=dt, device=dev)
            snT = torch.empty((n_samples, 12), dtype=dt, device=dev)
            P.purse_sample(h.h, p_tr, seed, seeds_d, s0, n_samples, qT, tT, None, snap=snT)
        else:
            tT, snT = tR, snR
        res = torch.empty(9, dtype=torch.float64, device=dev)
        far = torch.empty(2 * n_iters, dtype=torch.int32, device=dev)
        P.megb_solve(h.h, precision, n_iters, qR, n_samples, tT, n_samples, res, far)
        ctx.state = (h, precision, n_iters, qR, snR, tT, snT, far, res, n_samples, obs.shape, obs.dtype, obs.device)
        return res.clone()

    @staticmethod
    def backward(ctx, g):
        h, precision, n_iters, qR, snR, tT, snT, far, res, n, oshape, odt, odev = ctx.state
        g = g.detach().to(device=res.device, dtype=torch.float64).contiguous()
        gy = torch.empty(oshape, dtype=torch.float64, device=res.device)
        gr = torch.empty(oshape[0], dtype=torch.float64, device=res.device)
        P.megb_backward(h.h, precision, n_iters, qR, snR, n, tT, snT, n, far, res, g, gy, gr)
        P.purse_sync(h.h)
        return (gy.to(device=odev, dtype=odt), gr.to(device=odev, dtype=odt)) + (None,) * 11


def closure_balls(obs, radii, model, kind, intrinsics, p_rot, p_tr, seeds, n_samples, n_iters, seed=0,
                  tr_sampler=1, precision=0):
    """(C, c, D, d) of the PURSE (y = obs, r = radii); differentiable in obs and radii."""
    r = ClosureBalls.apply(obs, radii, model, kind, intrinsics, p_rot, p_tr, tr_sampler, seed, seeds, n_samples,
                           n_iters, precision)
    return r[:4], r[4:7], r[7], r[8]
