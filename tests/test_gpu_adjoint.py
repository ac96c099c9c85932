"""Parity of the boundary snap and of megb_backward (through the C ABI and the
torch.autograd.Function) with the FP64 oracle: snapped samples, snap
records, farthest sequences, balls and the gradients of the balls with
respect to the observations y_i and radii r_i; and against central finite
differences (h = 1e-6) of the oracle pipeline with the walks re-run."""
import numpy as np
import pytest
import torch

from oracle import adjoint, closure, snap
from oracle import purse as op
from oracle import megb as megb_o
from oracle.megb import canonical, megb_rotation, megb_translation
from oracle.so3 import quat_from_R
from paper_2403_09990_gb300 import autograd as AG
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn
from tests import parity
from tests.gpu_helpers import DT, params_from, to_dev

G_RES = np.array([0.2, -0.4, 0.1, 0.3, 0.5, -0.2, 0.7, 1.0, 1.0])


def case(kind, n=None, lam=False):
    if kind == 0:
        p = syn.purse_3d3d_ellipsoidal(n or 8, 3) if lam else syn.purse_3d3d(n or 8, 3)
        pr = closure.preset_3d3d(n_iter=3, rot_perturb=0.002, trans_perturb=0.002, perturb_units=1)
        pt = closure.preset_3d3d(n_iter=3, v0=0.02, rot_perturb=0.002, trans_perturb=0.002, perturb_units=1)
    else:
        p = syn.purse_2d3d_ellipsoidal(n or 10, 3) if lam else syn.purse_2d3d(n or 10, 3)
        pr = closure.preset_2d3d(n_iter=3, rot_perturb=0.002, trans_perturb=0.002, perturb_units=1)
        pt = pr
    return p, p.seed_pose()[None], pr, pt


def gpu_pipeline(p, seeds, pr, pt, seed, W, K, precision, g_res=G_RES):
    """purse_sample (snap) x 2 -> megb_solve -> megb_backward through the C ABI; numpy results."""
    dt = DT[precision]
    with P.Purse(p) as h:
        sd = to_dev(seeds.reshape(-1, 12))
        out = {}
        traces = {}
        for key, sampler, prm in (("rot", 0, pr), ("tr", 1, pt)):
            q = torch.empty((W, 4), dtype=dt, device="cuda")
            t = torch.empty((W, 3), dtype=dt, device="cuda")
            sn = torch.full((W, 12), np.nan, dtype=dt, device="cuda")
            tr = torch.full((W, prm.n_iter, prm.n_keep + 2), -7, dtype=torch.int16, device="cuda")
            P.purse_sample(h.h, params_from(prm, sampler, precision), seed, sd, sd.shape[0], W, q, t, tr, snap=sn)
            out[key] = (q, t, sn)
            traces[key] = tr
        res = torch.empty(9, dtype=torch.float64, device="cuda")
        far = torch.empty(2 * K, dtype=torch.int32, device="cuda")
        qR, _, snR = out["rot"]
        _, tT, snT = out["tr"]
        P.megb_solve(h.h, precision, K, qR, W, tT, W, res, far)
        gy = torch.full(p.obs.shape, np.nan, dtype=torch.float64, device="cuda")
        gr = torch.full((p.radii.shape[0],), np.nan, dtype=torch.float64, device="cuda")
        P.megb_backward(h.h, precision, K, qR, snR, W, tT, snT, W, far, res, to_dev(g_res), gy, gr)
        P.purse_sync(h.h)
        cpu = lambda x: x.cpu().numpy().astype(np.float64)
        return dict(qR=cpu(qR), snR=cpu(snR), tT=cpu(tT), qT=cpu(out["tr"][0]), snT=cpu(snT), res=cpu(res),
                    far=far.cpu().numpy().astype(np.int64), gy=cpu(gy), gr=cpu(gr),
                    trace_rot=traces["rot"].cpu().numpy().astype(np.int64),
                    trace_tr=traces["tr"].cpu().numpy().astype(np.int64))


def snap_ambiguous(p, R, t, d, ladder, rotation, precision):
    """Decisions of the snap taken inside the rounding band of the walk precision, per walk:
    (ladder, tie).  ladder: a ladder point scanned before (or at) tau_hi whose membership is
    undecided, so tau_hi, and with it the crossing the bisection finds, may differ; tie: the
    active constraint j* is within the band of the next smallest margin at the snapped pose."""
    W = R.shape[0]
    ladder_amb = np.zeros(W, bool)
    hi_found = np.zeros(W, bool)
    for tau in sorted(ladder):
        Rx, tx = snap.ray_pose(R, t, d, np.full(W, tau), rotation)
        cls = parity.classify(p, Rx, tx, precision)
        ladder_amb |= ~hi_found & (cls == 0)
        hi_found |= cls == -1
    Rs, ts, _, j = snap.snap(p, R, t, d, ladder, rotation=rotation)
    m = np.sort(op.margins(p, Rs, ts), axis=1)
    band = parity.constraint_bands(p, Rs, ts, precision).max(axis=1)
    tie = (j >= 0) & (m[:, 1] - m[:, 0] <= 2 * band)
    return ladder_amb, tie


def replayed_forward(p, seeds, pr, pt, seed, W, K, gp, precision):
    """The oracle pipeline on the GPU's decision path (the replay protocol): FP64 walks taking the
    top-k lists and ladder choices of the GPU traces (each checked against the oracle's own values
    outside the band), the oracle snap of their final poses, and the balls of those samples."""
    w = np.arange(W)
    out = {}
    for key, sampler, prm in (("rot", 0, pr), ("tr", 1, pt)):
        R, t, rep = parity.replay_walks(p, seeds, prm, seed, w, gp["trace_" + key], precision, sampler)
        assert rep.ok(), rep.inconsistent[:3]
        st = closure.center_stats(p, seeds, prm)
        R0, t0 = closure.start_walks(seeds, w)
        if sampler == 0:
            d = closure.init_angular_velocity(R0, st.Rbar, prm.omega0, seed, w)
        else:
            d = closure.init_center_velocity(t0, st.tbar, prm.v0, st.S, seed, w)
        rot = sampler == 0
        ladder = closure.step_ladder(prm)
        Rs, ts, _, j = snap.snap(p, R, t, d, ladder, rotation=rot)
        dh_dtau, dh_dy = snap.ray_derivatives(p, Rs, ts, d, j, rotation=rot)
        amb_ladder, tie = snap_ambiguous(p, R, t, d, ladder, rot, precision)
        out[key] = dict(R=R, t=t, Rs=Rs, ts=ts, dir=d, jstar=j, ray_rot=rot, dh_dtau=dh_dtau, dh_dy=dh_dy,
                        ambiguous=amb_ladder | tie, tie=tie)
    qs = canonical(quat_from_R(out["rot"]["Rs"]))
    C, D, f_rot = megb_rotation(qs, K)
    c, dd, f_tr = megb_translation(out["tr"]["ts"], K)
    out.update(q=qs, C=C, D=D, f_rot=f_rot, c=c, d=dd, f_tr=f_tr)
    return out


def check_records(g, o, ray_rot, mask, rtol):
    """Snap records of the walks in mask vs the oracle's (j*, ray kind, direction, h', dh/dy)."""
    j = o["jstar"]
    assert np.array_equal(g[mask, 0].astype(np.int64), j[mask])
    assert np.all(g[:, 1] == (0 if ray_rot else 1))
    ok = mask & (j >= 0)
    d = o["dir"]
    assert np.abs(g[ok, 2:5] - d[ok]).max() <= 1e-6 * np.abs(d).max()
    hp = o["dh_dtau"]
    err = np.abs(g[ok, 5] - hp[ok]) / (np.abs(hp[ok]) + 1e-3 * np.abs(hp).max())
    assert np.all(err <= rtol), (err.max(), g[ok, 5][np.argmax(err)], hp[ok][np.argmax(err)], np.nonzero(ok)[0][np.argmax(err)])
    dim = o["dh_dy"].shape[1]
    assert np.abs(g[ok, 6:6 + dim] - o["dh_dy"][ok]).max() <= rtol


def compare(p, fw, gp, precision):
    """Snapped samples, snap records, farthest sequences, balls and gradients against an oracle
    forward fw.  FP64: fw is the oracle's own free run and every walk matches.  FP32: fw follows the
    GPU's walk decisions (replay protocol); a snapped sample may differ only where the snap itself
    decides inside the FP32 band (a ladder point or an active-constraint tie), and none of those
    samples may define a ball."""
    qo = quat_from_R(fw["rot"]["Rs"])
    ang = np.array([parity.rot_angle(a, b) for a, b in zip(gp["qR"], qo)])
    dt = np.abs(gp["tT"] - fw["tr"]["ts"]).max(axis=1)
    if precision == 1:
        mR = ang <= 1e-9
        mT = dt <= 1e-12 * (1 + np.abs(fw["tr"]["ts"]).max())
        assert mR.all() and mT.all(), (ang.max(), dt.max())
        rtol, gtol = 1e-6, 1e-7
        rR, rT = mR, mT
    else:
        mR = ang <= 2e-6
        mT = dt <= 1e-6 * (1 + np.abs(fw["tr"]["ts"]).max())
        assert not (~mR & ~fw["rot"]["ambiguous"]).any(), (np.nonzero(~mR)[0], ang[~mR])
        assert not (~mT & ~fw["tr"]["ambiguous"]).any(), (np.nonzero(~mT)[0], dt[~mT])
        rtol, gtol = 1e-4, 1e-4
        # records (j* and its derivatives) of the matching samples whose active constraint is
        # decided outside the band
        rR, rT = mR & ~fw["rot"]["tie"], mT & ~fw["tr"]["tie"]
        print(f"FP32 snap: {int((~mR).sum())} / {int(fw['rot']['ambiguous'].sum())} rotation and "
              f"{int((~mT).sum())} / {int(fw['tr']['ambiguous'].sum())} translation samples differ / have a "
              f"band-ambiguous snap; records compared for {int(rR.sum())} and {int(rT.sum())} of {len(rR)}; "
              f"max angle {ang[mR].max():.2e} rad, max |dt| {dt[mT].max():.2e} m")
    check_records(gp["snR"], fw["rot"], True, rR, rtol)
    check_records(gp["snT"], fw["tr"], False, rT, rtol)
    K = len(fw["f_rot"])
    # GGD protocol: each farthest choice of the GPU is within the rounding band of the FP64 maximum
    # over its own samples (two samples at the ends of a diameter are equidistant from their
    # midpoint, so rounding may pick either, in FP64 too), then the oracle follows the GPU's sequence
    f_rot, f_tr = gp["far"][:K], gp["far"][K:]
    parity.check_rotation(gp["qR"], gp["res"], f_rot, precision)
    parity.check_translation(gp["tT"], gp["res"], f_tr, precision)
    qs = canonical(quat_from_R(fw["rot"]["Rs"]))
    C = megb_o.megb_rotation_replay(qs, f_rot)[-1]
    c = megb_o.megb_translation_replay(fw["tr"]["ts"], f_tr)[-1]
    fw = dict(fw, q=qs, C=C, D=float(megb_o.rotation_distances(C, qs).max()), f_rot=f_rot, c=c,
              d=float(np.sqrt(((fw["tr"]["ts"] - c) ** 2).sum(1)).max()), f_tr=f_tr)
    assert np.array_equal(gp["far"][:K], fw["f_rot"])
    assert np.array_equal(gp["far"][K:], fw["f_tr"])
    assert mR[fw["f_rot"]].all() and mT[fw["f_tr"]].all()
    assert abs(gp["res"][7] - fw["D"]) <= 1e-5 * fw["D"]
    assert abs(gp["res"][8] - fw["d"]) <= 1e-5 * fw["d"], (gp["res"][8], fw["d"], abs(gp["res"][8] - fw["d"]) / fw["d"])
    gy, gr = adjoint.closure_backward(p, fw, G_RES)
    scale = max(np.abs(gy).max(), np.abs(gr).max())
    assert np.abs(gp["gy"] - gy).max() <= gtol * scale, (np.abs(gp["gy"] - gy).max() / scale, gp["gy"], gy)
    assert np.abs(gp["gr"] - gr).max() <= gtol * scale, (np.abs(gp["gr"] - gr).max() / scale, gp["gr"], gr)
    return gy, gr


@pytest.mark.gpu
@pytest.mark.parametrize("lam", [False, True])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("precision", [1, 0])
def test_snap_balls_and_gradient_match_oracle(kind, precision, lam):
    """With lam: noise matrices (eq. 4); the snap, its records and the adjoint in the Lambda-norm."""
    p, seeds, pr, pt = case(kind, lam=lam)
    W, K, seed = 256, 100, 11
    gp = gpu_pipeline(p, seeds, pr, pt, seed, W, K, precision)
    if precision == 1:
        fw = adjoint.closure_balls(p, seeds, pr, pt, seed, W, K)
    else:
        fw = replayed_forward(p, seeds, pr, pt, seed, W, K, gp, precision)
    compare(p, fw, gp, precision)


@pytest.mark.gpu
@pytest.mark.parametrize("lam", [False, True])
def test_gradient_matches_central_differences_of_the_oracle_pipeline(lam):
    p, seeds, pr, pt = case(0, lam=lam)
    W, K, seed = 64, 60, 5
    fw = adjoint.closure_balls(p, seeds, pr, pt, seed, W, K)
    gp = gpu_pipeline(p, seeds, pr, pt, seed, W, K, 1)
    h = 1e-6
    checked = 0
    active = sorted(set(fw["rot"]["jstar"][fw["rot"]["jstar"] >= 0]) | set(fw["tr"]["jstar"][fw["tr"]["jstar"] >= 0]))
    for j in active:
        for c in range(4):
            vals = []
            for sgn in (1, -1):
                obs, radii = p.obs.copy(), p.radii.copy()
                if c < 3:
                    obs[j, c] += sgn * h
                else:
                    radii[j] += sgn * h
                fq = adjoint.closure_balls(syn.Purse(p.kind, p.model, obs, radii, p.K, lam=p.lam), seeds, pr, pt,
                                           seed, W, K)
                same = all(np.array_equal(fq[k][a], fw[k][a]) for k in ("rot", "tr") for a in ("R", "t", "jstar"))
                same = same and np.array_equal(fq["f_rot"], fw["f_rot"]) and np.array_equal(fq["f_tr"], fw["f_tr"])
                vals.append((float(G_RES @ np.concatenate([fq["C"], fq["c"], [fq["D"], fq["d"]]])), same))
            if not (vals[0][1] and vals[1][1]):
                continue
            fd = (vals[0][0] - vals[1][0]) / (2 * h)
            got = gp["gy"][j, c] if c < 3 else gp["gr"][j]
            assert abs(got - fd) <= 1e-7 + 1e-5 * abs(fd), (j, c, got, fd)
            checked += 1
    assert checked >= 6


@pytest.mark.gpu
@pytest.mark.parametrize("kind", [0, 1])
def test_autograd_function_gives_the_adjoint(kind):
    p, seeds, pr, pt = case(kind)
    W, K, seed = 256, 100, 11
    gp = gpu_pipeline(p, seeds, pr, pt, seed, W, K, 1)
    obs = torch.tensor(p.obs, dtype=torch.float64, requires_grad=True)
    radii = torch.tensor(p.radii, dtype=torch.float64, requires_grad=True)
    K_intr = p.K if kind == 1 else None
    C, c, D, d = AG.closure_balls(obs, radii, p.model, kind, K_intr, params_from(pr, 0, 1), params_from(pt, 1, 1),
                                  seeds, W, K, seed=seed, tr_sampler=1, precision=1)
    g = torch.as_tensor(G_RES)
    L = (g[:4].cuda() * C).sum() + (g[4:7].cuda() * c).sum() + g[7] * D + g[8] * d
    L.backward()
    assert np.allclose(C.detach().cpu().numpy(), gp["res"][:4], rtol=0, atol=0)
    assert np.array_equal(obs.grad.numpy(), gp["gy"])
    assert np.array_equal(radii.grad.numpy(), gp["gr"])


@pytest.mark.gpu
def test_translation_ball_from_rotation_walks_has_zero_gradient_and_empty_balls_are_skipped():
    p, seeds, pr, _ = case(0)
    W, K = 128, 30
    with P.Purse(p) as h:
        sd = to_dev(seeds.reshape(-1, 12))
        q = torch.empty((W, 4), dtype=torch.float64, device="cuda")
        t = torch.empty((W, 3), dtype=torch.float64, device="cuda")
        sn = torch.empty((W, 12), dtype=torch.float64, device="cuda")
        P.purse_sample(h.h, params_from(pr, 0, 1), 4, sd, 1, W, q, t, None, snap=sn)
        res = torch.empty(9, dtype=torch.float64, device="cuda")
        far = torch.empty(2 * K, dtype=torch.int32, device="cuda")
        P.megb_solve(h.h, 1, K, None, 0, t, W, res, far)
        gy = torch.full(p.obs.shape, np.nan, dtype=torch.float64, device="cuda")
        gr = torch.full((p.radii.shape[0],), np.nan, dtype=torch.float64, device="cuda")
        P.megb_backward(h.h, 1, K, None, None, 0, t, sn, W, far, res, to_dev(np.ones(9)), gy, gr)
        P.purse_sync(h.h)
        assert np.all(gy.cpu().numpy() == 0) and np.all(gr.cpu().numpy() == 0)


def test_megb_backward_rejects_bad_arguments():
    L = P.lib()
    buf = np.zeros(16).ctypes.data  # never dereferenced: validation fails first
    assert L.megb_backward(None, 0, 10, buf, buf, 1, buf, buf, 1, buf, buf, buf, buf, buf, None) == 1
