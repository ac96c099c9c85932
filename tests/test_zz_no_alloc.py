"""megb_solve_noalloc: the ball solver for callers that cannot allocate device memory.

Some callers must not allocate once running: real-time perception loops that
reserve all memory at start-up (cudaMalloc / cudaFree may synchronise the
device and take unbounded time), and hosts whose device memory belongs to
another allocator.  megb_solve_noalloc keeps its scratch in a static 64 KiB
device array instead; here it is checked, through the C ABI, against
megb_solve on calls in a row (each call finds the previous call's leftovers in
the shared array), up to 2^20 samples, where its grid is smaller than
megb_solve's.
"""
import numpy as np
import pytest
import torch

from oracle import so3
from paper_2403_09990_gb300 import purse as P
from paper_2403_09990_gb300 import synthetic as syn
from tests import parity


def _cluster(n, seed, dtype):
    rng = np.random.default_rng(seed)
    C0 = so3.quat_from_R(so3.exp_so3(rng.normal(size=3)))
    q = so3.quat_mul(so3.quat_exp(rng.normal(size=(n, 3)) * np.array([0.02, 0.05, 0.1])), C0[None])
    t = rng.normal(size=(n, 3)) * np.array([0.003, 0.003, 0.03]) + rng.normal(size=3)
    dt = torch.float32 if dtype == 0 else torch.float64
    return torch.as_tensor(q, dtype=dt).cuda(), torch.as_tensor(t, dtype=dt).cuda()


def _both(h, precision, K, q, nq, t, nt):
    ref = torch.full((9,), np.nan, dtype=torch.float64, device="cuda")
    got = torch.full((9,), np.nan, dtype=torch.float64, device="cuda")
    f_ref = torch.full((2 * K,), -1, dtype=torch.int32, device="cuda")
    f_got = torch.full((2 * K,), -1, dtype=torch.int32, device="cuda")
    P.megb_solve(h, precision, K, q, nq, t, nt, ref, f_ref)
    P.megb_solve_noalloc(precision, K, q, nq, t, nt, got, f_got)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), got.cpu().numpy(), f_ref.cpu().numpy(), f_got.cpu().numpy()


def _assert_same(ref, got, f_ref, f_got, nq, nt, K):
    if nq:
        assert np.array_equal(f_ref[:K], f_got[:K])
        assert parity.rot_angle(got[:4], ref[:4]) <= 1e-9
        assert abs(got[7] - ref[7]) <= 1e-5 * ref[7] + 1e-12
    if nt:
        assert np.array_equal(f_ref[K:], f_got[K:])
        assert np.abs(got[4:7] - ref[4:7]).max() <= 1e-12 * (1 + np.abs(ref[4:7]).max())
        assert abs(got[8] - ref[8]) <= 1e-5 * ref[8] + 1e-12


@pytest.mark.gpu
def test_noalloc_matches_megb_solve_on_two_calls_in_a_row():
    with P.Purse(syn.purse_3d3d(8, 0)) as h:
        # call 1: both balls, FP32 samples, 200 iterations
        q, t = _cluster(4096, 1, 0)
        ref, got, f_ref, f_got = _both(h.h, 0, 200, q, 4096, t, 4096)
        _assert_same(ref, got, f_ref, f_got, 4096, 4096, 200)
        # call 2: other sizes and precision, rotation ball only, fewer iterations
        q2, _ = _cluster(77777, 2, 1)
        ref, got, f_ref, f_got = _both(h.h, 1, 57, q2, 77777, None, 0)
        _assert_same(ref, got, f_ref, f_got, 77777, 0, 57)
        assert np.all(got[4:7] == 0) and got[8] == 0
        # call 3: 2^20 samples (the size of the single-PURSE workload), where the grid of this
        # entry point (at most 512 blocks) is smaller than megb_solve's (4 x SMs) and the
        # grid-stride loops take several samples per thread
        q3, t3 = _cluster(1 << 20, 3, 0)
        ref, got, f_ref, f_got = _both(h.h, 0, 200, q3, 1 << 20, t3, 1 << 20)
        _assert_same(ref, got, f_ref, f_got, 1 << 20, 1 << 20, 200)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = P.lib()
    buf = (np.zeros(9)).ctypes.data  # never dereferenced: validation fails first
    assert L.megb_solve_noalloc(0, 4097, buf, 10, buf, 10, buf, None, None) == 1
    assert b"4096" in L.purse_last_error()
    assert L.megb_solve_noalloc(0, 0, buf, 10, buf, 10, buf, None, None) == 1
    assert L.megb_solve_noalloc(0, 10, buf, 2**31 - 2**20, buf, 10, buf, None, None) == 1
    assert L.megb_solve_noalloc(2, 10, buf, 10, buf, 10, buf, None, None) == 1
