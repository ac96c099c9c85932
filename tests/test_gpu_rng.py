"""GPU random streams are bit-identical to the oracle's (Philox4x32-10 and lattice draws)."""
import numpy as np
import pytest
import torch

from oracle import philox
from paper_2403_09990_gb300 import purse as P

pytestmark = pytest.mark.gpu


def gpu_words(seed, phase, j, i, w0, n, n_words, unit=0):
    words = torch.empty((n, n_words), dtype=torch.int32, device="cuda")
    lat = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    P.purse_rng_words(seed, phase, j, i, w0, n, n_words, words, lat, unit)
    torch.cuda.synchronize()
    return words.cpu().numpy().view(np.uint32), lat.cpu().numpy()


def test_known_answer_on_gpu():
    # counter (0, 0, 0, 0) with key (0, 0) is stream (phase 0, j 0, i 0, w 0), block 0
    w, _ = gpu_words(0, 0, 0, 0, 0, 1, 4)
    assert [int(x) for x in w[0]] == [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]


@pytest.mark.parametrize("seed,phase,j,i,w0,unit", [
    (0, philox.PHASE_R_PERTURB, 0, 0, 0, 0),
    (0x0123456789ABCDEF, philox.PHASE_R_PERTURB, 149, 99, 1 << 20, 0),
    (7, philox.PHASE_T_PERTURB, 3, 4, 12345, 0),
    (7, philox.PHASE_OMEGA, 0, 0, 0, 1),
    (2**64 - 1, philox.PHASE_RANSAG, 2, 0, 2**32 - 4096, 0),
])
def test_streams_and_lattice_draws_bit_equal(seed, phase, j, i, w0, unit):
    n, nw = 4096, 12
    words, lat = gpu_words(seed, phase, j, i, w0, n, nw, unit)
    w = np.arange(w0, w0 + n, dtype=np.uint64)
    ref = philox.stream_words(seed, phase, j, i, w, nw).astype(np.uint32)
    assert np.array_equal(words, ref)
    pts, used = philox.ball_points(seed, phase, j, i, w, unit=bool(unit))
    X = lat[:, :3].astype(np.float64)
    if unit:
        got = X / np.linalg.norm(X, axis=1, keepdims=True)
        assert np.allclose(got, pts, rtol=0, atol=1e-15)
    else:
        assert np.array_equal(X / 1024.0, pts)
    assert np.array_equal(lat[:, 3], used)


def test_2_24_words_bit_equal():
    n, nw = 1 << 20, 16
    words, _ = gpu_words(42, philox.PHASE_R_PERTURB, 17, 3, 0, n, nw)
    ref = philox.stream_words(42, philox.PHASE_R_PERTURB, 17, 3, np.arange(n, dtype=np.uint64), nw)
    assert np.array_equal(words, ref.astype(np.uint32))
