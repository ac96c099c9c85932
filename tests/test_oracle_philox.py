"""Pins of the oracle's counter-based generator and draws (CPU only)."""
import os

import numpy as np
import pytest

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(x, 16) for x in line.split()])
    return rows


@pytest.mark.parametrize("row", _kat_rows())
def test_philox_known_answers(row):
    c, k, want = row[:4], row[4:6], row[6:]
    got = philox.philox4x32_10(*c, *k)
    assert [int(x) for x in got] == want


def test_stream_word_layout():
    # word k of stream (phase, j, i, w) is output lane k&3 of counter block k>>2
    seed = 0x0123456789ABCDEF
    words = philox.stream_words(seed, 3, 7, 11, 13, 10)
    lo, hi = philox.key_words(seed)
    for k in range(10):
        r = philox.philox4x32_10(k >> 2, (3 << 24) | 7, 11, 13, lo, hi)
        assert int(words[k]) == int(r[k & 3])
    # an offset window is the same words
    tail = philox.stream_words(seed, 3, 7, 11, 13, 4, start=6)
    assert np.array_equal(tail, words[6:10])


def test_ball_points_uniform_in_ball():
    w = np.arange(200_000)
    pts, used = philox.ball_points(5, philox.PHASE_R_PERTURB, 0, 0, w)
    r2 = (pts ** 2).sum(1)
    assert r2.max() <= 1.0
    # acceptance rate of a cube -> ball rejection is pi/6
    rate = len(w) / used.sum()
    assert abs(rate - np.pi / 6) < 0.005
    # uniform in the unit 3-ball: E|x|^2 = 3/5, mean 0, isotropic
    assert abs(r2.mean() - 0.6) < 0.005
    assert np.abs(pts.mean(0)).max() < 0.005
    assert np.abs((pts ** 2).mean(0) - 0.2).max() < 0.005


def test_lattice_is_symmetric_and_decodes_each_word():
    words = np.array([0, 0x3FFFFFFF, (5 << 20) | (7 << 10) | 1023])
    X = philox.lattice_point(words)
    assert X.tolist() == [[-1023, -1023, -1023], [1023, 1023, 1023], [1023, 2 * 7 - 1023, 2 * 5 - 1023]]
    all_vals = 2 * np.arange(1024) - 1023
    assert all_vals.sum() == 0 and np.all(all_vals % 2 == 1)


def test_unit_vectors():
    w = np.arange(100_000)
    u, _ = philox.ball_points(9, philox.PHASE_OMEGA, 0, 0, w, unit=True)
    assert np.allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-15)
    assert np.abs(u.mean(0)).max() < 0.01
    assert np.abs((u ** 2).mean(0) - 1 / 3).max() < 0.01


def test_distinct_triple_uniform():
    words = philox.stream_words(1, philox.PHASE_RANSAG, 0, 0, np.arange(120_000), 3)
    n = 6
    idx = philox.distinct_triple(words, n)
    assert idx.min() >= 0 and idx.max() < n
    assert np.all(idx[:, 0] != idx[:, 1]) and np.all(idx[:, 0] != idx[:, 2]) and np.all(idx[:, 1] != idx[:, 2])
    # each ordered triple of distinct indices equally likely: 6*5*4 = 120 cells
    code = idx[:, 0] * 36 + idx[:, 1] * 6 + idx[:, 2]
    counts = np.bincount(code, minlength=216)
    cells = counts[counts > 0]
    assert len(cells) == 120
    chi2 = ((cells - 1000.0) ** 2 / 1000.0).sum()
    assert chi2 < 200  # 119 dof; p ~ 1e-5 at 200


def test_hatbox_points_decode_the_stream_words():
    seed, n_points = 77, 150
    w = np.array([0, 5, 123456])
    pts = philox.hatbox_points(seed, philox.PHASE_R_PERTURB, 3, w, n_points)
    assert pts.shape == (3, n_points, 3)
    for wi, ww in enumerate(w):
        for j in (0, 1, 2, 77, 148, 149):
            wd = [int(x) for x in philox.stream_words(seed, philox.PHASE_R_PERTURB, j >> 1, 3, ww, 4)]
            w0, w1 = wd[2 * (j & 1)], wd[2 * (j & 1) + 1]
            z = ((w0 >> 16) + 0.5) / 32768 - 1
            x = ((w0 & 0xFFFF) + 0.5) / 32768
            rho = (max(w1 & 1023, (w1 >> 10) & 1023, (w1 >> 20) & 1023) + 0.5) / 1024
            s = np.sqrt(1 - z * z)
            ref = rho * np.array([s * np.cos(np.pi * x), s * np.sin(np.pi * x), z])
            assert np.allclose(pts[wi, j], ref, rtol=0, atol=1e-15)


def test_hatbox_points_uniform_in_ball():
    pts = philox.hatbox_points(3, philox.PHASE_T_PERTURB, 0, np.arange(2000), 150).reshape(-1, 3)
    r = np.linalg.norm(pts, axis=1)
    assert r.max() <= 1.0
    # radius law of the uniform ball: P(|x| <= rho) = rho^3
    for rho in (0.3, 0.5, 0.8, 0.95):
        assert abs((r <= rho).mean() - rho ** 3) < 0.004
    assert abs((r ** 2).mean() - 0.6) < 0.003
    assert np.abs(pts.mean(0)).max() < 0.003
    assert np.abs((pts ** 2).mean(0) - 0.2).max() < 0.003
    # isotropy of the direction: octant frequencies
    oct_ = (pts > 0).astype(int) @ np.array([1, 2, 4])
    f = np.bincount(oct_, minlength=8) / len(pts)
    assert np.abs(f - 0.125).max() < 0.003
