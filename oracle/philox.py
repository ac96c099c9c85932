"""Philox4x32-10 and the random streams the walks draw from (oracle side).

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and
Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of
two 32x32->64 multiplies (constants 0xD2511F53 on word 0, 0xCD9E8D57 on
word 2) mixed with the key, the key advanced by the Weyl constants
(0x9E3779B9, 0xBB67AE85) before every round after the first.
Pinned by the published known-answer vectors (tests/golden/).

Stream layout (the CUDA side implements the same definition on its own):
a stream is named by (key, phase, j, i, w) and its word k is
    philox(ctr = (k >> 2, (phase << 24) | j, i, w), key = (lo32, hi32))[k & 3].
phase: 1 translation perturbations of the rotation-boundary walk (Alg. 3),
2 rotation perturbations of the translation-boundary walk (Alg. 5) -- for
these two, perturbations j = 2b and 2b + 1 of iteration i of walk w are the
two points of block 0 of stream (phase, b, i, w) (see hatbox_points);
3 the random unit vector of init_angular_velocity, 4 that of
init_center_velocity, 5 one RANSAG trial (w = trial index; j = 0 gives
the three constraint indices, j = 1, 2, 3 the three points drawn inside
the chosen noise balls -- disks of pixels for 2D-3D, see disk_points).
A batched PURSE p uses key = seed + p (mod 2^64).

Perturbation points (phases 1, 2) use no rejection: point h of a block takes
words 2h, 2h + 1 = (w0, w1); the direction follows Archimedes' hat-box theorem
with z = ((w0 >> 16) + 1/2) / 2^15 - 1 and azimuth pi x, x = ((w0 & 0xFFFF) +
1/2) / 2^15; the radius is (max of the three 10-bit fields of w1 + 1/2) / 2^10,
whose cube is uniform, so the point is uniform in the unit ball.

Other uniform ball points are drawn by integer rejection on a symmetric lattice so
both sides take the same accept decisions: attempt a uses word a of the
stream and X_c = 2 ((word >> 10c) & 1023) - 1023 for c = 0, 1, 2 (odd
integers in [-1023, 1023]); it is accepted when sum X_c^2 <= 2^20 and the
point is X / 1024.  Random unit vectors accept 2^14 <= sum X_c^2 <= 2^20
and return X / |X|.  After MAX_ATTEMPTS rejections the draw is the zero
vector.
"""
from __future__ import annotations

import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)

PHASE_R_PERTURB = 1
PHASE_T_PERTURB = 2
PHASE_OMEGA = 3
PHASE_V = 4
PHASE_RANSAG = 5

MAX_ATTEMPTS = 64
BALL_R2 = 1 << 20
UNIT_R2_MIN = 1 << 14


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10; arguments are integer arrays of 32-bit values."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK32 for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def key_words(seed: int):
    s = int(seed) & 0xFFFFFFFFFFFFFFFF
    return s & 0xFFFFFFFF, s >> 32


def stream_words(seed: int, phase: int, j, i, w, n_words: int, start: int = 0) -> np.ndarray:
    """Words [start, start + n_words) of the streams named by broadcast (j, i, w).

    Returns uint64 array of shape broadcast(j, i, w).shape + (n_words,).
    """
    k0, k1 = key_words(seed)
    j, i, w = np.broadcast_arrays(np.asarray(j, np.uint64), np.asarray(i, np.uint64),
                                  np.asarray(w, np.uint64))
    ks = np.arange(start, start + n_words, dtype=np.uint64)
    blocks = np.unique(ks >> np.uint64(2))
    out = np.empty(j.shape + (n_words,), dtype=np.uint64)
    c1 = (np.uint64(phase) << np.uint64(24)) | j
    for b in blocks:
        r = philox4x32_10(np.full(j.shape, b, np.uint64), c1, i, w, k0, k1)
        for pos, k in enumerate(ks):
            if (k >> np.uint64(2)) == b:
                out[..., pos] = r[int(k & np.uint64(3))]
    return out


def lattice_point(words: np.ndarray) -> np.ndarray:
    """Odd-integer lattice coordinates (..., 3) of each word."""
    w = np.asarray(words, dtype=np.int64)
    return np.stack([2 * ((w >> (10 * c)) & 1023) - 1023 for c in range(3)], axis=-1)


def ball_points(seed: int, phase: int, j, i, w, unit: bool = False):
    """First accepted rejection attempt of each stream.

    Returns (points float64 (..., 3), words_used int64 (...)).  ``unit``
    selects the random-unit-vector acceptance region.
    """
    shape = np.broadcast_shapes(np.shape(j), np.shape(i), np.shape(w))
    pts = np.zeros(shape + (3,))
    used = np.full(shape, MAX_ATTEMPTS, dtype=np.int64)
    done = np.zeros(shape, dtype=bool)
    chunk = 8  # attempts (words) per batch
    for a0 in range(0, MAX_ATTEMPTS, chunk):
        if done.all():
            break
        X = lattice_point(stream_words(seed, phase, j, i, w, chunk, start=a0))   # (..., chunk, 3)
        r2 = (X * X).sum(axis=-1)
        ok = r2 <= BALL_R2
        if unit:
            ok &= r2 >= UNIT_R2_MIN
        for a in range(chunk):
            take = ok[..., a] & ~done
            if take.any():
                Xa = X[..., a, :].astype(np.float64)
                if unit:
                    val = Xa / np.sqrt(r2[..., a].astype(np.float64))[..., None]
                else:
                    val = Xa / 1024.0
                pts[take] = val[take]
                used[take] = a0 + a + 1
                done |= take
    return pts, used


def disk_points(seed: int, phase: int, j, i, w):
    """First accepted attempt of each stream in the unit disk: attempt a uses word a,
    X = 2 (word & 1023) - 1023, Y = 2 ((word >> 10) & 1023) - 1023, accepted when
    X^2 + Y^2 <= 2^20; the point is (X, Y) / 1024 (zero after MAX_ATTEMPTS rejections).

    Returns (points float64 (..., 2), words_used int64 (...))."""
    shape = np.broadcast_shapes(np.shape(j), np.shape(i), np.shape(w))
    pts = np.zeros(shape + (2,))
    used = np.full(shape, MAX_ATTEMPTS, dtype=np.int64)
    done = np.zeros(shape, dtype=bool)
    chunk = 8
    for a0 in range(0, MAX_ATTEMPTS, chunk):
        if done.all():
            break
        X = lattice_point(stream_words(seed, phase, j, i, w, chunk, start=a0))[..., :2]   # (..., chunk, 2)
        ok = (X * X).sum(axis=-1) <= BALL_R2
        for a in range(chunk):
            take = ok[..., a] & ~done
            if take.any():
                pts[take] = (X[..., a, :].astype(np.float64) / 1024.0)[take]
                used[take] = a0 + a + 1
                done |= take
    return pts, used


def hatbox_points(seed: int, phase: int, i, w, n_points: int):
    """Perturbation points j = 0..n_points-1 of iteration i of walks w: (..., n_points, 3)."""
    w = np.asarray(w, dtype=np.uint64)
    j = np.arange(n_points)
    words = stream_words(seed, phase, (j >> 1).astype(np.uint64), i, w[..., None], 4)     # (..., n_points, 4)
    h = (j & 1)[None, :] if w.ndim else (j & 1)
    w0 = np.take_along_axis(words, np.broadcast_to(2 * h, words.shape[:-1])[..., None], -1)[..., 0].astype(np.int64)
    w1 = np.take_along_axis(words, np.broadcast_to(2 * h + 1, words.shape[:-1])[..., None], -1)[..., 0].astype(np.int64)
    z = ((w0 >> 16) + 0.5) / 32768.0 - 1.0
    x = ((w0 & 0xFFFF) + 0.5) / 32768.0
    k = np.maximum(np.maximum(w1 & 1023, (w1 >> 10) & 1023), (w1 >> 20) & 1023)
    rho = (k + 0.5) / 1024.0
    s = np.sqrt(1.0 - z * z)
    return rho[..., None] * np.stack([s * np.cos(np.pi * x), s * np.sin(np.pi * x), z], axis=-1)


def uniform_index(word, n):
    """Multiply-shift map of a 32-bit word to {0, ..., n-1}."""
    return ((np.asarray(word, np.uint64) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)


def distinct_triple(words, n):
    """Three distinct indices in {0..n-1} from three words (n >= 3)."""
    i1 = uniform_index(words[..., 0], n)
    i2 = uniform_index(words[..., 1], n - 1)
    i2 = i2 + (i2 >= i1)
    i3 = uniform_index(words[..., 2], n - 2)
    lo, hi = np.minimum(i1, i2), np.maximum(i1, i2)
    i3 = i3 + (i3 >= lo)
    i3 = i3 + (i3 >= hi)
    return np.stack([i1, i2, i3], axis=-1)
