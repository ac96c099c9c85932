"""Autotuner cache (host logic, no GPU): keys by operation, PURSE kind, keypoint-count bucket
ceil(log2 n), sample-count bucket floor(log2 samples), variant and GPU name; persistence through
the PURSE_TUNE_CACHE file; clearing."""
import subprocess
import sys

from paper_2403_09990_gb300 import purse as P

GPU = "NVIDIA GB300"


def test_buckets_variants_and_gpus():
    P.purse_tune_cache_clear()
    P.purse_tune_cache_put(P.TUNE_MEGB, 1, 16, 1 << 20, 0, GPU, 16, 1.5)
    # the same buckets: n in (8, 16], samples in [2^20, 2^21)
    for n, s in ((16, 1 << 20), (9, (1 << 21) - 1), (12, 1500000)):
        got = P.purse_tune_cache_get(P.TUNE_MEGB, 1, n, s, 0, GPU)
        assert got is not None and got["config"] == 16 and abs(got["ms"] - 1.5) < 1e-6
    # another bucket, variant, kind, operation or GPU has no entry
    for args in ((P.TUNE_MEGB, 1, 17, 1 << 20, 0, GPU), (P.TUNE_MEGB, 1, 16, 1 << 21, 0, GPU),
                 (P.TUNE_MEGB, 1, 16, 1 << 20, 1, GPU), (P.TUNE_MEGB, 0, 16, 1 << 20, 0, GPU),
                 (P.TUNE_WALK, 1, 16, 1 << 20, 0, GPU), (P.TUNE_MEGB, 1, 16, 1 << 20, 0, "NVIDIA B200")):
        assert P.purse_tune_cache_get(*args) is None, args
    # a later choice replaces the earlier one
    P.purse_tune_cache_put(P.TUNE_MEGB, 1, 16, 1 << 20, 0, GPU, 8, 1.2)
    assert P.purse_tune_cache_get(P.TUNE_MEGB, 1, 16, 1 << 20, 0, GPU)["config"] == 8
    P.purse_tune_cache_clear()
    assert P.purse_tune_cache_get(P.TUNE_MEGB, 1, 16, 1 << 20, 0, GPU) is None


def test_cache_file_survives_the_process(tmp_path):
    path = tmp_path / "tune.txt"
    code = ("from paper_2403_09990_gb300 import purse as P; P.purse_tune_cache_put(P.TUNE_WALK, 0, 8, 4096, 2, "
            "'NVIDIA GB300', 4, 0.25); P.purse_tune_cache_put(P.TUNE_DIST, 1, 64, 1 << 24, 3, 'NVIDIA GB300', 2, 3.0)")
    env = {"PURSE_TUNE_CACHE": str(path)}
    import os
    subprocess.run([sys.executable, "-c", code], check=True, env=dict(os.environ, **env))
    assert path.read_text().count("\n") == 2
    check = ("from paper_2403_09990_gb300 import purse as P; a = P.purse_tune_cache_get(P.TUNE_WALK, 0, 7, 5000, 2, "
             "'NVIDIA GB300'); b = P.purse_tune_cache_get(P.TUNE_DIST, 1, 50, (1 << 24) + 5, 3, 'NVIDIA GB300'); "
             "print(a['config'], b['config'], P.purse_tune_cache_get(P.TUNE_WALK, 0, 7, 5000, 0, 'NVIDIA GB300'))")
    out = subprocess.run([sys.executable, "-c", check], check=True, capture_output=True, text=True,
                         env=dict(os.environ, **env)).stdout.split()
    assert out == ["4", "2", "None"]


def test_bad_arguments():
    L = P.lib()
    assert L.purse_tune_cache_put(9, 0, 8, 100, 0, b"x", 1, 0.0) == 1
    assert L.purse_tune_cache_put(0, 0, 0, 100, 0, b"x", 1, 0.0) == 1
    assert L.purse_tune_walk(None, None, 0, None, 0, 0, None, None, None, None) == 1
    assert L.purse_tune_dist(None, 1, None, 0, None, None, None) == 1
