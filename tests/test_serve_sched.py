"""Host-side checks of the reconstruction server (no GPU).

* The job scheduler and the evaluation batcher (paper_2110_08868_gb300/csrc/
  serve_sched.h) are compiled with g++ against a fake device whose jobs sleep, and
  checked for: the byte budget and the slot count bound what runs at once, admission
  is FIFO without overtaking, a job that can never fit is refused, failures keep their
  code, timed waits, destruction with jobs in flight, many submitting threads; each
  batched request gets its own result, concurrent requests share batches, batches are
  capped, the batching window, and the batcher's worker shutdown.
* The admission footprint (sdot_server_footprint) is computed on the host from the
  allocation list of a context; it is checked against the arrays a context holds.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_scheduler_with_fake_device(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "serve_sched_test")
    cmd = [gxx, "-std=c++17", "-O1", "-Wall", "-Wextra", "-pthread",
           "-I", os.path.join(ROOT, "paper_2110_08868_gb300", "csrc"),
           "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "serve_sched_test.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "FAIL" not in r.stdout
    assert r.stdout.count("ok") >= 40


def _fp(n, box=(1.0, 1.0, 1.0), **opts):
    from paper_2110_08868_gb300 import binding as B
    from paper_2110_08868_gb300 import build

    build.build()
    return B.sdot_server_footprint(n, box, B.sdot_default_options(**opts) if opts else None)


def test_footprint_counts_the_context_arrays():
    from paper_2110_08868_gb300 import binding as B

    rc, b32 = _fp(32 ** 3)
    assert rc == B.SDOT_OK
    rc, b128 = _fp(128 ** 3)
    assert rc == B.SDOT_OK
    # per seed: positions/offsets/psi/masses (~130 B), kNN 24 x 4 B, facet slab
    # 64 x 12 B, stored topology 257 B, carried certificate ~157 B (ball and reserves,
    # FP16 supports, 16 seeds, count, previous psi), CG vectors, staging, and the CSR
    # reserve of 25 x 12 B
    per = (b128 - b32) / (128 ** 3 - 32 ** 3)
    assert 1600 < per < 1950, per
    # fixed part: the 8 MB reduction buffer and small arrays
    fixed = b32 - per * 32 ** 3
    assert 8e6 < fixed < 12e6, fixed
    # each extra neighbour in the kNN list costs 4 bytes per seed
    rc, b48 = _fp(64 ** 3, k=48)
    rc, b24 = _fp(64 ** 3, k=24)
    assert abs((b48 - b24) - 24 * 4 * 64 ** 3) < 4096
    # scale-free in the box size (grid and pyramid follow N, not L)
    assert _fp(64 ** 3, box=(1000.0,) * 3)[1] == b24


def test_footprint_rejects_bad_input():
    from paper_2110_08868_gb300 import binding as B

    assert _fp(1)[0] == B.SDOT_ERR_ARG
    assert _fp(100, box=(1.0, -1.0, 1.0))[0] == B.SDOT_ERR_ARG
    assert _fp(10, k=24)[0] == B.SDOT_ERR_ARG  # k >= N
    assert _fp(1000, precision=7)[0] == B.SDOT_ERR_ARG


def test_serving_stream_recipe():
    from paper_2110_08868_gb300 import ics

    s1, g1 = ics.serving_stream(64)
    s2, g2 = ics.serving_stream(64)
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(g1, g2)
    assert s1.min() >= 32 and s1.max() <= 128 and len(s1) == 64
    # log-uniform in the side: median near exp((ln 32 + ln 128) / 2) = 64
    assert 45 <= np.median(s1) <= 90
    assert g1[0] == 0.0 and (g1[1:] > 0).all() and 0.6 < g1[1:].mean() < 1.5


def test_nearest_rank_quantiles():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    v = list(range(1, 101))
    assert bench.nearest_rank(v, 0.50) == 50
    assert bench.nearest_rank(v, 0.99) == 99
    assert bench.nearest_rank([3.0], 0.99) == 3.0
    assert bench.nearest_rank(list(range(1, 65)), 0.99) == 64  # ceil(63.36) = 64
