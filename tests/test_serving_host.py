"""Host side of the serving benchmark (no GPU): the seeded request stream
has the specified mix, valid non-isolated sources and Poisson arrivals, and
is reproducible."""
import numpy as np
import pytest

import graphgen as gg


def small_pool():
    out = []
    for kind, a, b, seed in [("rmat", 10, 8, 1), ("grid", 32, 0, 2)]:
        if kind == "rmat":
            r, c = gg.rmat(a, b, seed=seed)
        else:
            r, c = gg.grid(a, p_del=0.05, seed=seed)
        out.append((kind, a, b, seed, r, c, None))
    return out


def test_request_stream_mix_sources_and_arrivals():
    import bench
    pool = small_pool()
    reqs, unit = bench.serving_requests(pool, 20000, seed=6)
    assert len(reqs) == 20000 and unit.shape == (20000,)
    kinds = np.array([k for _, k, _ in reqs])
    frac = np.bincount(kinds, minlength=3) / kinds.size
    # 60 / 30 / 10 within a few standard deviations of a multinomial draw
    assert np.allclose(frac, [0.6, 0.3, 0.1], atol=0.02)
    for gi, _, s in reqs:
        r = pool[gi][4]
        assert 0 <= s < r.size - 1 and r[s + 1] > r[s]  # non-isolated
    gaps = np.diff(np.concatenate([[0.0], unit]))
    assert np.all(gaps > 0)
    # unit-rate exponential gaps: mean 1, coefficient of variation 1
    assert abs(gaps.mean() - 1.0) < 0.05 and abs(gaps.std() / gaps.mean() - 1.0) < 0.05
    reqs2, unit2 = bench.serving_requests(pool, 20000, seed=6)
    assert reqs2 == reqs and np.array_equal(unit2, unit)
    reqs3, _ = bench.serving_requests(pool, 200, seed=7)
    assert reqs3 != reqs[:200]


def test_server_core_lifecycle_and_admission(tmp_path):
    """The query server's host-only core, built with g++ and a fake device:
    a batch that fails after enqueueing work is waited for before the slot
    reallocates or reuses any buffer (a fake of the earlier order, which
    skipped that wait on error, is caught), and admission counts result
    buffers and the workspaces a batch must create against the budget."""
    import os
    import shutil
    import subprocess
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    exe = str(tmp_path / "server_core_check")
    subprocess.check_call([gxx, "-std=c++17", "-O1", "-Wall",
                           "-I", os.path.join(root, "include"),
                           "-I", os.path.join(root, "paper_1501_05387_gb300", "csrc"),
                           os.path.join(root, "tests", "server_core_check.cpp"), "-o", exe])
    res = subprocess.run([exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout + res.stderr
    assert res.stdout.strip().endswith("ok")
