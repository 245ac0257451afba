"""Host-side logic on the CPU: the seeded input generators, the warm-start
helpers that run on the host (problem keywords, resampling of the
prediction, the holdout split, the stratified sweep subset) and the
benchmark's bookkeeping (strict JSON, whole-job throughput, peaks, the
traffic figure's source check).  Nothing here launches a kernel."""
import json
import math
import os
import sys

import numpy as np
import pytest

from paper_2306_08216_gb300 import warmstart as WS
from paper_2306_08216_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


# ------------------------------------------------------------ input generators

def test_seeded_generators_repeat_and_differ_by_seed():
    a = W.random_fields(17, 11, 0.02, 3)
    b = W.random_fields(17, 11, 0.02, 3)
    c = W.random_fields(17, 11, 0.02, 4)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    assert any(not np.array_equal(x, z) for x, z in zip(a, c))
    assert all(x.shape == (11, 17) for x in a)
    r1, n1 = W.warm_start_draws(50, 7)
    r2, n2 = W.warm_start_draws(50, 7)
    np.testing.assert_array_equal(r1, r2)
    np.testing.assert_array_equal(n1, n2)


def test_parameter_draws_cover_their_ranges():
    re, n = W.warm_start_draws(4000, 1)
    assert re.min() >= 100.0 and re.max() <= 1000.0
    assert n.min() >= 0.5 and n.max() <= 1.5
    # log-uniform: log Re has the mean of its range to a few standard errors
    lo, hi = math.log(100.0), math.log(1000.0)
    se = (hi - lo) / math.sqrt(12 * re.size)
    assert abs(np.log(re).mean() - 0.5 * (lo + hi)) < 4 * se
    re, n, sides = W.cavity_batch_draws(512)
    assert re.min() >= 100.0 and re.max() <= 5000.0
    assert set(np.unique(sides)) == {65, 129, 257, 513}


def test_grid_generators():
    x = W.tanh_nodes(41, 1.5)
    assert abs(x[0]) < 1e-15 and abs(x[-1] - 1.0) < 1e-15
    assert np.all(np.diff(x) > 0)
    np.testing.assert_allclose(x + x[::-1], 1.0, atol=1e-15)  # symmetric about the middle
    assert np.diff(x)[0] < np.diff(x)[20]                       # clustered at the walls
    X, Y = W.trapezoid_grid(9, 7)
    assert X.shape == (7, 9)
    np.testing.assert_allclose([X[0, 0], X[0, -1], X[-1, 0], X[-1, -1]], [0.25, 0.75, 0.0, 1.0], atol=1e-15)
    np.testing.assert_allclose(Y[:, 0], np.linspace(0.0, 1.0, 7), atol=1e-15)
    np.testing.assert_allclose(W.periodic_nodes(8, 2.0), np.arange(8) * 0.25)


def test_warm_start_input_planes():
    x = W.warm_start_inputs([100.0, 1000.0], [0.5, 1.5], 16, geometry=["square", "trapezoid"])
    assert x.shape == (2, W.WARM_IN_PLANES, 16, 16) and x.dtype == np.float32
    np.testing.assert_allclose(x[0, 0], -1.0)
    np.testing.assert_allclose(x[1, 0], 1.0, rtol=1e-6)
    np.testing.assert_allclose(x[0, 1], -1.0)
    np.testing.assert_allclose(x[1, 1], 1.0)
    np.testing.assert_allclose(x[0, 4:], np.stack([np.ones((16, 16)), np.zeros((16, 16)),
                                                   np.zeros((16, 16)), np.ones((16, 16))]))


# ------------------------------------------------------------ warm-start helpers

@pytest.mark.parametrize("n_index", [0.5, 1.0, 1.4])
def test_cavity_problem_keywords(n_index):
    """Re = u0^(2-n) L^n / K with L = 1; nu_ref = K (u0/L)^(n-1) = u0 L / Re;
    clamps at nu_ref / 20 and 20 nu_ref; the trapezoid carries its grid."""
    re = 400.0
    kw = WS.cavity_problem(33, re, n_index)
    K, n, lo, hi = kw["power_law"]
    assert n == n_index
    np.testing.assert_allclose(WS.U_LID ** (2 - n_index) / K, re, rtol=1e-12)
    np.testing.assert_allclose(kw["nu"], WS.U_LID / re, rtol=1e-12)
    np.testing.assert_allclose([lo, hi], [kw["nu"] / 20, kw["nu"] * 20], rtol=1e-12)
    assert kw["walls"] == (True, True) and kw["u_wall"][3] == WS.U_LID
    kt = WS.cavity_problem(33, re, n_index, geometry="trapezoid")
    assert kt["grid"] == "curvilinear" and kt["x"].shape == (33, 33)


def test_resample_keeps_corners_and_linear_planes():
    rng = np.random.default_rng(0)
    f = rng.standard_normal((3, 12, 12))
    g = WS.resample(f, 29)
    assert g.shape == (3, 29, 29)
    for (i, j) in [(0, 0), (0, -1), (-1, 0), (-1, -1)]:
        np.testing.assert_allclose(g[:, i, j], f[:, i, j], rtol=1e-12)
    s = np.linspace(0.0, 1.0, 12)
    lin = 3.0 * s[None, :] - 2.0 * s[:, None] + 0.5
    t = np.linspace(0.0, 1.0, 29)
    np.testing.assert_allclose(WS.resample(lin, 29), 3.0 * t[None, :] - 2.0 * t[:, None] + 0.5, atol=1e-13)
    np.testing.assert_allclose(WS.resample(f, 12), f, atol=1e-13)  # same grid: unchanged


def test_holdout_split_is_seeded_and_disjoint():
    tr, ho = WS.split_holdout(385 * 10 + 4, 0.1, 3)
    assert len(ho) == round(0.1 * 3854) and len(tr) + len(ho) == 3854
    assert not set(tr) & set(ho)
    tr2, ho2 = WS.split_holdout(3854, 0.1, 3)
    np.testing.assert_array_equal(ho, ho2)
    assert not np.array_equal(ho, WS.split_holdout(3854, 0.1, 4)[1])


def test_sweep_subset_is_stratified_and_in_the_trained_range():
    idx, re, nn, sides = WS.sweep_subset(per_side=3)
    assert len(idx) == 12
    for k, side in enumerate((65, 129, 257, 513)):
        sel = idx[3 * k:3 * k + 3]
        assert all(sides[i] == side and re[i] <= 1000.0 for i in sel)
        # the first ones of that side in draw order
        first = [i for i in range(512) if sides[i] == side and re[i] <= 1000.0][:3]
        assert list(sel) == first


def test_shipped_network_record_matches_its_weights():
    with open(os.path.join(WS.WEIGHTS_DIR, "warmstart_cavity_R128.json")) as fp:
        rec = json.load(fp)
    w = np.load(os.path.join(WS.WEIGHTS_DIR, "warmstart_cavity_R128.npy"))
    assert w.dtype == np.float32 and w.size == 1755619
    assert np.isfinite(w).all()
    sweep = rec["sweep"]
    idx, re, nn, sides = WS.sweep_subset(per_side=10)
    assert all(sides[i] == s for i, s in zip(sweep["indices"], sweep["sides"]))
    assert set(sweep["indices"]) <= set(int(i) for i in idx)


# ------------------------------------------------------------ benchmark bookkeeping

def test_finite_json_and_whole_job_throughput():
    line = bench.finite_json({"a": float("nan"), "b": [1.0, float("inf")], "c": {"d": 2.5}, "e": "x"})
    assert line == {"a": None, "b": [1.0, None], "c": {"d": 2.5}, "e": "x"}
    json.dumps(line, allow_nan=False)
    assert bench.job_mlups(4096 * 4096, 20, 1, 0.0056) == pytest.approx(4096 * 4096 * 20 / 0.0056 / 1e6)
    assert bench.job_mlups(100, 10, 4, 2.0) == pytest.approx(4 * 100 * 10 / 2.0 / 1e6)
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_measured_peak_and_traffic_source_check(tmp_path, monkeypatch):
    peak, kind = bench.measured_peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fp:
            assert peak == float(json.load(fp)["hbm_gbs"]) and kind == "measured"
    else:
        assert kind == "fallback"
    # the traffic figure is kept only for the kernel source it was taken on
    src = tmp_path / "k.cu"
    src.write_bytes(b"kernel v1")
    import hashlib
    digest = hashlib.sha256(b"kernel v1").hexdigest()[:16]
    tf = tmp_path / "t.json"
    tf.write_text(json.dumps({"source_sha256_16": digest, "dram_bytes_per_launch": 1234}))
    monkeypatch.setattr(bench, "STEP_SOURCE", str(src))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tf))
    assert bench.ncu_traffic_per_launch() == 1234
    src.write_bytes(b"kernel v2")
    assert bench.ncu_traffic_per_launch() is None
