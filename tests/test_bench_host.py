"""The host-side parts of bench.py (no GPU): Sec. 8.1's error rate, recall,
precision and F-value of a mask against ground truth on hand-counted cases, the
summary of the min cut's per-frame statistics, and the reference arm's JSON line."""
import math
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_confusion_counts_by_hand():
    gt = np.array([[1, 1, 0, 0],
                   [1, 1, 0, 0]], np.uint8)
    m = np.array([[1, 0, 1, 0],
                  [1, 1, 0, 0]], np.uint8)
    tp, tn, fp, fn = bench.confusion(m, gt)
    assert (tp, tn, fp, fn) == (3, 3, 1, 1)


def test_measures_by_hand():
    # TP 3, TN 3, FP 1, FN 1: error 2/8, recall 3/4, precision 3/4, F 3/4
    a = bench.seg_accuracy([3, 3, 1, 1])
    assert a["error"] == pytest.approx(0.25)
    assert a["recall"] == pytest.approx(0.75)
    assert a["precision"] == pytest.approx(0.75)
    assert a["f_value"] == pytest.approx(0.75)
    # recall 1/2, precision 1: F = 2 * 0.5 / 1.5
    a = bench.seg_accuracy([1, 6, 0, 1])
    assert a["f_value"] == pytest.approx(2.0 / 3.0)
    assert a["error"] == pytest.approx(1.0 / 8.0)


def test_perfect_and_degenerate_masks():
    gt = np.zeros((5, 7), np.uint8)
    gt[1:3, 2:6] = 1
    a = bench.seg_accuracy(bench.confusion(gt, gt))
    assert a == {"error": 0.0, "recall": 1.0, "precision": 1.0, "f_value": 1.0}
    # an empty mask: nothing labelled object, so precision (and F) are undefined
    a = bench.seg_accuracy(bench.confusion(np.zeros_like(gt), gt))
    assert a["recall"] == 0.0 and a["precision"] is None and a["f_value"] is None
    assert a["error"] == pytest.approx(8 / 35)
    # the complement: every pixel wrong
    a = bench.seg_accuracy(bench.confusion(1 - gt, gt))
    assert a["error"] == 1.0 and a["recall"] == 0.0 and a["precision"] == 0.0 and a["f_value"] is None


def test_counts_sum_over_frames_and_shapes_checked():
    rng = np.random.default_rng(7)
    gts = rng.integers(0, 2, (4, 6, 9)).astype(np.uint8)
    ms = rng.integers(0, 2, (4, 6, 9)).astype(np.uint8)
    tot = sum(bench.confusion(m, g) for m, g in zip(ms, gts))
    assert tot.sum() == gts.size
    assert (tot == bench.confusion(ms, gts)).all()
    a = bench.seg_accuracy(tot)
    assert math.isclose(a["error"], float(np.mean(ms != gts)))
    with pytest.raises(ValueError):
        bench.confusion(ms[0], gts[0, :5])


def test_clip_with_ground_truth_has_the_same_frames():
    f1 = bench.make_clip(3)
    f2, gt = bench.make_clip(3, with_gt=True)
    assert f1.shape == f2.shape == (3, 480, 640, 3) and (f1 == f2).all()
    assert gt.shape == (3, 480, 640) and gt.dtype == np.uint8 and set(np.unique(gt)) <= {0, 1}


def test_mincut_profile_summary():
    # (cycles, relabels, rounds, init, relabel, discharge, final) in 0.1 us
    stats = [(1, 1, 3, 3, 90, 250, 150), (1, 1, 3, 3, 92, 248, 146), (2, 2, 6, 3, 290, 600, 157),
             (4, 4, 12, 3, 1100, 1900, 200)]
    p = bench.mincut_profile(stats)
    assert p["frames"] == 4
    assert p["by_cycles"]["<=1"]["frames"] == 2 and p["by_cycles"]["<=1"]["mean_us"] == pytest.approx(49.1)
    assert p["by_cycles"]["2"]["mean_us"] == pytest.approx(105.0)
    assert p["by_cycles"][">=3"]["mean_us"] == pytest.approx(320.3)
    total = 49.3 + 48.9 + 105.0 + 320.3
    assert p["by_cycles"][">=3"]["share_of_time"] == pytest.approx(320.3 / total)
    assert sum(g["share_of_time"] for g in p["by_cycles"].values()) == pytest.approx(1.0)
    assert p["phase_us_mean"]["discharge"] == pytest.approx((250 + 248 + 600 + 1900) / 40)
    assert bench.mincut_profile([]) == {"frames": 0, "by_cycles": {}, "phase_us_mean": {},
                                        "of": "device-timer spans inside the cut kernel, profiled frames"}
    # the binding's format: a list of 7-tuples, as many as frames were recorded
    assert bench.mincut_profile([(0, 1, 1, 2, 10, 0, 100)])["by_cycles"]["<=1"]["frames"] == 1


def test_spread_frames_cover_the_clip():
    assert bench.spread_frames(1) == [0]
    assert bench.spread_frames(4) == [0, 75, 150, 225]
    idx = bench.spread_frames(20)
    assert len(set(idx)) == 20 and max(idx) >= 280 and any(200 <= f < 250 for f in idx)
    assert bench.spread_frames(300) == list(range(300))


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the oracle on the host cores, rank 0) prints one JSON
    line with the same metric and config as the CUDA arm, impl = reference, and an e2e
    object with no host-device bytes."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0"))
    assert r.returncode == 0, r.stderr[-800:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "frames/s"
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["config"] == bench.bench_config()
    assert d["e2e"] == {"value": d["value"], "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
