"""The accuracy criterion of bench.py (an estimate is an outlier when it is
off by at least 3 pixels and by at least 5 %), on hand-made maps."""
import numpy as np

import bench


def test_outlier_criterion():
    gt = np.array([[10, 10, 100, 100, 0, 40]])
    # exact; 2 off (absolute below 3); 4 off at 100 (relative 4 %); 6 off at
    # 100 (both); 3 off at 0 (relative infinite); invalid
    d = np.array([[10, 12, 104, 106, 3, -1]])
    r = bench.kitti_outliers(d, gt)
    assert r["density"] == 5 / 6
    assert r["outliers_of_valid"] == 2 / 5
    assert r["outliers_all"] == 3 / 6


def test_perfect_and_empty_maps():
    gt = np.arange(12).reshape(3, 4)
    assert bench.kitti_outliers(gt, gt) == {"density": 1.0, "outliers_of_valid": 0.0, "outliers_all": 0.0}
    r = bench.kitti_outliers(np.full_like(gt, -1), gt)
    assert r["density"] == 0.0 and r["outliers_of_valid"] == 0.0 and r["outliers_all"] == 1.0
