"""The bench's accuracy metrics (Sec. IV-A, Eq. ea_ep): e_A is the mean angle and e_P(phi) the share of
angles at most phi, checked on vector pairs with known angles."""
import numpy as np

import bench


def test_ea_ep_on_known_angles():
    ang = np.array([0.0, 5.0, 9.0, 15.0, 25.0, 40.0])  # (none on a boundary)
    t = np.radians(ang)
    gt = np.stack([np.zeros_like(t), np.zeros_like(t), np.ones_like(t)])
    n = np.stack([np.sin(t), np.zeros_like(t), np.cos(t)]) * 3.0  # the metric ignores length
    r = bench.ea_ep(n, gt, np.ones(6, bool))
    assert r["m"] == 6
    assert abs(r["e_A_deg"] - ang.mean()) < 1e-3
    assert r["e_P_10"] == round(3 / 6, 4) and r["e_P_20"] == round(4 / 6, 4) and r["e_P_30"] == round(5 / 6, 4)


def test_ea_ep_selects_pixels():
    gt = np.zeros((3, 2, 2))
    gt[2] = 1
    n = gt.copy()
    n[:, 0, 0] = [1, 0, 0]  # 90 degrees off, but not selected
    sel = np.array([[False, True], [True, True]])
    r = bench.ea_ep(n, gt, sel)
    assert r["m"] == 3 and r["e_A_deg"] == 0.0 and r["e_P_10"] == 1.0
