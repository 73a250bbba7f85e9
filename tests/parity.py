"""Comparison rules between the CUDA path and the FP64 oracle.

- mask: bit-exact;
- mean: every evaluable pixel within TOL_DEG (1e-3 degree) of the oracle;
- median: at least 99.9% of evaluable pixels within TOL_DEG; every other
  pixel within TOL_DEG of the normal obtained by moving the oracle's n_z by
  the largest gap between sorted candidates next to the median (a near-tie
  decided the other way in FP32).
"""
import numpy as np

import oracle

TOL_DEG = 1e-3


def median_gap_bound(cands, nprime, idx):
    """Angle (deg) that one near-tie swap around the median can cause, per pixel of idx."""
    out = np.zeros(len(idx[0]))
    for k, (y, x) in enumerate(zip(*idx)):
        c = np.sort(cands[:, y, x][np.isfinite(cands[:, y, x])])
        m = len(c)
        if m < 2:
            continue
        lo, hi = (m - 1) // 2, m // 2
        ks = [i for i in range(lo - 1, hi + 1) if 0 <= i < m - 1]
        gap = max(c[i + 1] - c[i] for i in ks)
        n0 = nprime[:, y, x]
        worst = 0.0
        for s in (-gap, gap):
            n1 = n0.copy()
            n1[2] += s
            worst = max(worst, float(oracle.angle_deg(n0[:, None], n1[:, None])[0]))
        out[k] = worst
    return out


def compare(gpu_n, gpu_m, img, cam, *, grad, phi, disparity=False, baseline=1.0, disp_scale=1.0 / 16,
            tol=TOL_DEG, weights=None):
    """Raises AssertionError with details when the GPU result breaks the rules; returns stats."""
    ref_n, ref_m, cands, npr = oracle.normals(img, cam["fx"], cam["fy"], cam["u0"], cam["v0"], grad=grad, phi=phi,
                                              disparity=disparity, baseline=baseline, disp_scale=disp_scale,
                                              diagnostics=True, weights=weights)
    gpu_n = np.asarray(gpu_n, np.float64)
    gpu_m = np.asarray(gpu_m)
    bad_mask = gpu_m != ref_m
    assert not bad_mask.any(), f"mask differs at {np.argwhere(bad_mask)[:5].tolist()} ({bad_mask.sum()} px)"
    v = ref_m == 1
    assert (gpu_n[:, ~v] == 0).all(), "non-evaluable pixels must be (0,0,0)"
    ang = oracle.angle_deg(gpu_n, ref_n)
    ang = np.where(v, np.nan_to_num(ang, nan=180.0), 0.0)
    over = v & (ang > tol)
    stats = {"pixels": int(v.sum()), "max_deg": float(ang.max()) if v.any() else 0.0, "over": int(over.sum())}
    if phi == "mean":
        assert not over.any(), (f"{over.sum()} of {v.sum()} px over {tol} deg, max {ang.max():.3g} deg at "
                                f"{np.unravel_index(np.argmax(ang), ang.shape)}")
    else:
        assert over.sum() <= 0.001 * max(1, v.sum()), f"{over.sum()} of {v.sum()} px over {tol} deg"
        if over.any():
            idx = np.nonzero(over)
            bound = median_gap_bound(cands, npr, idx)
            assert (ang[idx] <= bound + tol).all(), "median pixels beyond the adjacent-candidate gap"
    norms = np.sqrt((gpu_n[:, v] ** 2).sum(0))
    assert np.abs(norms - 1).max(initial=0) < 1e-5
    return stats
