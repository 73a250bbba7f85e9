"""Pins of the oracle's weighted gradient family: the 3x3 kernels of the paper's brute-force kernel
search (Sec. IV), row weights (w0 w1 w2) on the [-1 0 1] correlation and the transposed weights on
the vertical one.

The named filters must be members of the family (FD (0 1 0), Sobel (1 2 1), Scharr (3 10 3),
Prewitt (1 1 1)); planes must come out exact for any weights (1/Z is affine on a plane, so every
gradient filter measures its exact gradient); the taps an asymmetric weighting needs (and only
those) decide which pixels are evaluable, which fixes the weights' orientation; a half turn of the
image maps the weights to their reverse; symmetric weights converge at second order on a sphere.
"""
import numpy as np
import pytest

import oracle
import scenes
from tests.geometry import plane_depth, sphere_depth, tilted_normal

CAM = dict(fx=48.12, fy=46.37, u0=31.13, v0=24.79)
NAMED = {"fd": (0, 1, 0), "sobel": (1, 2, 1), "scharr": (3, 10, 3), "prewitt": (1, 1, 1)}


def _noisy(seed=31, H=40, W=56):
    r = scenes.Recipe(H=H, W=W, fx=CAM["fx"], fy=CAM["fy"], u0=CAM["u0"], v0=CAM["v0"], noise_k=0.0012,
                      hole_frac=0.03)
    return scenes.render(seed, r)


def _mask_pattern(w, lib=None):
    """Mask of the centre pixel of a 3x3 image with one hole, for each hole position."""
    out = np.zeros((3, 3), np.uint8)
    for a in range(3):
        for b in range(3):
            if (a, b) == (1, 1):
                continue
            img = np.full((5, 5), 2.0, np.float32)
            img[1:4, 1:4] += np.arange(9, dtype=np.float32).reshape(3, 3) * 0.01
            img[1 + a, 1 + b] = 0.0
            _, m = oracle.normals(img, 3.0, 3.0, 2.0, 2.0, grad="weighted", weights=w, lib=lib)
            out[a, b] = m[2, 2]
    return out


def check_weighted(lib=None):
    """Names of the failed pins of the weighted family (empty when all hold)."""
    fails = []
    d = _noisy()
    for name, w in NAMED.items():
        for phi in ("mean", "median"):
            a, ma = oracle.normals(d, **CAM, grad=name, phi=phi, lib=lib)
            b, mb = oracle.normals(d, **CAM, grad="weighted", weights=w, phi=phi, lib=lib)
            if not ((ma == mb).all() and np.nanmax(oracle.angle_deg(a, b)[ma == 1]) < 1e-9):
                fails.append(f"member {name} {phi}")
    # exact planes for arbitrary (also asymmetric) weights
    Z = plane_depth(24, 32, CAM, tilted_normal(33, 140), [0.2, -0.1, 3.5])
    for w in ((1.0, 0.5, 0.25), (0.0, 1.0, 3.0), (2.0, -1.0, 0.5)):
        n, m = oracle.normals(Z, **CAM, grad="weighted", weights=w, lib=lib)
        inner = m == 1
        if not (inner.sum() > 300 and np.nanmax(oracle.angle_deg(n, tilted_normal(33, 140)[:, None, None]
                                                                 * np.ones((1, 24, 32)))[inner]) < 1e-9):
            fails.append(f"plane {w}")
    # the taps (1 0 0) needs: the top row's outer two (horizontal) and the left column's (vertical)
    want = np.array([[0, 1, 0], [1, 0, 1], [0, 1, 1]], np.uint8)  # 0 where a hole there is fatal
    if not np.array_equal(_mask_pattern((1.0, 0.0, 0.0), lib), want):
        fails.append("taps (1 0 0)")
    # (0 1 0) needs the four axis neighbours only, as FD
    if not np.array_equal(_mask_pattern((0.0, 1.0, 0.0), lib), np.array([[1, 0, 1], [0, 0, 0], [1, 0, 1]])):
        fails.append("taps (0 1 0)")
    # half turn (u -> W-1-u, v -> H-1-v, with the principal point): x and y flip and both filters'
    # weights reverse (a one-axis mirror would reverse only one filter's weights)
    H, W = d.shape
    w = (1.0, 0.7, 0.2)
    a, ma = oracle.normals(d, **CAM, grad="weighted", weights=w[::-1], lib=lib)
    b, mb = oracle.normals(d[::-1, ::-1].copy(), CAM["fx"], CAM["fy"], W - 1 - CAM["u0"], H - 1 - CAM["v0"],
                           grad="weighted", weights=w, lib=lib)
    b = b[:, ::-1, ::-1] * np.array([-1, -1, 1.0])[:, None, None]
    if not ((ma == mb[::-1, ::-1]).all() and np.nanmax(oracle.angle_deg(a, b)[ma == 1]) < 1e-8):
        fails.append("half turn")
    return fails


def test_weighted_family_pins_hold():
    assert check_weighted() == []


def test_symmetric_weights_converge_at_second_order_on_a_sphere():
    # as the pins of the named filters: the median error on a sphere falls about 4x each time the
    # image scale doubles
    errs = []
    for f in (100.0, 200.0, 400.0):
        S = int(0.6 * f)
        cam = dict(fx=f, fy=f, u0=(S - 1) / 2, v0=(S - 1) / 2)
        Z, gt = sphere_depth(S, S, cam, [0.1, -0.05, 3.0], 1.0)
        n, m = oracle.normals(Z, **cam, grad="weighted", weights=(1.0, 3.0, 1.0), phi="mean")
        sel = (m == 1) & (-gt[2] > np.cos(np.deg2rad(50)))
        errs.append(np.median(oracle.angle_deg(n, gt)[sel]))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 <= o <= 2.3 for o in orders), orders


def test_weights_are_validated():
    img = np.full((4, 4), 2.0, np.float32)
    for w in ((0.0, 0.0, 0.0), (np.nan, 1.0, 1.0), None):
        with pytest.raises(ValueError):
            oracle.normals(img, 3.0, 3.0, 1.5, 1.5, grad="weighted", weights=w)
