"""Pins of the oracle's 5x5 gradient filters (reading R15: Fig. 2 compares filter types and sizes).

A 5x5 filter is separable: a derivative profile (d1 at offsets +-1, d2 at +-2) along its axis times
a symmetric smoothing profile (s0, s1, s2) across it, divided by 2 (d1 + 2 d2) (s0 + 2 s1 + 2 s2) so
that it returns the derivative of an affine image.  The pins fix each part by a property the
mathematics decides, not by retyping the oracle's sums:

- the symmetric 3x3 filters are the members with d2 = s2 = 0;
- planes come out exact for any profiles (1/Z is affine on a plane);
- on polynomial inverse-depth images the filters' values have closed forms: the fourth-order
  central difference (FD5) is exact up to degree 4, Sobel5 and Prewitt5 carry the truncation
  terms (5/12) p''' and (17/30) p''', and the smoothing profile's second moment shows in the
  gradient of u v^2;
- the taps a filter needs (and only those) decide which pixels are evaluable;
- transposing the image swaps the normal's x and y (the vertical filter is the transpose);
- the symmetric members converge at second order on a sphere.
"""
import numpy as np
import pytest

import oracle
from tests.geometry import plane_depth, sphere_depth, tilted_normal
from tests.test_oracle_weighted import _noisy

CAM = dict(fx=48.12, fy=46.37, u0=31.13, v0=24.79)
NAMED5 = {"fd5": (8.0, -1.0, 1.0, 0.0, 0.0), "sobel5": (2.0, 1.0, 6.0, 4.0, 1.0),
          "prewitt5": (1.0, 2.0, 1.0, 1.0, 1.0)}
# symmetric 3x3 members: row weights (w0 w1 w0) -> d = (1, 0), s = (w1, w0, 0)
NAMED3 = {"fd": (1.0, 0.0, 1.0, 0.0, 0.0), "sobel": (1.0, 0.0, 2.0, 1.0, 0.0),
          "scharr": (1.0, 0.0, 10.0, 3.0, 0.0), "prewitt": (1.0, 0.0, 1.0, 1.0, 0.0)}


def _nprime(img, grad, weights=None, lib=None, cam=None):
    cam = cam or dict(fx=1.0, fy=1.0, u0=0.0, v0=0.0)
    _, m, _, npr = oracle.normals(img, **cam, grad=grad, weights=weights, diagnostics=True, lib=lib)
    return npr, m


def _poly_image(H, W, p, axis):
    """Depth image whose inverse is p(u) (axis 1) or p(v) (axis 0), p a numpy polynomial."""
    uu, vv = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    return 1.0 / p(uu if axis == 1 else vv)


def _mask_pattern5(grad, w=None, lib=None):
    """Mask of the centre pixel of a 5x5 image with one hole, for each hole position."""
    out = np.zeros((5, 5), np.uint8)
    for a in range(5):
        for b in range(5):
            if (a, b) == (2, 2):
                continue
            img = np.full((9, 9), 2.0, np.float64)
            img[2:7, 2:7] += np.arange(25, dtype=np.float64).reshape(5, 5) * 0.01
            img[2 + a, 2 + b] = 0.0
            _, m = oracle.normals(img, 3.0, 3.0, 4.0, 4.0, grad=grad, weights=w, lib=lib)
            out[a, b] = m[4, 4]
    return out


def check_sep5(lib=None):
    """Names of the failed 5x5 pins (empty when all hold)."""
    fails = []
    d = _noisy()
    # members: the symmetric 3x3 filters, and the named 5x5 ones at the profiles of reading R15
    for name, w in list(NAMED3.items()) + list(NAMED5.items()):
        for phi in ("mean", "median"):
            a, ma = oracle.normals(d, **CAM, grad=name, phi=phi, lib=lib)
            b, mb = oracle.normals(d, **CAM, grad="sep5", weights=w, phi=phi, lib=lib)
            if not ((ma == mb).all() and np.nanmax(oracle.angle_deg(a, b)[ma == 1]) < 1e-9):
                fails.append(f"member {name} {phi}")
    # exact planes for arbitrary profiles
    Z = plane_depth(24, 32, CAM, tilted_normal(33, 140), [0.2, -0.1, 3.5])
    for w in ((1.0, 0.3, 2.0, 0.5, 0.1), (0.0, 1.0, 1.0, 0.0, 0.0), (3.0, -1.0, 1.0, 2.0, -0.5)):
        n, m = oracle.normals(Z, **CAM, grad="sep5", weights=w, lib=lib)
        inner = m == 1
        if not (inner.sum() > 300 and np.nanmax(oracle.angle_deg(n, tilted_normal(33, 140)[:, None, None]
                                                                 * np.ones((1, 24, 32)))[inner]) < 1e-9):
            fails.append(f"plane {w}")
    # closed forms on polynomial inverse depth (fx = fy = 1, so n'x = G_u and n'y = G_v)
    p = np.polynomial.Polynomial([0.5, 0.01, 1e-4, 1e-6, 1e-8])
    dp, d3p = p.deriv(1), p.deriv(3)
    H, W = 12, 40
    for axis, comp in ((1, 0), (0, 1)):
        img = _poly_image(H, W, p, axis) if axis == 1 else _poly_image(W, H, p, axis)
        coord = np.arange(img.shape[axis], dtype=np.float64)
        for grad, extra in (("fd5", 0.0), ("sobel5", 5.0 / 12.0), ("prewitt5", 17.0 / 30.0)):
            npr, m = _nprime(img, grad, lib=lib)
            want = dp(coord) + extra * d3p(coord)
            got = npr[comp]
            want = want[None, :] * np.ones((img.shape[0], 1)) if axis == 1 else want[:, None] * np.ones((1, img.shape[1]))
            sel = m == 1
            if not (sel.sum() > 100 and np.abs(got[sel] - want[sel]).max() < 1e-10 * np.abs(want[sel]).max()):
                fails.append(f"closed form {grad} axis {axis}")
    # smoothing: for 1/Z = 1 + 1e-3 u v^2, G_u = 1e-3 (v^2 + M2), M2 = sum_a s_|a| a^2 / sum_a s_|a|
    uu, vv = np.meshgrid(np.arange(30.0), np.arange(30.0))
    img = 1.0 / (1.0 + 1e-3 * uu * vv * vv)
    for grad, m2 in (("fd5", 0.0), ("sobel5", 1.0), ("prewitt5", 2.0)):
        npr, m = _nprime(img, grad, lib=lib)
        want = 1e-3 * (vv * vv + m2)
        sel = m == 1
        if not (sel.sum() > 100 and np.abs(npr[0][sel] - want[sel]).max() < 1e-10 * np.abs(want[sel]).max()):
            fails.append(f"smoothing moment {grad}")
    # the taps each filter needs
    cross = np.zeros((5, 5), np.uint8) + 1
    cross[2, :] = 0
    cross[:, 2] = 0
    if not np.array_equal(_mask_pattern5("fd5", lib=lib), cross):
        fails.append("taps fd5")
    if not np.array_equal(_mask_pattern5("sobel5", lib=lib), np.zeros((5, 5), np.uint8)):
        fails.append("taps sobel5")
    # d = (1, 0), s = (1, 0, 1): rows -2, 0, 2 at columns +-1 (horizontal), transposed (vertical)
    want = np.ones((5, 5), np.uint8)
    want[2, 2] = 0  # (the centre is not probed)
    for a in (-2, 0, 2):
        for b in (-1, 1):
            want[2 + a, 2 + b] = 0
            want[2 + b, 2 + a] = 0
    if not np.array_equal(_mask_pattern5("sep5", (1.0, 0.0, 1.0, 0.0, 1.0), lib), want):
        fails.append("taps (1 0 | 1 0 1)")
    # Sec. III special case (reading R6): every neighbour at the centre's depth gives [0, 0, -1] even
    # though a 5x5 filter sees the depth change in its outer taps
    img = np.full((9, 9), 2.0)
    img[:, 6:] = 2.5
    img[6:, :] = 2.25
    for grad in ("fd5", "sobel5"):
        for phi in ("mean", "median"):
            n, m = oracle.normals(img, 3.0, 3.0, 4.0, 4.0, grad=grad, phi=phi, lib=lib)
            if not (m[4, 4] == 1 and np.array_equal(n[:, 4, 4], [0.0, 0.0, -1.0])):
                fails.append(f"no-candidate special case {grad} {phi}")
    # (the window is what it claims: no neighbour of the centre gives a candidate, while FD5's outer
    # taps (4, 2) and (4, 6) differ)
    _, _, c1, npr = oracle.normals(img, 1.0, 1.0, 4.0, 4.0, grad="fd", diagnostics=True, lib=lib)
    if np.isfinite(c1[:, 4, 4]).any() or npr[:, 4, 4].any() or img[4, 2] == img[4, 6]:
        fails.append("no-candidate window")
    # transpose: x and y of the normal swap
    w = (1.0, 0.4, 3.0, 1.0, 0.2)
    a, ma = oracle.normals(d, **CAM, grad="sep5", weights=w, lib=lib)
    b, mb = oracle.normals(np.ascontiguousarray(d.T), CAM["fy"], CAM["fx"], CAM["v0"], CAM["u0"], grad="sep5",
                           weights=w, lib=lib)
    b = np.stack([b[1].T, b[0].T, b[2].T])
    if not ((ma == mb.T).all() and np.nanmax(oracle.angle_deg(a, b)[ma == 1]) < 1e-8):
        fails.append("transpose")
    return fails


def test_sep5_pins_hold():
    assert check_sep5() == []


@pytest.mark.parametrize("grad", ["fd5", "sobel5"])
def test_5x5_filters_converge_at_second_order_on_a_sphere(grad):
    # the candidates and Phi keep the 8-connected neighbourhood, so the order stays 2
    errs = []
    for f in (100.0, 200.0, 400.0):
        S = int(0.6 * f)
        cam = dict(fx=f, fy=f, u0=(S - 1) / 2, v0=(S - 1) / 2)
        Z, gt = sphere_depth(S, S, cam, [0.1, -0.05, 3.0], 1.0)
        n, m = oracle.normals(Z, **cam, grad=grad, phi="mean")
        sel = (m == 1) & (-gt[2] > np.cos(np.deg2rad(50)))
        errs.append(np.median(oracle.angle_deg(n, gt)[sel]))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 <= o <= 2.3 for o in orders), orders


def test_sep5_weights_are_validated():
    img = np.full((6, 6), 2.0, np.float32)
    # (the derivative sum d1 + 2 d2 and the smoothing sum s0 + 2 s1 + 2 s2 must not vanish)
    for w in ((0.0, 0.0, 1.0, 0.0, 0.0), (1.0, 0.0, 0.0, 0.0, 0.0), (2.0, -1.0, 1.0, 0.0, 0.0),
              (1.0, 0.0, 1.0, -0.5, 0.0), (np.nan, 1.0, 1.0, 0.0, 0.0), None):
        with pytest.raises(ValueError):
            oracle.normals(img, 3.0, 3.0, 2.5, 2.5, grad="sep5", weights=w)
