"""Pins of the oracle's fused outputs: the back-projected point cloud (Sec. III, Eq. intrinsic
matrix; disparity through Eq. z_d) and the octahedral normal encoding (Cigolle et al., JCGT 2014).

The points are checked against values derived by hand, against ray-cast geometry (each point of an
analytic plane or sphere is the ray through its pixel times the hit distance, built without the
back-projection formula), against the disparity-to-depth relation and the hole rule.  The
octahedral map is checked on the coordinate axes (values fixed by its definition), on round trips,
and on its quantisation error.
"""
import numpy as np
import pytest

import oracle
from tests.geometry import plane_depth, rays, sphere_depth, tilted_normal

CAM = dict(fx=48.12, fy=46.37, u0=31.13, v0=24.79)


def check_points(lib=None):
    """Names of the failed point pins (empty when all hold)."""
    fails = []
    # hand-derived: Z = 2, fx = 2, fy = 4, u0 = v0 = 1: X = Z (u - 1)/2 = u - 1, Y = Z (v - 1)/4 = (v - 1)/2
    img = np.full((3, 3), 2.0, np.float32)
    P = oracle.points(img, 2.0, 4.0, 1.0, 1.0, lib=lib)
    uu, vv = np.meshgrid(np.arange(3.0), np.arange(3.0))
    if not (np.array_equal(P[0], uu - 1) and np.array_equal(P[1], (vv - 1) / 2) and (P[2] == 2).all()):
        fails.append("hand")
    # an analytic plane: the points are the ray-cast hits and satisfy the plane equation
    n = tilted_normal(35, 60)
    P0 = np.array([0.3, -0.2, 4.0])
    Z = plane_depth(40, 56, CAM, n, P0)
    P = oracle.points(Z, CAM["fx"], CAM["fy"], CAM["u0"], CAM["v0"], lib=lib)
    hits = rays(40, 56, CAM["fx"], CAM["fy"], CAM["u0"], CAM["v0"]) * Z
    if not (np.abs(P - hits).max() < 1e-12 * np.abs(hits).max() and
            np.abs(np.tensordot(n, P, 1) - n @ P0).max() < 1e-12):
        fails.append("plane")
    # an analytic sphere: every hit is at distance r from the centre
    C, r = np.array([0.4, 0.1, 5.0]), 1.5
    Z, _ = sphere_depth(40, 56, CAM, C, r)
    Zs = np.where(Z > 0, Z, 0.0)
    P = oracle.points(Zs, CAM["fx"], CAM["fy"], CAM["u0"], CAM["v0"], lib=lib)
    hit = Zs > 0
    dist = np.sqrt(((P - C[:, None, None]) ** 2).sum(0))
    if not (hit.sum() > 100 and np.abs(dist[hit] - r).max() < 1e-12 and (P[:, ~hit] == 0).all()):
        fails.append("sphere")
    # disparity: the same points as the depth image Z = f t_c / (raw * scale)
    rng = np.random.default_rng(3)
    raw = rng.integers(16, 1536, size=(9, 11)).astype(np.uint16)
    raw[4, 5] = 0
    f, tc, sc = 615.0, 0.1, 1.0 / 16
    Pd = oracle.points(raw, f, f, 5.0, 4.0, disparity=True, baseline=tc, disp_scale=sc, lib=lib)
    Zd = np.where(raw > 0, f * tc / np.maximum(raw * sc, 1e-300), 0.0)
    Pz = oracle.points(Zd, f, f, 5.0, 4.0, lib=lib)
    if not (np.abs(Pd - Pz).max() < 1e-12 * np.abs(Pz).max() and (Pd[:, 4, 5] == 0).all()):
        fails.append("disparity")
    # holes (reading R1) give (0, 0, 0); valid samples give Z itself
    img = np.array([[1.0, np.nan, -1.0], [0.0, np.inf, 2.0 ** 17], [2.0 ** -17, 3.0, 2.0 ** 16]], np.float32)
    P = oracle.points(img, 10.0, 10.0, 1.0, 1.0, lib=lib)
    valid = np.array([[1, 0, 0], [0, 0, 0], [0, 1, 1]], bool)
    if not ((P[:, ~valid] == 0).all() and np.array_equal(P[2][valid], img[valid].astype(np.float64))):
        fails.append("holes")
    return fails


def test_point_pins_hold():
    assert check_points() == []


def test_points_are_perpendicular_to_the_estimated_normal_on_a_plane():
    # two oracle functions from the same Eq. (intrinsic matrix): on a plane every point
    # difference lies in the plane, so it is perpendicular to the estimated normal
    n = tilted_normal(40, 200)
    Z = plane_depth(32, 40, CAM, n, [0.1, 0.2, 3.0])
    P = oracle.points(Z, CAM["fx"], CAM["fy"], CAM["u0"], CAM["v0"])
    N, m = oracle.normals(Z, CAM["fx"], CAM["fy"], CAM["u0"], CAM["v0"])
    inner = m[1:-1, 1:-1] == 1
    for dP in (P[:, 1:-1, 2:] - P[:, 1:-1, 1:-1], P[:, 2:, 1:-1] - P[:, 1:-1, 1:-1]):
        dot = (N[:, 1:-1, 1:-1] * dP).sum(0) / np.sqrt((dP * dP).sum(0))
        assert np.abs(dot[inner]).max() < 1e-9


AXES = {(1, 0, 0): (1, 0), (-1, 0, 0): (-1, 0), (0, 1, 0): (0, 1), (0, -1, 0): (0, -1), (0, 0, 1): (0, 0),
        (0, 0, -1): (1, 1)}


def check_oct(encode=oracle.oct_encode, decode=oracle.oct_decode):
    """Names of the failed octahedral pins for an encode/decode pair."""
    fails = []
    # the axes: the upper pole maps to the centre, the lower pole (folded, sgn 0 = +1) to the corner (1, 1)
    for v, p in AXES.items():
        if not np.array_equal(encode(np.array(v, float)[:, None])[:, 0], np.array(p, float)):
            fails.append(f"axis {v}")
    rng = np.random.default_rng(5)
    v = rng.normal(size=(3, 20000))
    v /= np.sqrt((v * v).sum(0))
    p = encode(v)
    # the upper hemisphere fills the diamond |px| + |py| <= 1, the lower one the corners outside it
    l1 = np.abs(p[0]) + np.abs(p[1])
    if not ((l1[v[2] > 0] <= 1 + 1e-12).all() and (l1[v[2] < 0] >= 1 - 1e-12).all() and (np.abs(p) <= 1).all()):
        fails.append("square")
    if not oracle.angle_deg(v, decode(p)).max() < 1e-9:
        fails.append("round trip")
    return fails


def test_octahedral_pins_hold():
    assert check_oct() == []


def test_octahedral_pins_catch_plausible_mistakes():
    def no_fold(n):
        n = np.asarray(n, float)
        s = np.abs(n).sum(0)
        return np.stack([n[0] / s, n[1] / s])

    def swapped_fold(n):
        p = oracle.oct_encode(n)
        low = np.asarray(n, float)[2] < 0
        return np.where(low, p[::-1], p)

    def plain_sign(n):  # sgn(0) = 0 leaves the lower pole at the centre
        n = np.asarray(n, float)
        s = np.abs(n).sum(0)
        px, py = n[0] / s, n[1] / s
        low = n[2] < 0
        return np.stack([np.where(low, (1 - np.abs(py)) * np.sign(px), px),
                         np.where(low, (1 - np.abs(px)) * np.sign(py), py)])

    for bad in (no_fold, swapped_fold, plain_sign):
        assert check_oct(encode=bad), f"{bad.__name__} passes every octahedral pin"


def test_octahedral_16_bit_quantisation_error():
    # 16-bit codes: round-to-nearest of p * 32767; over a million random directions the decoded
    # direction stays within 0.005 degrees (the grid step 1/32767 stretched by the map)
    rng = np.random.default_rng(7)
    v = rng.normal(size=(3, 1000000))
    v /= np.sqrt((v * v).sum(0))
    q = oracle.oct_quantize(oracle.oct_encode(v))
    assert q.dtype == np.int16
    assert oracle.angle_deg(v, oracle.oct_decode(q)).max() < 0.005
