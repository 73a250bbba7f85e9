"""Exact FP64 test geometry: depth images of analytic planes and spheres.

Input construction for the oracle pins only (ray casting through a pinhole
camera); nothing here estimates normals.
"""
import numpy as np


def rays(H, W, fx, fy, u0, v0):
    uu, vv = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    return np.stack([(uu - u0) / fx, (vv - v0) / fy, np.ones_like(uu)])


def plane_depth(H, W, cam, normal, point):
    """Depth Z(u, v) of the plane through `point` with unit `normal` (facing the camera)."""
    d = rays(H, W, cam["fx"], cam["fy"], cam["u0"], cam["v0"])
    n = np.asarray(normal, np.float64)
    P = np.asarray(point, np.float64)
    t = (n @ P) / np.tensordot(n, d, 1)
    return t


def tilted_normal(tilt_deg, azimuth_deg):
    th, ph = np.deg2rad(tilt_deg), np.deg2rad(azimuth_deg)
    return np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), -np.cos(th)])


def sphere_depth(H, W, cam, centre, radius):
    """Depth of the visible sphere surface (0 where the ray misses) and its unit normal."""
    d = rays(H, W, cam["fx"], cam["fy"], cam["u0"], cam["v0"])
    C = np.asarray(centre, np.float64)[:, None, None]
    a = (d * d).sum(0)
    b = -2 * (d * C).sum(0)
    c = (C * C).sum() - radius * radius
    disc = b * b - 4 * a * c
    t = np.where(disc >= 0, (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a), 0.0)
    n = (t * d - C) / radius
    return t, n


def backproject(Z, cam):
    """Camera-frame points (3, H, W) of a depth image, Sec. III Eq. (intrinsic matrix)."""
    H, W = Z.shape
    return rays(H, W, cam["fx"], cam["fy"], cam["u0"], cam["v0"]) * Z
