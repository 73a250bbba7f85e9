"""PlanePCA surface normals, FP64 -- TEST INFRASTRUCTURE ONLY (part of the oracle package).

The comparison estimator of Sec. II, item 2 (Eq. planepca): for each pixel i, the points
Q_i^+ = [p_i, q_i1 .. q_ik] of its neighbourhood (Eq. intrinsic matrix back-projection) have their
empirical mean removed, and the normal is the principal component of smallest covariance, i.e. the
eigenvector of the smallest eigenvalue of the scatter matrix sum_j (q_j - q_mean)(q_j - q_mean)^T.
A library symmetric eigensolver (numpy.linalg.eigh, LAPACK) is the step that finds it.

Readings where the paper is silent (reading R16):
- the neighbourhood is the 8-connected one, k = 8 (the paper's 3F2N uses the same);
- a pixel is evaluable iff it and all 8 neighbours are inside the image and valid (the hole rule
  of the 3F2N oracle); others get (0, 0, 0) and mask 0;
- the eigenvector's sign is chosen so that the normal faces the camera, n . p_i < 0 (as 3F2N's
  output, reading R7); if n . p_i is exactly 0, so that n_z < 0, then n_y < 0, then n_x < 0.
"""
from __future__ import annotations

import numpy as np

from . import points as _points

OFFSETS = [(dv, du) for dv in (-1, 0, 1) for du in (-1, 0, 1)]  # the centre and its 8 neighbours


def _valid(img, disparity):
    img = np.asarray(img)
    if disparity and img.dtype == np.uint16:
        return img > 0
    v = img.astype(np.float64)
    return np.isfinite(v) & (v >= 2.0 ** -16) & (v <= 2.0 ** 16)


def scatter(img, fx, fy, u0, v0, *, disparity=False, baseline=1.0, disp_scale=1.0 / 16):
    """Per-pixel 3x3 scatter matrices (H, W, 3, 3) of the centred 9-point neighbourhoods, and the
    evaluable mask (H, W).  Eq. planepca: rows of Q_i^+ minus their mean."""
    P = _points(img, fx, fy, u0, v0, disparity=disparity, baseline=baseline, disp_scale=disp_scale)
    H, W = P.shape[1:]
    ok = _valid(img, disparity)
    pad = np.zeros((3, H + 2, W + 2))
    pad[:, 1:-1, 1:-1] = P
    okp = np.zeros((H + 2, W + 2), bool)
    okp[1:-1, 1:-1] = ok
    Q = np.stack([pad[:, 1 + dv:1 + dv + H, 1 + du:1 + du + W] for dv, du in OFFSETS])  # (9, 3, H, W)
    mask = np.all(np.stack([okp[1 + dv:1 + dv + H, 1 + du:1 + du + W] for dv, du in OFFSETS]), axis=0)
    D = Q - Q.mean(axis=0, keepdims=True)
    S = np.einsum("jahw,jbhw->hwab", D, D)
    return S, mask, P


def planepca(img, fx, fy, u0, v0, *, disparity=False, baseline=1.0, disp_scale=1.0 / 16, eig=False):
    """PlanePCA normals of one H x W image: ``(n, mask)`` with n (3, H, W) float64, mask (H, W) uint8;
    with ``eig=True`` also the scatter eigenvalues (H, W, 3), ascending."""
    S, mask, P = scatter(img, fx, fy, u0, v0, disparity=disparity, baseline=baseline, disp_scale=disp_scale)
    H, W = mask.shape
    n = np.zeros((3, H, W))
    lam = np.zeros((H, W, 3))
    if mask.any():
        w, V = np.linalg.eigh(S[mask])  # ascending eigenvalues; columns are eigenvectors
        v = V[:, :, 0]  # (m, 3): the smallest eigenvalue's
        p = P[:, mask].T
        d = (v * p).sum(1)
        # face the camera: n . p_i < 0; ties by n_z, n_y, n_x < 0
        key = np.where(d != 0, d, np.where(v[:, 2] != 0, v[:, 2], np.where(v[:, 1] != 0, v[:, 1], v[:, 0])))
        v = np.where((key > 0)[:, None], -v, v)
        n[:, mask] = v.T
        lam[mask] = w
    out = (n, mask.astype(np.uint8))
    return out + (lam,) if eig else out
