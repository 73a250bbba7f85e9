"""Pins of the oracle's PlanePCA estimator (Sec. II item 2, Eq. planepca; reading R16).

The normal must be exact on planes (every centred point then lies in the plane) and face the
camera; on noisy windows it must minimise the centred residual sum_j ((q_j - q_mean) . n)^2, which
a brute-force search over a dense set of directions checks without any eigensolver; it must not
change when every depth is scaled; a hole among the 8 neighbours (and only there) makes a pixel
non-evaluable; disparity input must give the normals of the depth image Z = f t_c / d.
"""
import inspect
import types

import numpy as np
import pytest

import oracle
import oracle.pca as opca
from tests.geometry import backproject, plane_depth, tilted_normal
from tests.test_oracle_weighted import _noisy

CAM = dict(fx=48.12, fy=46.37, u0=31.13, v0=24.79)


def _fib_directions(n):
    """n unit vectors spread evenly over the upper hemisphere (a Fibonacci lattice)."""
    k = np.arange(n) + 0.5
    z = k / n
    phi = np.pi * (1 + 5 ** 0.5) * k
    r = np.sqrt(1 - z * z)
    return np.stack([r * np.cos(phi), r * np.sin(phi), z])


def check_planepca(fn=None):
    """Names of the failed PlanePCA pins (empty when all hold)."""
    fn = fn or opca.planepca
    fails = []
    # planes, fx != fy: exact, facing the camera
    for tilt, az, P0 in ((33, 140, [0.2, -0.1, 3.5]), (70, 20, [-0.3, 0.4, 5.0]), (0, 0, [0.0, 0.0, 2.0])):
        nrm = tilted_normal(tilt, az)
        Z = plane_depth(24, 32, CAM, nrm, P0)
        n, m = fn(Z, **CAM)
        sel = m == 1
        if not (sel.sum() == 22 * 30 and
                np.abs(n[:, sel] - nrm[:, None]).max() < 1e-9):
            fails.append(f"plane {tilt} {az}")
    # brute force on noisy windows: the normal minimises the centred residual
    d = _noisy(seed=7, H=12, W=14)
    n, m = fn(d, **CAM)
    pts = backproject(d.astype(np.float64), CAM)
    dirs = _fib_directions(200000)
    checked = 0
    H, W = d.shape
    inner = np.argwhere(m == 1)
    inner = inner[(inner[:, 0] >= 1) & (inner[:, 0] <= H - 2) & (inner[:, 1] >= 1) & (inner[:, 1] <= W - 2)]
    for (y, x) in inner[::5][:12]:
        Q = pts[:, y - 1:y + 2, x - 1:x + 2].reshape(3, 9)
        D = Q - Q.mean(axis=1, keepdims=True)
        res = lambda v: ((D.T @ v) ** 2).sum(0)  # noqa: E731
        r_grid = res(dirs)
        best = dirs[:, np.argmin(r_grid)]
        r_o = res(n[:, y, x])
        if not (abs(np.linalg.norm(n[:, y, x]) - 1) < 1e-12 and r_o <= r_grid.min() * (1 + 1e-9) + 1e-300):
            fails.append(f"not the minimiser at {y},{x}")
            break
        # and the dense search (upper hemisphere; the residual is even in n) lands next to it
        if oracle.angle_deg(np.sign(best @ n[:, y, x]) * n[:, y, x][:, None], best[:, None])[0] > 1.5:
            fails.append(f"far from the search's best at {y},{x}")
            break
        checked += 1
    if checked < 5:
        fails.append("too few windows checked")
    # faces the camera everywhere
    P = backproject(d.astype(np.float64), CAM)
    if not ((n * P).sum(0)[m == 1] < 0).all():
        fails.append("orientation")
    # scale invariance
    n3, m3 = fn(d.astype(np.float64) * 3.0, **CAM)
    if not ((m3 == m).all() and np.abs(n3 - n).max() < 1e-9):
        fails.append("depth scale")
    # holes: one among the 8 neighbours is fatal, one two pixels away is not
    img = 2.0 + 0.01 * np.arange(49, dtype=np.float64).reshape(7, 7) ** 1.3
    for (a, b) in [(2, 2), (2, 3), (2, 4), (3, 2), (3, 4), (4, 2), (4, 3), (4, 4)]:
        bad = img.copy()
        bad[a, b] = 0.0
        if fn(bad, 5.0, 5.0, 3.0, 3.0)[1][3, 3] != 0:
            fails.append(f"hole at {a},{b}")
    far = img.copy()
    far[1, 3] = np.nan
    if fn(far, 5.0, 5.0, 3.0, 3.0)[1][3, 3] != 1:
        fails.append("hole two away")
    # disparity: the normals of Z = f t_c / d
    rng = np.random.default_rng(3)
    raw = (600 + 40 * rng.standard_normal((10, 12))).astype(np.uint16)
    f, tc = 615.0, 0.1
    nd, md = fn(raw, f, f, 5.5, 4.5, disparity=True, baseline=tc, disp_scale=1.0 / 16)
    Zd = f * tc / (raw * (1.0 / 16))
    nz, mz = fn(Zd, f, f, 5.5, 4.5)
    if not ((md == mz).all() and np.abs(nd - nz).max() < 1e-9):
        fails.append("disparity")
    return fails


def test_planepca_pins_hold():
    assert check_planepca() == []


def test_planepca_agrees_with_3f2n_on_planes():
    # two estimators from the paper, both exact on a plane
    nrm = tilted_normal(50, 300)
    Z = plane_depth(20, 26, CAM, nrm, [0.1, 0.1, 4.0])
    a, ma = oracle.planepca(Z, **CAM)
    b, mb = oracle.normals(Z, **CAM)
    both = (ma == 1) & (mb == 1)
    assert both.sum() > 300 and np.nanmax(oracle.angle_deg(a, b)[both]) < 1e-9


MUTANTS = {
    "largest_eigenvector": ("v = V[:, :, 0]", "v = V[:, :, 2]"),
    "no_mean_removal": ("D = Q - Q.mean(axis=0, keepdims=True)", "D = Q"),
    "centre_left_out": ("OFFSETS = [(dv, du) for dv in (-1, 0, 1) for du in (-1, 0, 1)]",
                        "OFFSETS = [(dv, du) for dv in (-1, 0, 1) for du in (-1, 0, 1) if (dv, du) != (0, 0)]"),
    "orientation_away": ("v = np.where((key > 0)[:, None], -v, v)", "v = np.where((key < 0)[:, None], -v, v)"),
    "mask_centre_only": ("mask = np.all(np.stack([okp[1 + dv:1 + dv + H, 1 + du:1 + du + W] for dv, du in OFFSETS]), axis=0)",
                         "mask = okp[1:-1, 1:-1]"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planepca_mutant_is_caught(name):
    old, new = MUTANTS[name]
    src = inspect.getsource(opca)
    assert src.count(old) == 1, name
    mod = types.ModuleType("planepca_mutant")
    mod.__dict__["__package__"] = "oracle"
    exec(compile(src.replace(old, new), "planepca_mutant", "exec"), mod.__dict__)
    assert check_planepca(mod.planepca), f"{name} passes every PlanePCA pin"
