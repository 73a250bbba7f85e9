"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: hand-derived
values (tests/golden), closed forms (planes: 1/Z is affine in (u, v), Sec. III
Eq. 1/z_n, so every linear-exact filter recovers the plane normal exactly),
convergence order on spheres, a textbook estimator (PlanePCA, Sec. II), the
disparity/depth identity (Sec. III Eqs. z_d, dd_2_dz), invariances and
hand-enumerated validity cases.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from tests import geometry

GRADS = ["fd", "sobel", "scharr", "prewitt"]
PHIS = ["mean", "median"]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_derived.json")


def _golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


def _run_case(case, phi, lib=None):
    cam = case["camera"]
    kind = case["kind"]
    if kind == "depth":
        img = np.array(case["grid"], np.float64)
        n, m = oracle.normals(img, cam["fx"], cam["fy"], cam["u0"], cam["v0"], grad=case["grad"], phi=phi, lib=lib)
    elif kind == "disparity_u16":
        img = np.array(case["grid"], np.uint16)
        n, m = oracle.normals(img, cam["fx"], cam["fy"], cam["u0"], cam["v0"], grad=case["grad"], phi=phi,
                              disparity=True, baseline=cam["baseline"], disp_scale=case["disp_scale"], lib=lib)
    else:
        img = np.array(case["grid"], np.float32)
        n, m = oracle.normals(img, cam["fx"], cam["fy"], cam["u0"], cam["v0"], grad=case["grad"], phi=phi,
                              disparity=True, baseline=cam["baseline"], lib=lib)
    return n, m


def check_golden(lib=None):
    """Returns a list of failures (empty when every hand-derived case holds)."""
    bad = []
    for case in _golden_cases():
        for phi, exp in case["expect"].items():
            n, m = _run_case(case, phi, lib)
            want = np.array(exp["vec"], np.float64) / math.sqrt(exp["norm2"])
            mask_ok = m[1, 1] == 1 and m.sum() == 1
            got = n[:, 1, 1]
            tol = case.get("tol_deg", 1e-9)
            ang = oracle.angle_deg(got[:, None], want[:, None])[0]
            if not mask_ok or not np.isfinite(got).all() or not (ang <= tol) or abs(np.linalg.norm(got) - 1) > 1e-12:
                bad.append((case["name"], phi, got.tolist(), want.tolist(), float(ang)))
    return bad


def test_hand_derived_golden_values():
    assert check_golden() == []


# Plane azimuths away from multiples of 45 deg keep every neighbour's dz far from
# zero (a neighbour along an iso-depth line would give the 0/0 the paper excludes).
PLANE_CASES = [(15.0, 20.0), (35.0, 65.0), (42.0, 200.0), (38.0, 115.0), (25.0, 335.0)]
CAM = dict(fx=48.12, fy=46.37, u0=31.13, v0=24.79)  # the 480x640 field of view on a small image


def plane_max_error(grad, phi, lib=None, H=48, W=64):
    worst = 0.0
    for tilt, az in PLANE_CASES:
        nrm = geometry.tilted_normal(tilt, az)
        P = np.array([0.3, -0.2, 3.0])
        if nrm @ P > 0:
            nrm = -nrm
        Z = geometry.plane_depth(H, W, CAM, nrm, P)
        n, m = oracle.normals(Z, **CAM, grad=grad, phi=phi, lib=lib)
        interior = np.zeros((H, W), bool)
        interior[1:-1, 1:-1] = True
        if not (m.astype(bool) == interior).all():
            return float("inf")
        ang = oracle.angle_deg(n[:, interior], np.broadcast_to(nrm[:, None], (3, interior.sum())))
        worst = max(worst, float(np.max(ang)))
    return worst


@pytest.mark.parametrize("grad", GRADS)
@pytest.mark.parametrize("phi", PHIS)
def test_plane_closed_form_exact(grad, phi):
    # Sec. III Eq. (1/z_n): on a plane 1/Z is affine in (u, v), so every
    # candidate equals the true n_z and the analytic normal is recovered.
    assert plane_max_error(grad, phi) < 1e-9


@pytest.mark.parametrize("grad", GRADS)
def test_plane_mean_equals_median(grad):
    Z = geometry.plane_depth(40, 50, CAM, geometry.tilted_normal(40, 30), [0, 0, 2.0])
    a, _ = oracle.normals(Z, **CAM, grad=grad, phi="mean")
    b, _ = oracle.normals(Z, **CAM, grad=grad, phi="median")
    assert np.nanmax(oracle.angle_deg(a, b)[1:-1, 1:-1]) < 1e-9


def test_frontal_plane_special_case():
    # Sec. III: equal depths -> [0, 0, -1]; the border has no full stencil.
    Z = np.full((12, 17), 2.5, np.float32)
    for grad in GRADS:
        for phi in PHIS:
            n, m = oracle.normals(Z, **CAM, grad=grad, phi=phi)
            assert (m[1:-1, 1:-1] == 1).all() and m.sum() == 10 * 15
            assert (n[:, 1:-1, 1:-1] == np.array([0, 0, -1.0])[:, None, None]).all()
            assert (n[:, m == 0] == 0).all()


def sphere_orders(phi, lib=None):
    """Median angle error on a sphere vs its analytic normal as the image
    scale doubles; returns the observed convergence orders."""
    errs = []
    for f in (100.0, 200.0, 400.0):
        S = int(0.6 * f)
        cam = dict(fx=f, fy=f, u0=(S - 1) / 2, v0=(S - 1) / 2)
        Z, gt = geometry.sphere_depth(S, S, cam, [0.1, -0.05, 3.0], 1.0)
        n, m = oracle.normals(Z, **cam, phi=phi, lib=lib)
        sel = (m == 1) & (-gt[2] > np.cos(np.deg2rad(50)))
        if sel.sum() < 100:
            return [float("nan")]
        errs.append(np.median(oracle.angle_deg(n, gt)[sel]))
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("phi", PHIS)
def test_sphere_second_order(phi):
    # Central differences are O(h^2) and the +-j candidates cancel the O(h)
    # curvature term, so the typical error falls 4x per halving of the pixel.
    orders = sphere_orders(phi)
    assert all(1.8 <= o <= 2.3 for o in orders), orders


def test_unit_norm_and_faces_camera():
    import scenes
    d, d64, prim, gt = scenes.render(11, with_truth=True)
    P = geometry.backproject(d.astype(np.float64), scenes.CAMERA)
    for grad in GRADS:
        for phi in PHIS:
            n, m = oracle.normals(d, **scenes.CAMERA, grad=grad, phi=phi)
            v = m == 1
            assert np.abs(np.sqrt((n[:, v] ** 2).sum(0)) - 1).max() < 1e-12
    for grad in GRADS:
        n, m = oracle.normals(d64, **scenes.CAMERA, grad=grad)
        planes = (m == 1) & (prim >= 0) & (prim < 6)
        from numpy.lib.stride_tricks import sliding_window_view as swv
        w = swv(np.pad(prim, 1, constant_values=-2), (3, 3))
        planes &= (w == prim[:, :, None, None]).all((2, 3))
        assert ((n * P).sum(0)[planes] < 0).all()


def test_planepca_crosscheck():
    # Sec. II, Eq. (planepca): on a noise-free plane the least-variance axis of
    # the 9 back-projected points is the plane normal, as is 3F2N's estimate.
    nrm = geometry.tilted_normal(50, 160)
    Z = geometry.plane_depth(20, 24, CAM, nrm, [0.2, 0.1, 2.0])
    P = geometry.backproject(Z, CAM)
    for grad in GRADS:
        n, m = oracle.normals(Z, **CAM, grad=grad, phi="median")
        for v in range(1, 19, 3):
            for u in range(1, 23, 3):
                Q = P[:, v - 1:v + 2, u - 1:u + 2].reshape(3, 9).T
                Q = Q - Q.mean(0)
                w_, V = np.linalg.eigh(Q.T @ Q)
                pca = V[:, 0]
                a = oracle.angle_deg(pca[:, None], n[:, v, u][:, None])[0]
                assert min(a, 180 - a) < 1e-6


def test_literal_and_algebraic_forms_agree():
    import scenes
    d = scenes.render(1005, scenes.Recipe(noise_k=0.0012, hole_frac=0.03, H=96, W=128, u0=63.5, v0=47.5,
                                          fx=96.24, fy=96.24))
    for grad in GRADS:
        for phi in PHIS:
            a, ma = oracle.normals(d, 96.24, 96.24, 63.5, 47.5, grad=grad, phi=phi, form=oracle.LITERAL)
            b, mb = oracle.normals(d, 96.24, 96.24, 63.5, 47.5, grad=grad, phi=phi, form=oracle.ALGEBRAIC)
            assert (ma == mb).all()
            assert np.nanmax(oracle.angle_deg(a, b)[ma == 1]) < 1e-8


@pytest.mark.parametrize("grad", GRADS)
def test_depth_scale_invariance(grad):
    import scenes
    d = scenes.render(7, scenes.Recipe(noise_k=0.0012, hole_frac=0.02, H=60, W=80, u0=39.5, v0=29.5,
                                       fx=60.15, fy=60.15))
    cam = dict(fx=60.15, fy=60.15, u0=39.5, v0=29.5)
    a, ma = oracle.normals(d, **cam, grad=grad, phi="median")
    b, mb = oracle.normals(d * np.float32(4.0), **cam, grad=grad, phi="median")  # exact power-of-2 scale
    assert (ma == mb).all() and np.nanmax(oracle.angle_deg(a, b)[ma == 1]) < 1e-9


@pytest.mark.parametrize("grad", GRADS)
def test_mirror_and_transpose(grad):
    import scenes
    H, W = 50, 70
    d = scenes.render(9, scenes.Recipe(noise_k=0.0012, hole_frac=0.02, H=H, W=W, u0=30.2, v0=21.7,
                                       fx=55.0, fy=61.0))
    cam = dict(fx=55.0, fy=61.0, u0=30.2, v0=21.7)
    for phi in PHIS:
        a, ma = oracle.normals(d, **cam, grad=grad, phi=phi)
        # u -> W-1-u with u0 -> W-1-u0 flips x.
        b, mb = oracle.normals(d[:, ::-1].copy(), cam["fx"], cam["fy"], W - 1 - cam["u0"], cam["v0"],
                               grad=grad, phi=phi)
        b = b[:, :, ::-1]
        mb = mb[:, ::-1]
        assert (ma == mb).all()
        b = b * np.array([-1, 1, 1.0])[:, None, None]
        assert np.nanmax(oracle.angle_deg(a, b)[ma == 1]) < 1e-8
        # swapping the image axes (and fx<->fy, u0<->v0) swaps x and y.
        c, mc = oracle.normals(d.T.copy(), cam["fy"], cam["fx"], cam["v0"], cam["u0"], grad=grad, phi=phi)
        c = c.transpose(0, 2, 1)[[1, 0, 2]]
        assert (ma == mc.T).all()
        assert np.nanmax(oracle.angle_deg(a, c)[ma == 1]) < 1e-8


@pytest.mark.parametrize("grad", GRADS)
@pytest.mark.parametrize("phi", PHIS)
def test_disparity_form_equals_depth_form(grad, phi):
    # Sec. III Eqs. (z_d), (dd_2_dz): the disparity form is the depth form
    # on Z = f t_c / d, up to the positive factor t_c.
    import scenes
    dep = scenes.render(21, scenes.Recipe(H=64, W=80, u0=39.5, v0=31.5, fx=61.5, fy=61.5, zmin=0.640625,
                                          zmax=61.5, plane_z0=0.640625, plane_z1=61.5, sphere_z0=2,
                                          sphere_z1=50, radius0=0.5, radius1=5.0))
    raw = scenes.disparity_u16(dep, 61.5 * 0.1, frac_bits=4, hole_frac=0.05, seed=5)
    cam = dict(fx=61.5, fy=61.5, u0=39.5, v0=31.5)
    a, ma = oracle.normals(raw, **cam, grad=grad, phi=phi, disparity=True, baseline=0.1, disp_scale=1 / 16)
    with np.errstate(divide="ignore"):
        Z = np.where(raw > 0, 61.5 * 0.1 / (raw.astype(np.float64) / 16), 0.0)
    b, mb = oracle.normals(Z, **cam, grad=grad, phi=phi)
    assert (ma == mb).all()
    assert np.nanmax(oracle.angle_deg(a, b)[ma == 1]) < 1e-8
    # baseline and disparity scale cancel from the direction
    c, mc = oracle.normals(raw, **cam, grad=grad, phi=phi, disparity=True, baseline=0.37, disp_scale=1 / 16)
    assert (mc == ma).all() and np.nanmax(oracle.angle_deg(a, c)[ma == 1]) < 1e-9


def test_fp16_input_decodes_exactly():
    import scenes
    d = scenes.render(31, scenes.Recipe(H=40, W=56, u0=27.5, v0=19.5, fx=40.0, fy=40.0))
    h = d.astype(np.float16)
    with np.errstate(over="ignore"):
        specials = np.array([np.inf, -np.inf, np.nan, 0.0, -0.0, 6e-8, 65504.0], np.float16)
    h[0, :7] = specials
    for grad in ("fd", "sobel"):
        a, ma = oracle.normals(h, 40.0, 40.0, 27.5, 19.5, grad=grad)
        b, mb = oracle.normals(h.astype(np.float32), 40.0, 40.0, 27.5, 19.5, grad=grad)
        assert (ma == mb).all() and (a == b).all()


def _validity_grid(value, H=7, W=7, hole=(3, 3)):
    Z = np.full((H, W), 2.0, np.float32)
    Z[hole] = value
    return Z


@pytest.mark.parametrize("value", [0.0, -1.0, np.nan, np.inf, -np.inf, 2.0 ** -17, 2.0 ** 17])
def test_holes_and_range(value):
    # Reading R1 (valid iff finite and in [2^-16, 2^16]) and R2 (every filter tap valid).
    cam = dict(fx=5.0, fy=5.0, u0=3.0, v0=3.0)
    Z = _validity_grid(value)
    n, m = oracle.normals(Z, **cam, grad="fd")
    expect = np.zeros((7, 7), np.uint8)
    expect[1:-1, 1:-1] = 1
    for (y, x) in [(3, 3), (2, 3), (4, 3), (3, 2), (3, 4)]:  # the hole and its FD users
        expect[y, x] = 0
    assert (m == expect).all()
    n, m = oracle.normals(Z, **cam, grad="sobel")
    expect = np.zeros((7, 7), np.uint8)
    expect[1:-1, 1:-1] = 1
    expect[2:5, 2:5] = 0  # every pixel whose 3x3 stencil holds the hole
    assert (m == expect).all()
    assert (n[:, m == 0] == 0).all()


def test_range_edges_are_valid():
    cam = dict(fx=5.0, fy=5.0, u0=3.0, v0=3.0)
    for value in (2.0 ** -16, 2.0 ** 16):
        Z = _validity_grid(value)
        _, m = oracle.normals(Z, **cam)
        assert m[1:-1, 1:-1].all()


def test_fd_diagonal_hole_reduces_candidates():
    # A hole on a diagonal is not an FD tap: the pixel stays valid and the
    # hole gives no candidate (reading R4).
    cam = dict(fx=10.0, fy=10.0, u0=2.0, v0=2.0)
    nrm = geometry.tilted_normal(30, 20)
    Z = geometry.plane_depth(5, 5, cam, nrm, [0, 0, 2.0])
    Z[1, 1] = 0.0
    n, m, cands, _ = oracle.normals(Z, **cam, diagnostics=True)
    assert m[2, 2] == 1 and np.isnan(cands[0, 2, 2]) and np.isfinite(cands[1:, 2, 2]).all()
    assert oracle.angle_deg(n[:, 2, 2][:, None], nrm[:, None])[0] < 1e-9


def test_phi_matches_library_mean_and_median():
    import scenes
    d = scenes.render(41, scenes.Recipe(noise_k=0.0012, hole_frac=0.05, H=40, W=48, u0=23.5, v0=19.5,
                                        fx=40.0, fy=40.0))
    for phi, fn in (("mean", np.nanmean), ("median", np.nanmedian)):
        n, m, cands, npr = oracle.normals(d, 40.0, 40.0, 23.5, 19.5, phi=phi, diagnostics=True)
        has = (m == 1) & (np.isfinite(cands).any(0))
        import warnings
        with np.errstate(all="ignore"), warnings.catch_warnings():
            warnings.simplefilter("ignore", RuntimeWarning)
            want = -fn(cands, axis=0)
        assert np.allclose(npr[2][has], want[has], rtol=1e-12, atol=0)


def test_batch_matches_single_and_threads():
    import scenes
    r = scenes.Recipe(noise_k=0.0012, hole_frac=0.03, H=48, W=64, u0=31.5, v0=23.5, fx=48.0, fy=48.0)
    frames = scenes.render_batch(50, 6, r)
    nb, mb = oracle.normals_batch(frames, 48.0, 48.0, 31.5, 23.5, grad="scharr", phi="median", threads=3)
    for k in range(6):
        n, m = oracle.normals(frames[k], 48.0, 48.0, 31.5, 23.5, grad="scharr", phi="median")
        assert (m == mb[k]).all() and np.array_equal(n, nb[k], equal_nan=True)


def test_rejects_bad_arguments():
    Z = np.ones((4, 4), np.float32)
    with pytest.raises(ValueError):
        oracle.normals(Z, 0.0, 1.0, 0, 0)
    with pytest.raises(ValueError):
        oracle.normals(Z.astype(np.uint16), 1.0, 2.0, 0, 0, disparity=True)  # fx != fy


@pytest.mark.parametrize("phi", PHIS)
def test_brute_force_back_projection_4x4(phi):
    # tiny images done the long way: every pixel back-projected through the inverse of the intrinsic
    # matrix (numpy.linalg.inv, not the oracle's per-axis formula), the FD gradients by scipy's
    # correlation of 1/Z, each candidate from the back-projected difference vectors, and numpy's mean
    # or median; the interior normals must match the oracle's
    from scipy.ndimage import correlate
    rng = np.random.default_rng(11)
    for trial in range(20):
        fx, fy = rng.uniform(3, 9), rng.uniform(3, 9)
        u0, v0 = rng.uniform(0.5, 2.5), rng.uniform(0.5, 2.5)
        Z = rng.uniform(1.0, 1.6, size=(4, 4))
        K = np.array([[fx, 0, u0], [0, fy, v0], [0, 0, 1.0]])
        Kinv = np.linalg.inv(K)
        P = np.zeros((4, 4, 3))
        for v in range(4):
            for u in range(4):
                P[v, u] = Z[v, u] * (Kinv @ np.array([u, v, 1.0]))
        w = 1.0 / Z
        gu = correlate(w, np.array([[0, 0, 0], [-1, 0, 1], [0, 0, 0]]) / 2.0, mode="constant")
        gv = correlate(w, np.array([[0, -1, 0], [0, 0, 0], [0, 1, 0]]) / 2.0, mode="constant")
        n_or, m_or = oracle.normals(Z, fx, fy, u0, v0, phi=phi)
        for v in (1, 2):
            for u in (1, 2):
                nx, ny = fx * gu[v, u], fy * gv[v, u]
                cands = []
                for dv in (-1, 0, 1):
                    for du in (-1, 0, 1):
                        if (dv, du) == (0, 0):
                            continue
                        r = P[v + dv, u + du] - P[v, u]
                        if r[2] != 0:
                            cands.append((r[0] * nx + r[1] * ny) / r[2])
                nz = -(np.mean(cands) if phi == "mean" else np.median(cands))
                npr = np.array([nx, ny, nz])
                want = -npr / np.linalg.norm(npr)
                assert m_or[v, u] == 1
                ang = oracle.angle_deg(want[:, None], n_or[:, v, u][:, None])[0]
                assert ang < 1e-8, (trial, v, u, ang)
