"""Parity of the CUDA path's PlanePCA estimator (TFN_EST_PLANEPCA; Sec. II item 2, Eq. planepca) with the FP64
oracle, through the C ABI.

The mask must match bit for bit.  The normal is the eigenvector of the scatter matrix's smallest
eigenvalue; an FP32 scatter matrix perturbed by E moves it by at most ||E|| / (lambda_2 - lambda_3)
(Davis-Kahan).  With the coordinates computed relative to the centre pixel, ||E|| stays within a
small multiple of u tr(M) (u = 2^-24), so each pixel must lie within
1e-3 deg + K u tr(M) / (lambda_2 - lambda_3) of the oracle, K = 8, with the eigenvalues of the
oracle's own scatter matrix (the noisy test scenes reach at most a third of u tr(M) / gap beyond the
1e-3 deg floor; the kernel's Rayleigh-quotient step is what keeps it that small).  Where the oracle's normal is perpendicular to the viewing ray to
within 1e-4, the sign that turns it to the camera is a near-tie, and either sign is accepted.
"""
import math

import numpy as np
import pytest

import oracle
from tests.test_gpu_parity import SIZES, depth_frames, disparity_frames, to_dev

pytestmark = pytest.mark.gpu

K = 8.0
U = 2.0 ** -24


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def tfn(torch):
    import paper_2005_08165_gb300 as tfn
    return tfn


@pytest.fixture(scope="module")
def ctx(tfn):
    c = tfn.Context(0)
    yield c
    assert c.device_status() == 0
    c.close()


def compare_pca(gpu_n, gpu_m, img, cam, **kw):
    ref_n, ref_m, lam = oracle.planepca(img, cam["fx"], cam["fy"], cam["u0"], cam["v0"], eig=True, **kw)
    gpu_n = np.asarray(gpu_n, np.float64)
    gpu_m = np.asarray(gpu_m)
    assert np.array_equal(gpu_m, ref_m), f"mask differs at {np.argwhere(gpu_m != ref_m)[:5].tolist()}"
    v = ref_m == 1
    assert (gpu_n[:, ~v] == 0).all(), "non-evaluable pixels must be (0,0,0)"
    ang = oracle.angle_deg(gpu_n, ref_n)
    H, W = ref_m.shape
    uu, vv = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    ray = np.stack([(uu - cam["u0"]) / cam["fx"], (vv - cam["v0"]) / cam["fy"], np.ones_like(uu)])
    grazing = np.abs((ref_n * ray).sum(0)) < 1e-4 * np.sqrt((ray * ray).sum(0))
    ang = np.where(grazing, np.minimum(ang, 180.0 - ang), ang)
    gap = lam[..., 1] - lam[..., 0]
    tr = lam.sum(-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        excess = np.where(gap > 0, np.degrees(K * U * tr / gap), np.inf)
    bound = 1e-3 + excess
    bad = v & ~(ang <= bound)
    assert not bad.any(), (f"{bad.sum()} of {v.sum()} px beyond the bound; worst "
                           f"{ang[bad].max():.3g} deg at {np.argwhere(bad)[0].tolist()}")
    norms = np.sqrt((gpu_n[:, v] ** 2).sum(0))
    assert np.abs(norms - 1).max(initial=0) < 1e-5
    # the share of pixels held to the plain 1e-3 deg (the well-conditioned ones)
    tight = v & (excess < 1e-3)
    return {"pixels": int(v.sum()), "tight": int(tight.sum()),
            "max_tight_deg": float(ang[tight].max()) if tight.any() else 0.0,
            "max_ratio": float(np.max(np.where(v & np.isfinite(excess) & (excess > 0),
                                              (ang - 1e-3).clip(0) / np.where(excess > 0, excess, 1), 0)))}


def test_planepca_depth(torch, tfn, ctx):
    frames = depth_frames(SIZES + [(480, 640)], 2800)
    inputs = [to_dev(torch, tfn, img) for img, _ in frames]
    n, m = ctx.normals_batch(inputs, [cam for _, cam in frames], grad="planepca")
    torch.cuda.synchronize()
    tight = 0
    for k, (img, cam) in enumerate(frames):
        st = compare_pca(n[k].cpu().numpy(), m[k].cpu().numpy(), img, cam)
        tight += st["tight"]
        print(img.shape, st)
    assert tight > 1000


def test_planepca_clean_scenes_are_tight(torch, tfn, ctx):
    # noise-free scenes (planes and spheres): apart from windows across a depth edge, the pixels are well
    # conditioned (tr / gap < 36, so held to 1e-3 deg), and there the FP32 normal sits within 2e-4 deg
    frames = depth_frames([(120, 160), (96, 128)], 2850, noise=0.0, holes=0.01)
    inputs = [to_dev(torch, tfn, img) for img, _ in frames]
    n, m = ctx.normals_batch(inputs, [cam for _, cam in frames], grad="planepca")
    torch.cuda.synchronize()
    for k, (img, cam) in enumerate(frames):
        st = compare_pca(n[k].cpu().numpy(), m[k].cpu().numpy(), img, cam)
        assert st["tight"] > 0.75 * st["pixels"] and st["max_tight_deg"] < 2e-4, st


def test_planepca_steep_planes(torch, tfn, ctx):
    # planes seen at grazing angles: the scatter matrix is strongly anisotropic (lambda_2 / tr down to
    # about 1e-4), where the characteristic cubic alone can land on the wrong eigenvalue
    from tests.geometry import plane_depth, tilted_normal
    cam = dict(fx=481.2, fy=481.2, u0=63.5, v0=47.5)
    for tilt, az in ((80, 30), (86, 200), (88.5, 120)):
        nrm = tilted_normal(tilt, az)
        Z = plane_depth(96, 128, cam, nrm, [0.0, 0.0, 2.0]).astype(np.float32)
        Z = np.where((Z > 0.05) & (Z < 50), Z, 0).astype(np.float32)
        n, m = ctx.normals(to_dev(torch, tfn, Z), cam, grad="planepca")
        torch.cuda.synchronize()
        st = compare_pca(n.cpu().numpy(), m.cpu().numpy(), Z, cam)
        assert st["pixels"] > 1000


@pytest.mark.parametrize("kind", ["f16", "u16", "dispf32"])
def test_planepca_other_inputs(torch, tfn, ctx, kind):
    if kind == "f16":
        img, cam = depth_frames([(67, 131)], 2900)[0]
        img = img.astype(np.float16)
        n, m = ctx.normals(to_dev(torch, tfn, img), cam, grad="planepca")
        torch.cuda.synchronize()
        compare_pca(n.cpu().numpy(), m.cpu().numpy(), img, cam)
        return
    raw, cam = disparity_frames([(67, 131)], 2950)[0]
    if kind == "u16":
        n, m = ctx.normals(to_dev(torch, tfn, raw), cam, grad="planepca", disparity=True)
        torch.cuda.synchronize()
        compare_pca(n.cpu().numpy(), m.cpu().numpy(), raw, cam, disparity=True, baseline=0.1)
    else:
        d = (raw / 16.0).astype(np.float32)
        n, m = ctx.normals(to_dev(torch, tfn, d), cam, grad="planepca", disparity=True, disp_scale=1.0)
        torch.cuda.synchronize()
        compare_pca(n.cpu().numpy(), m.cpu().numpy(), d, cam, disparity=True, baseline=0.1, disp_scale=1.0)


def test_planepca_tile_shapes_points_and_plan(torch, tfn, ctx):
    img, cam = depth_frames([(61, 99)], 3000)[0]
    d = to_dev(torch, tfn, img)
    ref = None
    with tfn.Context(0) as c:
        for shape in range(tfn.tfn_tile_shape_count()):
            c.set_tile_shape(shape)
            nn, mm = c.normals(d, cam, grad="planepca")
            torch.cuda.synchronize()
            got = (nn.cpu(), mm.cpu())
            if ref is None:
                ref = got
            assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1]), f"shape {shape} differs"
        assert c.device_status() == 0
    # the fused point cloud and a plan give the same normals
    pts = tfn.empty_points(61, 99)
    n2, m2 = ctx.normals(d, cam, grad="planepca", points=pts)
    plan = ctx.plan([d], cam, grad="planepca")
    plan.launch()
    torch.cuda.synchronize()
    assert torch.equal(n2.cpu(), ref[0]) and torch.equal(plan.normals[0].cpu(), ref[0])
    plan.close()


def test_planepca_estimator_is_validated(torch, tfn, ctx):
    import ctypes
    d = to_dev(torch, tfn, np.full((16, 16), 2.0, np.float32))
    cam = dict(fx=20.0, fy=20.0, u0=7.5, v0=7.5)
    f = tfn.make_frame(d, tfn.empty_normals(16, 16), tfn.empty_image((16, 16), torch.uint8), cam)
    m = tfn.make_method()
    m.estimator = 2
    assert tfn.tfn_normals(ctx.handle, ctypes.byref(f), ctypes.byref(m), None) == tfn.TFN_ERR_INVALID_ARG
    assert math.isfinite(K)
