"""Parity of the CUDA path's 5x5 gradient filters (TFN_GRAD_SEP5 and its named members FD5, Sobel5,
Prewitt5) with the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from tests.parity import compare
from tests.test_gpu_parity import SIZES, depth_frames, disparity_frames, to_dev

pytestmark = pytest.mark.gpu

NAMED = ["fd5", "sobel5", "prewitt5"]
PROFILES = [(1.0, 0.3, 2.0, 0.5, 0.1), (1.0, 0.0, 1.0, 0.0, 1.0), (3.0, -1.0, 1.0, 2.0, -0.5),
            (1.0, 0.0, 2.0, 1.0, 0.0)]


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


@pytest.mark.parametrize("grad", NAMED)
@pytest.mark.parametrize("phi", ["mean", "median"])
def test_named_5x5_filters(torch, tfn, ctx, grad, phi):
    frames = depth_frames(SIZES + [(480, 640)], 2300)
    inputs = [to_dev(torch, tfn, img) for img, _ in frames]
    n, m = ctx.normals_batch(inputs, [cam for _, cam in frames], grad=grad, phi=phi)
    torch.cuda.synchronize()
    for k, (img, cam) in enumerate(frames):
        compare(n[k].cpu().numpy(), m[k].cpu().numpy(), img, cam, grad=grad, phi=phi)


@pytest.mark.parametrize("weights", PROFILES)
@pytest.mark.parametrize("phi", ["mean", "median"])
def test_sep5_profiles(torch, tfn, ctx, weights, phi):
    frames = depth_frames(SIZES, 2400)
    inputs = [to_dev(torch, tfn, img) for img, _ in frames]
    n, m = ctx.normals_batch(inputs, [cam for _, cam in frames], grad="sep5", phi=phi, weights=weights)
    torch.cuda.synchronize()
    for k, (img, cam) in enumerate(frames):
        compare(n[k].cpu().numpy(), m[k].cpu().numpy(), img, cam, grad="sep5", phi=phi, weights=weights)


@pytest.mark.parametrize("kind", ["f16", "u16", "dispf32"])
def test_5x5_filters_on_other_inputs(torch, tfn, ctx, kind):
    if kind == "f16":
        img, cam = depth_frames([(67, 131)], 2500)[0]
        img = img.astype(np.float16)
        n, m = ctx.normals(to_dev(torch, tfn, img), cam, grad="sobel5")
        torch.cuda.synchronize()
        compare(n.cpu().numpy(), m.cpu().numpy(), img, cam, grad="sobel5", phi="mean")
        return
    raw, cam = disparity_frames([(67, 131)], 2550)[0]
    if kind == "u16":
        for grad, phi in (("fd5", "median"), ("sobel5", "mean")):
            n, m = ctx.normals(to_dev(torch, tfn, raw), cam, grad=grad, phi=phi, disparity=True)
            torch.cuda.synchronize()
            compare(n.cpu().numpy(), m.cpu().numpy(), raw, cam, grad=grad, phi=phi, disparity=True, baseline=0.1)
    else:
        d = (raw / 16.0).astype(np.float32)
        n, m = ctx.normals(to_dev(torch, tfn, d), cam, grad="prewitt5", disparity=True, disp_scale=1.0)
        torch.cuda.synchronize()
        compare(n.cpu().numpy(), m.cpu().numpy(), d, cam, grad="prewitt5", phi="mean", disparity=True,
                baseline=0.1, disp_scale=1.0)


def test_5x5_double_float_path_and_tile_shapes(torch, tfn, ctx):
    img, cam = depth_frames([(61, 99)], 2600)[0]
    d = to_dev(torch, tfn, img)
    for grad, w in (("sobel5", None), ("sep5", (3.0, -1.0, 1.0, 2.0, -0.5))):
        n, m = ctx.normals(d, cam, grad=grad, weights=w, flags=tfn.TFN_FLAG_REFINE_ALL)
        torch.cuda.synchronize()
        compare(n.cpu().numpy(), m.cpu().numpy(), img, cam, grad=grad, phi="mean", weights=w, tol=1e-5)
    ref = None
    with tfn.Context(0) as c:
        for shape in range(tfn.tfn_tile_shape_count()):
            c.set_tile_shape(shape)
            nn, mm = c.normals(d, cam, grad="fd5", phi="median")
            torch.cuda.synchronize()
            got = (nn.cpu(), mm.cpu())
            if ref is None:
                ref = got
            assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1]), f"shape {shape} differs"
        assert c.device_status() == 0


def test_5x5_filters_through_host_path_and_plan(torch, tfn, ctx):
    frames = depth_frames([(96, 128)] * 3, 2700)
    cam = frames[0][1]
    imgs = [img for img, _ in frames]
    dev_in = [to_dev(torch, tfn, x) for x in imgs]
    ref_n, ref_m = ctx.normals_batch(dev_in, cam, grad="sobel5")
    torch.cuda.synchronize()
    stack = torch.from_numpy(np.stack(imgs)).pin_memory()
    hn = torch.empty((3, 3, 96, 128), dtype=torch.float32).pin_memory()
    hm = torch.empty((3, 96, 128), dtype=torch.uint8).pin_memory()
    ctx.normals_batch_host([stack[k] for k in range(3)], cam, [hn[k] for k in range(3)], [hm[k] for k in range(3)],
                           grad="sobel5")
    for k in range(3):
        assert torch.equal(hn[k], ref_n[k].cpu()) and torch.equal(hm[k], ref_m[k].cpu())
    plan = ctx.plan(dev_in, cam, grad="sobel5")
    plan.launch()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(plan.normals, ref_n))
    plan.close()


@pytest.mark.parametrize("phi", ["mean", "median"])
def test_no_candidate_special_case(torch, tfn, ctx, phi):
    # plateaus of equal depth: pixels whose 8 neighbours all share their depth while a 5x5 filter's outer
    # taps see the next plateau get [0, 0, -1] (Sec. III special case)
    img = np.full((40, 48), 2.0, np.float32)
    img[:, 20:] = 2.5
    img[24:, :] += 0.25
    img[10, 10] = 0.0  # a hole
    cam = dict(fx=40.0, fy=40.0, u0=23.5, v0=19.5)
    for grad in ("fd5", "sobel5", "fd"):
        n, m = ctx.normals(to_dev(torch, tfn, img), cam, grad=grad, phi=phi)
        torch.cuda.synchronize()
        compare(n.cpu().numpy(), m.cpu().numpy(), img, cam, grad=grad, phi=phi)
    n, m = ctx.normals(to_dev(torch, tfn, img), cam, grad="fd5", phi=phi)
    torch.cuda.synchronize()
    assert n[:, 19, 18].tolist() == [0.0, 0.0, -1.0]


def test_sep5_weights_are_validated(torch, tfn, ctx):
    d = to_dev(torch, tfn, np.full((16, 16), 2.0, np.float32))
    cam = dict(fx=20.0, fy=20.0, u0=7.5, v0=7.5)
    for w in ((2.0, -1.0, 1.0, 0.0, 0.0), (1.0, 0.0, 1.0, -0.5, 0.0), (float("nan"), 0.0, 1.0, 0.0, 0.0)):
        with pytest.raises(tfn.TfnError) as e:
            ctx.normals(d, cam, grad="sep5", weights=w)
        assert e.value.status == tfn.TFN_ERR_INVALID_ARG


@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (4, 4), (5, 5), (6, 9), (9, 1)])
def test_5x5_and_planepca_tiny_images(torch, tfn, ctx, shape):
    from tests.test_gpu_planepca import compare_pca
    rng = np.random.default_rng(2)
    img = rng.uniform(1, 2, size=shape).astype(np.float32)
    cam = dict(fx=3.0, fy=3.0, u0=(shape[1] - 1) / 2, v0=(shape[0] - 1) / 2)
    d = to_dev(torch, tfn, img)
    for grad in ("fd5", "sobel5"):
        for phi in ("mean", "median"):
            n, m = ctx.normals(d, cam, grad=grad, phi=phi)
            torch.cuda.synchronize()
            compare(n.cpu().numpy(), m.cpu().numpy(), img, cam, grad=grad, phi=phi)
    n, m = ctx.normals(d, cam, grad="planepca")
    torch.cuda.synchronize()
    compare_pca(n.cpu().numpy(), m.cpu().numpy(), img, cam)


def test_special_values_5x5_and_planepca(torch, tfn, ctx):
    from tests.test_gpu_planepca import compare_pca
    H, W = 23, 37
    img = np.full((H, W), 2.5, np.float32)
    img += np.linspace(0, 0.3, W, dtype=np.float32)[None, :]
    img[3, 4:11] = [np.nan, np.inf, -np.inf, -1.0, 0.0, 2.0 ** -17, 2.0 ** 17]
    img[10, 10] = 2.0 ** -16
    img[12, 12] = 2.0 ** 16
    cam = dict(fx=20.0, fy=21.0, u0=18.0, v0=11.0)
    d = to_dev(torch, tfn, img)
    for grad in ("fd5", "sobel5", "prewitt5"):
        for phi in ("mean", "median"):
            n, m = ctx.normals(d, cam, grad=grad, phi=phi)
            torch.cuda.synchronize()
            compare(n.cpu().numpy(), m.cpu().numpy(), img, cam, grad=grad, phi=phi)
    n, m = ctx.normals(d, cam, grad="planepca")
    torch.cuda.synchronize()
    compare_pca(n.cpu().numpy(), m.cpu().numpy(), img, cam)


@pytest.mark.parametrize("grad,phi", [("sobel5", "mean"), ("fd5", "median"), ("planepca", "mean")])
def test_full_batch_256_sampled(torch, tfn, ctx, grad, phi):
    # the bench's variant launch: 256 noisy 480x640 frames in one plan; three frames are compared with
    # the oracle pixel by pixel, all frames for properties that hold at any size
    import scenes
    from tests.test_gpu_planepca import compare_pca
    depth = scenes.noisy_batch(256)
    d = tfn.empty_image(depth.shape, torch.float32)
    d.copy_(torch.from_numpy(depth))
    normals = tfn.empty_normals(480, 640, lead=(256,))
    masks = tfn.empty_image((256, 480, 640), torch.uint8)
    plan = ctx.plan([d[k] for k in range(256)], scenes.CAMERA, grad=grad, phi=phi,
                    normals=[normals[k] for k in range(256)], masks=[masks[k] for k in range(256)])
    plan.launch()
    torch.cuda.synchronize()
    plan.close()
    for k in (3, 50, 200):
        if grad == "planepca":
            compare_pca(normals[k].cpu().numpy(), masks[k].cpu().numpy(), depth[k], scenes.CAMERA)
        else:
            compare(normals[k].cpu().numpy(), masks[k].cpu().numpy(), depth[k], scenes.CAMERA, grad=grad, phi=phi)
    v = masks.bool()
    nn = (normals.float() ** 2).sum(1)
    assert torch.isfinite(normals).all()
    assert ((nn - 1).abs()[v] < 1e-5).all() and (nn[~v] == 0).all()
    halo = 1 if grad == "planepca" else 2  # the estimator's border of non-evaluable pixels
    border = torch.zeros((480, 640), dtype=torch.bool, device=v.device)
    border[:halo, :] = border[-halo:, :] = True
    border[:, :halo] = border[:, -halo:] = True
    assert not v[:, border].any()


@pytest.mark.parametrize("grad", ["fd5", "planepca"])
def test_server_runs_the_new_estimators(torch, tfn, ctx, grad):
    # device requests through a server give the bits of a direct call
    frames = depth_frames([(96, 128), (61, 99), (96, 128)], 3100)
    with tfn.Server(ctx, grad=grad) as srv:
        outs = []
        for img, cam in frames:
            d = to_dev(torch, tfn, img)
            n = tfn.empty_normals(img.shape[0], img.shape[1])
            m = tfn.empty_image(img.shape, torch.uint8)
            outs.append((srv.submit(d, cam, n, m), d, cam, n, m))
        for t, d, cam, n, m in outs:
            assert srv.wait(t, 20000) == tfn.TFN_OK
            rn, rm = ctx.normals(d, cam, grad=grad)
            torch.cuda.synchronize()
            assert torch.equal(n, rn) and torch.equal(m, rm)
