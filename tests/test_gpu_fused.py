"""Fused outputs of the CUDA path against the oracle: the back-projected point cloud written in the
same pass as the normals, and the octahedral 16-bit normal layout."""
import numpy as np
import pytest

import oracle
import scenes
from tests.test_gpu_parity import depth_frames, disparity_frames, to_dev

pytestmark = pytest.mark.gpu

# X = Z fl((u - u0)/fx): the sample (or f t_c / d), one quotient and one product, each within half
# an ulp, plus the rounding of u - u0: a few units of 2^-24 relative
REL = 2.0 ** -21


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


def check_points(got, img, cam, disparity=False, baseline=1.0):
    ref = oracle.points(img, cam["fx"], cam["fy"], cam["u0"], cam["v0"], disparity=disparity, baseline=baseline)
    got = np.asarray(got, np.float64)
    hole = ref[2] == 0
    assert (got[:, hole] == 0).all(), "holes must give (0, 0, 0)"
    err = np.abs(got - ref)
    assert (err <= REL * np.abs(ref) + 1e-30).all(), f"max relative error {(err / (np.abs(ref) + 1e-300)).max():.3g}"


@pytest.mark.parametrize("kind", ["f32", "f16", "u16", "dispf32"])
def test_points_match_the_oracle(torch, tfn, ctx, kind):
    if kind in ("f32", "f16"):
        frames = depth_frames([(67, 131), (480, 640), (5, 7)], 1900)
        if kind == "f16":
            frames = [(img.astype(np.float16), cam) for img, cam in frames]
        disparity, base = False, 1.0
    else:
        frames = disparity_frames([(67, 131), (130, 200)], 1950)
        if kind == "dispf32":
            frames = [((raw / 16.0).astype(np.float32), cam) for raw, cam in frames]
        disparity, base = True, 0.1
    inputs = [to_dev(torch, tfn, img) for img, _ in frames]
    cams = [cam for _, cam in frames]
    pts = [tfn.empty_points(x.shape[0], x.shape[1]) for x in inputs]
    n_with, m_with = ctx.normals_batch(inputs, cams, disparity=disparity, points=pts,
                                       disp_scale=1.0 if kind == "dispf32" else 1.0 / 16)
    n_without, m_without = ctx.normals_batch(inputs, cams, disparity=disparity,
                                             disp_scale=1.0 if kind == "dispf32" else 1.0 / 16)
    torch.cuda.synchronize()
    for k, (img, cam) in enumerate(frames):
        # the oracle reads u16 disparity with disp_scale 1/16 and float disparity as pixels
        if kind == "u16":
            check_points(pts[k].cpu().numpy(), img, cam, disparity=True, baseline=base)
        elif kind == "dispf32":
            ref = oracle.points(img, cam["fx"], cam["fy"], cam["u0"], cam["v0"], disparity=True, baseline=base,
                                disp_scale=1.0)
            got = pts[k].cpu().numpy().astype(np.float64)
            assert (np.abs(got - ref) <= REL * np.abs(ref) + 1e-30).all()
        else:
            check_points(pts[k].cpu().numpy(), img, cam)
        # the normals do not change when points are written too
        assert torch.equal(n_with[k], n_without[k]) and torch.equal(m_with[k], m_without[k])


def test_octahedral_codes_match_the_oracle(torch, tfn, ctx):
    frames = depth_frames([(67, 131), (480, 640)], 1960)
    inputs = [to_dev(torch, tfn, img) for img, _ in frames]
    cams = [cam for _, cam in frames]
    codes, masks = ctx.normals_batch(inputs, cams, output="oct16")
    n32, m32 = ctx.normals_batch(inputs, cams)
    torch.cuda.synchronize()
    for k, (img, cam) in enumerate(frames):
        q = codes[k].cpu().numpy()  # (H, W, 2) int16
        assert torch.equal(masks[k], m32[k])
        ref_n, ref_m = oracle.normals(img, cam["fx"], cam["fy"], cam["u0"], cam["v0"])
        v = ref_m == 1
        assert (q[~v] == 0).all()
        ref_q = oracle.oct_quantize(oracle.oct_encode(ref_n))  # (2, H, W)
        diff = np.abs(np.moveaxis(q, -1, 0).astype(np.int32) - ref_q.astype(np.int32))
        assert diff[:, v].max() <= 1, "codes within one step of the FP64 oracle's"
        dec = oracle.oct_decode(np.moveaxis(q, -1, 0))
        assert oracle.angle_deg(dec, ref_n)[v].max() < 0.005 + 1e-3
        # and they encode the kernel's own FP32 normal (one step: FP32 against FP64 arithmetic)
        own = oracle.oct_quantize(oracle.oct_encode(n32[k].cpu().numpy().astype(np.float64)))
        assert np.abs(np.moveaxis(q, -1, 0).astype(np.int32) - own.astype(np.int32))[:, v].max() <= 1


def test_octahedral_codes_through_the_double_float_path(torch, tfn, ctx):
    img, cam = depth_frames([(61, 99)], 1970)[0]
    d = to_dev(torch, tfn, img)
    q, m = ctx.normals(d, cam, output="oct16", flags=tfn.TFN_FLAG_REFINE_ALL)
    torch.cuda.synchronize()
    ref_n, ref_m = oracle.normals(img, cam["fx"], cam["fy"], cam["u0"], cam["v0"])
    v = ref_m == 1
    ref_q = oracle.oct_quantize(oracle.oct_encode(ref_n))
    diff = np.abs(np.moveaxis(q.cpu().numpy(), -1, 0).astype(np.int32) - ref_q.astype(np.int32))
    assert diff[:, v].max() <= 1


def test_points_through_host_path_server_and_plan(torch, tfn, ctx):
    frames = depth_frames([(96, 128)] * 4, 1980)
    cam = frames[0][1]
    imgs = [img for img, _ in frames]
    dev_in = [to_dev(torch, tfn, x) for x in imgs]
    ref_pts = [tfn.empty_points(96, 128) for _ in imgs]
    ref_n, ref_m = ctx.normals_batch(dev_in, cam, points=ref_pts)
    torch.cuda.synchronize()
    # host buffers, contiguous batch
    stack = torch.from_numpy(np.stack(imgs)).pin_memory()
    hn = torch.empty((4, 3, 96, 128), dtype=torch.float32).pin_memory()
    hm = torch.empty((4, 96, 128), dtype=torch.uint8).pin_memory()
    hp = torch.empty((4, 3, 96, 128), dtype=torch.float32).pin_memory()
    ctx.normals_batch_host([stack[k] for k in range(4)], cam, [hn[k] for k in range(4)], [hm[k] for k in range(4)],
                           points=[hp[k] for k in range(4)])
    for k in range(4):
        assert torch.equal(hp[k], ref_pts[k].cpu()) and torch.equal(hn[k], ref_n[k].cpu())
    # the server, host requests
    with tfn.Server(ctx) as srv:
        outs = []
        for k in range(4):
            n = torch.empty((3, 96, 128), dtype=torch.float32).pin_memory()
            m = torch.empty((96, 128), dtype=torch.uint8).pin_memory()
            p = torch.empty((3, 96, 128), dtype=torch.float32).pin_memory()
            outs.append((srv.submit(stack[k], cam, n, m, host=True, points=p), n, m, p))
        for k, (t, n, m, p) in enumerate(outs):
            assert srv.wait(t, 20000) == tfn.TFN_OK
            assert torch.equal(p, ref_pts[k].cpu()) and torch.equal(n, ref_n[k].cpu())
    # a plan
    plan_pts = [tfn.empty_points(96, 128) for _ in imgs]
    plan = ctx.plan(dev_in, cam, points=plan_pts)
    plan.launch()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(plan_pts, ref_pts))
    plan.close()


def test_points_are_validated(torch, tfn, ctx):
    img = to_dev(torch, tfn, np.full((32, 32), 1.0, np.float32))
    base = torch.empty(3 * 32 * 40 + 1, dtype=torch.float32, device="cuda")
    odd = base[1:].view(3, 32, 40)[:, :, :32]  # planes not on 16-byte boundaries
    with pytest.raises(tfn.TfnError) as e:
        ctx.normals(img, dict(fx=30.0, fy=30.0, u0=15.5, v0=15.5), points=odd)
    assert e.value.status == tfn.TFN_ERR_MISALIGNED
