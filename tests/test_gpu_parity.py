"""Parity of the CUDA path (through the C ABI) with the FP64 oracle."""
import ctypes

import numpy as np
import pytest

import scenes
from tests.parity import compare

pytestmark = pytest.mark.gpu

GRADS = ["fd", "sobel", "scharr", "prewitt"]
PHIS = ["mean", "median"]
SIZES = [(67, 131), (130, 200), (33, 64), (5, 7)]


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


def small_recipe(H, W, **kw):
    f = 481.2 * W / 640
    return scenes.Recipe(H=H, W=W, fx=f, fy=f, u0=(W - 1) / 2, v0=(H - 1) / 2, **kw)


def to_dev(torch, tfn, img):
    if img.dtype == np.uint16:  # raw u16 bits travel as int16
        t = tfn.empty_image(img.shape, torch.int16)
        t.copy_(torch.from_numpy(img.view(np.int16)))
        return t
    dt = {np.float32: torch.float32, np.float16: torch.float16}[img.dtype.type]
    t = tfn.empty_image(img.shape, dt)
    t.copy_(torch.from_numpy(img))
    return t


def depth_frames(sizes, seed, noise=0.0012, holes=0.03):
    out = []
    for k, (H, W) in enumerate(sizes):
        r = small_recipe(H, W, noise_k=noise, hole_frac=holes)
        out.append((scenes.render(seed + k, r), r.camera))
    return out


def disparity_frames(sizes, seed):
    out = []
    for k, (H, W) in enumerate(sizes):
        f = 615.0 * W / 640
        r = scenes.Recipe(H=H, W=W, fx=f, fy=f, u0=(W - 1) / 2, v0=(H - 1) / 2, zmin=0.640625, zmax=61.5,
                          plane_z0=0.640625, plane_z1=61.5, sphere_z0=2, sphere_z1=50, radius0=0.5, radius1=5)
        d = scenes.render(seed + k, r)
        raw = scenes.disparity_u16(d, f * 0.1, frac_bits=4, hole_frac=0.05, seed=seed + 100 + k)
        cam = dict(r.camera, baseline=0.1)
        out.append((raw, cam))
    return out


def run_batch(torch, tfn, ctx, frames, *, grad, phi, disparity=False, output="f32", flags=0):
    inputs = [to_dev(torch, tfn, img) for img, _ in frames]
    cams = [cam for _, cam in frames]
    n, m = ctx.normals_batch(inputs, cams, grad=grad, phi=phi, disparity=disparity, output=output, flags=flags)
    torch.cuda.synchronize()
    return [x.float().cpu().numpy() for x in n], [x.cpu().numpy() for x in m]


@pytest.mark.parametrize("grad", GRADS)
@pytest.mark.parametrize("phi", PHIS)
def test_depth_f32_ragged_sizes(torch, tfn, ctx, grad, phi):
    frames = depth_frames(SIZES, 500)
    n, m = run_batch(torch, tfn, ctx, frames, grad=grad, phi=phi)
    for (img, cam), nk, mk in zip(frames, n, m):
        compare(nk, mk, img, cam, grad=grad, phi=phi)


@pytest.mark.parametrize("grad", GRADS)
@pytest.mark.parametrize("phi", PHIS)
def test_depth_f16_input(torch, tfn, ctx, grad, phi):
    frames = [(img.astype(np.float16), cam) for img, cam in depth_frames(SIZES[:2], 600, noise=0.0)]
    n, m = run_batch(torch, tfn, ctx, frames, grad=grad, phi=phi)
    for (img, cam), nk, mk in zip(frames, n, m):
        compare(nk, mk, img, cam, grad=grad, phi=phi)


@pytest.mark.parametrize("grad", GRADS)
@pytest.mark.parametrize("phi", PHIS)
def test_disparity_u16(torch, tfn, ctx, grad, phi):
    frames = disparity_frames(SIZES[:3], 700)
    n, m = run_batch(torch, tfn, ctx, frames, grad=grad, phi=phi, disparity=True)
    for (img, cam), nk, mk in zip(frames, n, m):
        compare(nk, mk, img, cam, grad=grad, phi=phi, disparity=True, baseline=cam["baseline"])


@pytest.mark.parametrize("grad", ["fd", "scharr"])
@pytest.mark.parametrize("phi", PHIS)
def test_disparity_f32(torch, tfn, ctx, grad, phi):
    frames = []
    for raw, cam in disparity_frames(SIZES[:2], 800):
        frames.append(((raw.astype(np.float32) / 16).astype(np.float32), cam))
    n, m = run_batch(torch, tfn, ctx, frames, grad=grad, phi=phi, disparity=True)
    for (img, cam), nk, mk in zip(frames, n, m):
        compare(nk, mk, img, cam, grad=grad, phi=phi, disparity=True, baseline=cam["baseline"])


@pytest.mark.parametrize("grad", ["fd", "sobel", "scharr"])
@pytest.mark.parametrize("phi", PHIS)
def test_full_size_noisy_frames(torch, tfn, ctx, grad, phi):
    # the 480x640 workload: sigma = 0.0012 Z^2 noise, 3% holes
    frames = [(scenes.render_batch(1000 + k, 1, scenes.Recipe(noise_k=0.0012, hole_frac=0.03))[0], scenes.CAMERA)
              for k in (0, 1)]
    n, m = run_batch(torch, tfn, ctx, frames, grad=grad, phi=phi)
    for (img, cam), nk, mk in zip(frames, n, m):
        compare(nk, mk, img, cam, grad=grad, phi=phi)


def test_full_size_clean_frame_fd_mean(torch, tfn, ctx):
    frames = [(scenes.single_frame(), scenes.CAMERA)]
    n, m = run_batch(torch, tfn, ctx, frames, grad="fd", phi="mean")
    compare(n[0], m[0], frames[0][0], scenes.CAMERA, grad="fd", phi="mean")


@pytest.mark.parametrize("grad", GRADS)
@pytest.mark.parametrize("phi", PHIS)
def test_refine_all_path_is_tight(torch, tfn, ctx, grad, phi):
    # every pixel through the double-float path: agreement far below the tolerance
    frames = depth_frames(SIZES[:2], 900)
    n, m = run_batch(torch, tfn, ctx, frames, grad=grad, phi=phi, flags=tfn.TFN_FLAG_REFINE_ALL)
    for (img, cam), nk, mk in zip(frames, n, m):
        st = compare(nk, mk, img, cam, grad=grad, phi=phi, tol=1e-5)
        assert st["over"] == 0 or phi == "median"


def test_refinement_queue_takes_every_flagged_pixel(torch, tfn, ctx):
    # the FD mean refines its flagged pixels in its own kernel, 32 at a time from a per-warp queue:
    # with every pixel flagged, each warp fills and drains its queue many times per item, across
    # frames of different sizes (a ragged frame among 40 full ones keeps the default tile shape),
    # and the queue's last, partial round runs after the warp's last item
    imgs = list(scenes.noisy_batch(40, seed0=960))
    frames = [(img, scenes.CAMERA) for img in imgs] + depth_frames([(67, 131), (200, 333)], 970)
    ctx.refined_pixels()
    n, m = run_batch(torch, tfn, ctx, frames, grad="fd", phi="mean", flags=tfn.TFN_FLAG_REFINE_ALL)
    refined = ctx.refined_pixels()
    evaluable = sum(int((mk == 1).sum()) for mk in m)
    assert all(set(np.unique(mk).tolist()) <= {0, 1} for mk in m), "a refined pixel has mask bit 1"
    assert 0.9 * evaluable < refined <= evaluable, (refined, evaluable)  # (flat pixels are not refined)
    for k in (0, 39, 40, 41):
        img, cam = frames[k]
        st = compare(n[k], m[k], img, cam, grad="fd", phi="mean", tol=1e-5)
        assert st["over"] == 0
    # and without the flag (the usual few flagged pixels), against the oracle
    n2, m2 = run_batch(torch, tfn, ctx, frames, grad="fd", phi="mean")
    for k in (0, 40, 41):
        img, cam = frames[k]
        compare(n2[k], m2[k], img, cam, grad="fd", phi="mean")


@pytest.mark.parametrize("phi", PHIS)
def test_refinement_list_overflow_scans_the_mask(torch, tfn, ctx, phi):
    # every pixel of 40 noisy 480x640 frames flagged (Sobel: the filters other than the FD mean
    # refine in a second kernel): about 12M, past the 262144 entries of the launch's refinement list, so the
    # refinement kernel finds them by their mask bit instead.  40 frames take the default tile
    # shape (a launch of fewer items would refine in place).
    imgs = scenes.noisy_batch(40, seed0=950)
    ctx.refined_pixels()  # (reading the counter restarts it)
    n, m = run_batch(torch, tfn, ctx, [(img, scenes.CAMERA) for img in imgs], grad="sobel", phi=phi,
                     flags=tfn.TFN_FLAG_REFINE_ALL)
    refined = ctx.refined_pixels()
    evaluable = sum(int((mk == 1).sum()) for mk in m)
    assert all(set(np.unique(mk).tolist()) <= {0, 1} for mk in m), "a flagged pixel kept its mask bit"
    assert 262144 < refined <= evaluable and refined > 0.9 * evaluable, (refined, evaluable)
    for k in (0, 39):
        st = compare(n[k], m[k], imgs[k], scenes.CAMERA, grad="sobel", phi=phi, tol=1e-5)
        assert st["over"] == 0 or phi == "median"


WEIGHTS = [(1.0, 3.0, 1.0), (1.0, 0.0, 0.0), (2.0, -1.0, 0.5), (0.0, 1.0, 0.0)]


@pytest.mark.parametrize("weights", WEIGHTS)
@pytest.mark.parametrize("phi", PHIS)
def test_weighted_gradient_family(torch, tfn, ctx, weights, phi):
    frames = depth_frames(SIZES, 2100)
    inputs = [to_dev(torch, tfn, img) for img, _ in frames]
    cams = [cam for _, cam in frames]
    n, m = ctx.normals_batch(inputs, cams, grad="weighted", phi=phi, weights=weights)
    torch.cuda.synchronize()
    for k, (img, cam) in enumerate(frames):
        compare(n[k].cpu().numpy(), m[k].cpu().numpy(), img, cam, grad="weighted", phi=phi, weights=weights)
    # u16 disparity too
    dframes = disparity_frames([(67, 131)], 2150)
    raw, cam = dframes[0]
    dn, dm = ctx.normals(to_dev(torch, tfn, raw), cam, grad="weighted", phi=phi, weights=weights, disparity=True)
    torch.cuda.synchronize()
    compare(dn.cpu().numpy(), dm.cpu().numpy(), raw, cam, grad="weighted", phi=phi, disparity=True, baseline=0.1,
            weights=weights)


def test_weighted_family_double_float_path_and_shapes(torch, tfn, ctx):
    img, cam = depth_frames([(61, 99)], 2200)[0]
    d = to_dev(torch, tfn, img)
    w = (1.0, 0.7, 0.2)
    n, m = ctx.normals(d, cam, grad="weighted", weights=w, flags=tfn.TFN_FLAG_REFINE_ALL)
    torch.cuda.synchronize()
    compare(n.cpu().numpy(), m.cpu().numpy(), img, cam, grad="weighted", phi="mean", weights=w, tol=1e-5)
    ref = None
    with tfn.Context(0) as c:
        for shape in range(tfn.tfn_tile_shape_count()):
            c.set_tile_shape(shape)
            nn, mm = c.normals(d, cam, grad="weighted", weights=w)
            torch.cuda.synchronize()
            got = (nn.cpu(), mm.cpu())
            if ref is None:
                ref = got
            assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1]), f"shape {shape} differs"
    with pytest.raises(tfn.TfnError) as e:
        ctx.normals(d, cam, grad="weighted", weights=(0.0, 0.0, 0.0))
    assert e.value.status == tfn.TFN_ERR_INVALID_ARG


@pytest.mark.parametrize("output", ["f16", "bf16", "f16x4", "bf16x4"])
def test_reduced_precision_outputs_round_the_f32_result(torch, tfn, ctx, output):
    img, cam = depth_frames([(61, 99)], 1100)[0]
    d = to_dev(torch, tfn, img)
    n32, m32 = ctx.normals(d, cam)
    n16, m16 = ctx.normals(d, cam, output=output)
    torch.cuda.synchronize()
    dt = torch.float16 if output.startswith("f16") else torch.bfloat16
    want = n32.to(dt)
    got = n16 if output in ("f16", "bf16") else n16[..., :3].permute(2, 0, 1)
    assert torch.equal(got.contiguous().view(torch.int16), want.contiguous().view(torch.int16))
    if output in ("f16x4", "bf16x4"):
        assert (n16[..., 3] == 0).all()
    assert torch.equal(m16, m32)


@pytest.mark.parametrize("output", ["f16", "bf16", "f16x4", "bf16x4"])
def test_fp16_precision_form_angle_vs_oracle(torch, tfn, ctx, output):
    """FP16 depth in, FP16/BF16 normals out: per-frame mean and max angle against the FP64 oracle run on
    the same FP16-decoded depth (clean scenes rounded to FP16, 480x640).  FP16 outputs (11-bit significand)
    must keep the mean within 0.05 deg; BF16 outputs (8-bit significand) sit at their rounding floor, a
    mean of about 0.05 deg, and are held to that floor instead."""
    import oracle
    imgs = scenes.render_batch(3000, 3, scenes.Recipe()).astype(np.float16)
    inputs = [to_dev(torch, tfn, x) for x in imgs]
    n, m = ctx.normals_batch(inputs, scenes.CAMERA, output=output)
    torch.cuda.synchronize()
    rows = []
    for k, img in enumerate(imgs):
        got = n[k].float() if output in ("f16", "bf16") else n[k][..., :3].permute(2, 0, 1).float()
        got = got.cpu().numpy().astype(np.float64)
        cam = scenes.CAMERA
        ref_n, ref_m = oracle.normals(img, cam["fx"], cam["fy"], cam["u0"], cam["v0"], grad="fd", phi="mean")
        assert (m[k].cpu().numpy() == ref_m).all()
        v = ref_m == 1
        ang = oracle.angle_deg(got, ref_n)[v]
        rows.append((float(ang.mean()), float(ang.max())))
    print(f"\nFP16 in -> {output} out, angle vs FP64 oracle per frame (mean, max deg): "
          + ", ".join(f"({a:.4f}, {b:.4f})" for a, b in rows))
    # rounding each component to nearest moves it by at most 2^-11 (f16) / 2^-8 (bf16) of itself, so the
    # unit vector turns by at most about that many radians (sqrt(3) x for safety), plus the FP32 path's 1e-3
    half_ulp = 2.0 ** -11 if output.startswith("f16") else 2.0 ** -8
    floor = np.degrees(np.sqrt(3) * half_ulp) + 1e-3
    assert all(b <= floor for _, b in rows)
    if output.startswith("f16"):
        assert all(a <= 0.05 for a, _ in rows)
    else:
        assert all(a <= floor / 2 for a, _ in rows)


def test_batch_composition_and_alone_bit_identical(torch, tfn, ctx):
    frames = depth_frames([(67, 131), (480, 640), (33, 64)], 1200)
    n_mix, m_mix = run_batch(torch, tfn, ctx, frames, grad="scharr", phi="median")
    for k, fr in enumerate(frames):
        n1, m1 = run_batch(torch, tfn, ctx, [fr], grad="scharr", phi="median")
        assert np.array_equal(n1[0], n_mix[k]) and np.array_equal(m1[0], m_mix[k])


def test_mixed_input_kinds_in_one_call(torch, tfn, ctx):
    dep = depth_frames([(40, 52)], 1300)[0]
    inputs = [to_dev(torch, tfn, dep[0]), to_dev(torch, tfn, dep[0].astype(np.float16))]
    n, m = ctx.normals_batch(inputs, [dep[1], dep[1]])
    torch.cuda.synchronize()
    compare(n[0].cpu().numpy(), m[0].cpu().numpy(), dep[0], dep[1], grad="fd", phi="mean")
    compare(n[1].cpu().numpy(), m[1].cpu().numpy(), dep[0].astype(np.float16), dep[1], grad="fd", phi="mean")


@pytest.mark.parametrize("shape", [(1, 1), (2, 2), (3, 3), (1, 9), (9, 1), (3, 5)])
def test_tiny_images(torch, tfn, ctx, shape):
    rng = np.random.default_rng(1)
    img = rng.uniform(1, 2, size=shape).astype(np.float32)
    cam = dict(fx=3.0, fy=3.0, u0=(shape[1] - 1) / 2, v0=(shape[0] - 1) / 2)
    for grad in ("fd", "sobel"):
        for phi in PHIS:
            n, m = run_batch(torch, tfn, ctx, [(img, cam)], grad=grad, phi=phi)
            compare(n[0], m[0], img, cam, grad=grad, phi=phi)


@pytest.mark.parametrize("shape", [(3, 32768), (32768, 5)])
def test_maximum_extent_frames(torch, tfn, ctx, shape):
    # the largest width and height the ABI accepts (32768), on thin frames the oracle finishes quickly
    rng = np.random.default_rng(4)
    img = (3.0 + 0.002 * rng.standard_normal(shape)).astype(np.float32)
    img.ravel()[rng.integers(0, img.size, 50)] = 0.0
    cam = dict(fx=500.0, fy=480.0, u0=(shape[1] - 1) / 2, v0=(shape[0] - 1) / 2)
    for grad, phi in (("fd", "mean"), ("sobel", "median")):
        n, m = run_batch(torch, tfn, ctx, [(img, cam)], grad=grad, phi=phi)
        compare(n[0], m[0], img, cam, grad=grad, phi=phi)


def test_special_values_all_holes_constant(torch, tfn, ctx):
    H, W = 23, 37
    img = np.full((H, W), 2.5, np.float32)
    img[3, 4:11] = [np.nan, np.inf, -np.inf, -1.0, 0.0, 2.0 ** -17, 2.0 ** 17]
    img[10, 10] = 2.0 ** -16
    img[12, 12] = 2.0 ** 16
    cam = dict(fx=20.0, fy=21.0, u0=18.0, v0=11.0)
    for grad in GRADS:
        for phi in PHIS:
            n, m = run_batch(torch, tfn, ctx, [(img, cam)], grad=grad, phi=phi)
            compare(n[0], m[0], img, cam, grad=grad, phi=phi)
    holes = np.zeros((H, W), np.float32)
    n, m = run_batch(torch, tfn, ctx, [(holes, cam)], grad="fd", phi="mean")
    assert (m[0] == 0).all() and (n[0] == 0).all()


@pytest.mark.parametrize("kind", ["f32", "f16"])
def test_plateaus_give_exactly_the_special_case_at_the_default_shape(torch, tfn, ctx, kind):
    # The FD mean's kernel (one-pass gradients) gives a flat pixel its [0, 0, -1] without a test,
    # through n_z' = 2^-60 - Q: on 40 noisy 480x640 frames (the default tile shape) with constant-depth
    # plateaus, every evaluable pixel whose 4 axis neighbours share its depth must come out as exactly
    # (0, 0, -1), and every frame must still match the oracle.  FP16 depth runs the kernel without the
    # bound, FP32 the one with it (and its refinement queue).
    imgs = scenes.noisy_batch(40, seed0=980)
    for k, img in enumerate(imgs):
        y0, x0 = 37 + 9 * k, 41 + 11 * k
        img[y0:y0 + 60, x0:x0 + 90] = np.float32(1.25 + 0.125 * k)  # (exact in FP16 too)
        img[y0 + 70:y0 + 80, :] = np.float32(3.5)
    if kind == "f16":
        imgs = imgs.astype(np.float16)
    frames = [(img, scenes.CAMERA) for img in imgs]
    n, m = run_batch(torch, tfn, ctx, frames, grad="fd", phi="mean", output="f32")
    for k in (0, 17, 39):
        img = imgs[k]
        z = img.astype(np.float32)
        c = z[1:-1, 1:-1]
        flat = (z[1:-1, :-2] == c) & (z[1:-1, 2:] == c) & (z[:-2, 1:-1] == c) & (z[2:, 1:-1] == c)
        flat &= m[k][1:-1, 1:-1] == 1
        assert flat.sum() > 5000
        nk = n[k][:, 1:-1, 1:-1]
        assert (nk[0][flat] == 0.0).all() and (nk[1][flat] == 0.0).all() and (nk[2][flat] == -1.0).all()
        compare(n[k], m[k], img, scenes.CAMERA, grad="fd", phi="mean")


def test_invalid_arguments_are_rejected(torch, tfn, ctx):
    img = tfn.empty_image((16, 16), torch.float32)
    img.fill_(1.0)
    n = tfn.empty_normals(16, 16)
    m = tfn.empty_image((16, 16), torch.uint8)
    meth = tfn.make_method()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(**over):
        f = tfn.make_frame(img, n, m, dict(fx=10.0, fy=10.0, u0=8.0, v0=8.0))
        for k, v in over.items():
            setattr(f, k, v)
        return tfn.tfn_normals(ctx.handle, ctypes.byref(f), ctypes.byref(meth), s)

    assert call() == tfn.TFN_OK
    assert call(input_pitch=72) == tfn.TFN_ERR_MISALIGNED
    assert call(input=img.data_ptr() + 4) == tfn.TFN_ERR_MISALIGNED
    assert call(width=0) == tfn.TFN_ERR_INVALID_ARG
    assert call(input_type=9) == tfn.TFN_ERR_INVALID_ARG
    assert call(input=None) == tfn.TFN_ERR_INVALID_ARG
    f = tfn.make_frame(img, n, m, dict(fx=10.0, fy=11.0, u0=8.0, v0=8.0))
    f.input_type = tfn.TFN_DISP_F32
    assert tfn.tfn_normals(ctx.handle, ctypes.byref(f), ctypes.byref(meth), s) == tfn.TFN_ERR_UNSUPPORTED
    f = tfn.make_frame(img, n, m, dict(fx=float("nan"), fy=10.0, u0=8.0, v0=8.0))
    assert tfn.tfn_normals(ctx.handle, ctypes.byref(f), ctypes.byref(meth), s) == tfn.TFN_ERR_INVALID_ARG
    bad = tfn.make_method(grad=9)
    f = tfn.make_frame(img, n, m, dict(fx=10.0, fy=10.0, u0=8.0, v0=8.0))
    assert tfn.tfn_normals(ctx.handle, ctypes.byref(f), ctypes.byref(bad), s) == tfn.TFN_ERR_INVALID_ARG


def test_host_buffer_path_matches_device_path(torch, tfn, ctx):
    frames = depth_frames([(120, 160), (480, 640), (77, 90)], 1400)
    n_dev, m_dev = run_batch(torch, tfn, ctx, frames, grad="fd", phi="median")
    inputs = [torch.from_numpy(img).pin_memory() for img, _ in frames]
    normals = [torch.empty((3, img.shape[0], img.shape[1]), dtype=torch.float32).pin_memory() for img, _ in frames]
    masks = [torch.empty(img.shape, dtype=torch.uint8).pin_memory() for img, _ in frames]
    ctx.normals_batch_host(inputs, [c for _, c in frames], normals, masks, grad="fd", phi="median")
    for k in range(len(frames)):
        assert np.array_equal(normals[k].numpy(), n_dev[k]) and np.array_equal(masks[k].numpy(), m_dev[k])


def test_host_path_contiguous_batch_and_padded_views(torch, tfn, ctx):
    # a contiguous batch (copies merge into a few large ones) gives the device path's bits
    imgs = [img for img, _ in depth_frames([(96, 128)] * 6, 1450)]
    cam = small_recipe(96, 128).camera
    stack = torch.from_numpy(np.stack(imgs)).pin_memory()
    n_all = torch.empty((6, 3, 96, 128), dtype=torch.float32).pin_memory()
    m_all = torch.empty((6, 96, 128), dtype=torch.uint8).pin_memory()
    ctx.normals_batch_host([stack[k] for k in range(6)], cam, [n_all[k] for k in range(6)],
                           [m_all[k] for k in range(6)])
    n_dev, m_dev = run_batch(torch, tfn, ctx, [(x, cam) for x in imgs], grad="fd", phi="mean")
    for k in range(6):
        assert np.array_equal(n_all[k].numpy(), n_dev[k]) and np.array_equal(m_all[k].numpy(), m_dev[k])
    # outputs that are views with padding between rows: the padding keeps its bytes
    big_n = torch.full((6, 3, 96, 160), 7.0, dtype=torch.float32).pin_memory()
    big_m = torch.full((6, 96, 144), 9, dtype=torch.uint8).pin_memory()
    ctx.normals_batch_host([stack[k] for k in range(6)], cam, [big_n[k, :, :, :128] for k in range(6)],
                           [big_m[k, :, :128] for k in range(6)])
    assert (big_n[..., 128:] == 7.0).all() and (big_m[..., 128:] == 9).all()
    for k in range(6):
        assert np.array_equal(big_n[k, :, :, :128].numpy(), n_dev[k])
        assert np.array_equal(big_m[k, :, :128].numpy(), m_dev[k])


def test_host_path_stacks_over_many_chunks(torch, tfn, ctx):
    # the end-to-end call as the benchmark makes it: pinned stacks with a leading frame dimension, a
    # batch large enough to run through the three staging streams in several chunks (40 frames of
    # 480x640: 8 MB chunks of 6 frames, the last one partial), and per-frame intrinsics
    n = 40
    depth = scenes.noisy_batch(n, seed0=5000)
    hin = torch.from_numpy(depth).pin_memory()
    hn = torch.empty((n, 3, 480, 640), dtype=torch.float32).pin_memory()
    hm = torch.empty((n, 480, 640), dtype=torch.uint8).pin_memory()
    cams = [dict(scenes.CAMERA, fx=scenes.CAMERA["fx"] * (1 + 0.01 * k)) for k in range(n)]
    ctx.normals_batch_host(hin, cams, hn, hm, grad="fd", phi="mean")
    d = tfn.empty_image(depth.shape, torch.float32)
    d.copy_(hin)
    n_dev, m_dev = ctx.normals_batch([d[k] for k in range(n)], cams, grad="fd", phi="mean")
    torch.cuda.synchronize()
    for k in range(n):
        assert torch.equal(hn[k], n_dev[k].cpu()) and torch.equal(hm[k], m_dev[k].cpu()), f"frame {k}"
    # and the stack call gives the bits of the list-of-views call
    hn2 = torch.empty_like(hn).pin_memory()
    hm2 = torch.empty_like(hm).pin_memory()
    ctx.normals_batch_host([hin[k] for k in range(n)], cams, [hn2[k] for k in range(n)], [hm2[k] for k in range(n)])
    assert torch.equal(hn, hn2) and torch.equal(hm, hm2)


def test_full_batch_256_sampled_against_oracle(torch, tfn, ctx):
    # the benchmark's launch: 256 noisy 480x640 frames in one call; three
    # frames are compared with the oracle pixel by pixel, all frames for
    # properties that hold at any size.
    depth = scenes.noisy_batch(256)
    d = tfn.empty_image(depth.shape, torch.float32)
    d.copy_(torch.from_numpy(depth))
    normals = tfn.empty_normals(480, 640, lead=(256,))
    masks = tfn.empty_image((256, 480, 640), torch.uint8)
    ctx.normals_batch([d[k] for k in range(256)], scenes.CAMERA, normals=[normals[k] for k in range(256)],
                      masks=[masks[k] for k in range(256)])
    torch.cuda.synchronize()
    for k in (0, 97, 255):
        compare(normals[k].cpu().numpy(), masks[k].cpu().numpy(), depth[k], scenes.CAMERA, grad="fd", phi="mean")
    v = masks.bool()
    nn = (normals.float() ** 2).sum(1)
    assert torch.isfinite(normals).all()
    assert ((nn - 1).abs()[v] < 1e-5).all() and (nn[~v] == 0).all()
    border = torch.zeros((480, 640), dtype=torch.bool, device=v.device)
    border[0, :] = border[-1, :] = True
    border[:, 0] = border[:, -1] = True
    assert not v[:, border].any()


def test_disparity_batch_256_sampled_against_oracle(torch, tfn, ctx):
    # the u16 disparity workload in the bench's launch: 256 frames, 1/16 px, 5% zeros, FD median
    raw = scenes.disparity_batch(256)
    st = scenes.STEREO
    cam = dict(fx=st["f"], fy=st["f"], u0=st["u0"], v0=st["v0"], baseline=st["baseline"])
    dd = tfn.empty_image(raw.shape, torch.int16)
    dd.copy_(torch.from_numpy(raw.view(np.int16)))
    n, m = ctx.normals_batch([dd[k] for k in range(256)], cam, grad="fd", phi="median", disparity=True)
    torch.cuda.synchronize()
    for k in (0, 131, 255):
        compare(n[k].cpu().numpy(), m[k].cpu().numpy(), raw[k], cam, grad="fd", phi="median", disparity=True,
                baseline=st["baseline"])


def test_fp16_batch_1024_sampled_against_oracle(torch, tfn, ctx):
    # the precision form's launch: 1024 FP16 480x640 frames; FP32 normals held to the 1e-3 deg rule on the
    # FP16-decoded depth, FP16 normals within 0.05 deg on average per frame
    import oracle
    depth16 = scenes.fp16_batch(1024)
    d16 = tfn.empty_image(depth16.shape, torch.float16)
    d16.copy_(torch.from_numpy(depth16))
    ins = [d16[k] for k in range(1024)]
    n32, m32 = ctx.normals_batch(ins, scenes.CAMERA)
    n16, m16 = ctx.normals_batch(ins, scenes.CAMERA, output="f16")
    torch.cuda.synchronize()
    for k in (5, 1000):
        compare(n32[k].cpu().numpy(), m32[k].cpu().numpy(), depth16[k], scenes.CAMERA, grad="fd", phi="mean")
        ref, rm = oracle.normals(depth16[k], **scenes.CAMERA)
        assert torch.equal(m16[k], m32[k])
        ang = oracle.angle_deg(n16[k].cpu().numpy().astype(np.float64), ref)[rm == 1]
        assert ang.mean() < 0.05, ang.mean()


def test_plan_graph_replay_matches_batch(torch, tfn, ctx):
    # a frozen batch replayed as a CUDA graph gives the same bits as the direct call
    frames = depth_frames([(67, 131), (480, 640), (33, 64)], 1500)
    inputs = [to_dev(torch, tfn, img) for img, _ in frames]
    cams = [cam for _, cam in frames]
    n_ref, m_ref = ctx.normals_batch(inputs, cams, grad="sobel", phi="median")
    plan = ctx.plan(inputs, cams, grad="sobel", phi="median")
    s = torch.cuda.Stream()
    for _ in range(3):
        for x in plan.normals:
            x.zero_()
        plan.launch(s)
        s.synchronize()
        for a, b, ma, mb in zip(plan.normals, n_ref, plan.masks, m_ref):
            assert torch.equal(a, b) and torch.equal(ma, mb)
    # the plan reads the caller's buffers at each launch: new input, new result
    inputs[0].mul_(2.0)  # a global depth scale leaves the normals unchanged
    inputs[1].copy_(torch.from_numpy(depth_frames([(480, 640)], 1600)[0][0]))
    plan.launch(s)
    s.synchronize()
    assert torch.equal(plan.normals[0], n_ref[0])
    compare(plan.normals[1].cpu().numpy(), plan.masks[1].cpu().numpy(), inputs[1].cpu().numpy(), cams[1],
            grad="sobel", phi="median")
    plan.close()


@pytest.mark.parametrize("grad,phi", [("fd", "mean"), ("scharr", "median"), ("sobel", "mean"), ("prewitt", "median")])
def test_tile_shapes_give_identical_bits(torch, tfn, grad, phi):
    # every compiled tile shape (the autotuner's choices) computes the same bits; (sobel, mean) keeps
    # the rows' tap differences in the shared-memory ring, the medians compute them per row
    frames = depth_frames([(67, 131), (480, 640), (33, 64)], 1700)
    inputs = [to_dev(torch, tfn, img) for img, _ in frames]
    cams = [cam for _, cam in frames]
    ref = None
    with tfn.Context(0) as c:
        for shape in range(tfn.tfn_tile_shape_count()):
            c.set_tile_shape(shape)
            n, m = c.normals_batch(inputs, cams, grad=grad, phi=phi)
            torch.cuda.synchronize()
            got = [x.cpu() for x in n] + [x.cpu() for x in m]
            if ref is None:
                ref = got
                compare(n[1].cpu().numpy(), m[1].cpu().numpy(), frames[1][0], cams[1], grad=grad, phi=phi)
            else:
                assert all(torch.equal(a, b) for a, b in zip(got, ref)), f"tile shape {shape} differs"
        assert c.device_status() == 0
