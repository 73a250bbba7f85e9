"""The FP16 depth kind's kernel without the error bound.

For binary16 depth with the FD filter, two distinct samples a < b differ by at least one ulp of a,
which is at least 2^-11 a, so |rho_j| = Z_j / |Z_j - Z_i| <= 2^11 + 1 for every kept neighbour and
a pixel's bound / |n'| is at most c (2^11 + 1) / min(fx, fy) (c = 1.3 sqrt(2) for the mean, sqrt(2)
for the median), whatever the depths.  Where that is below the refinement threshold (every frame of
the launch), the library runs a kernel that computes neither the bound nor the refinement test and
launches no refinement kernel.  These tests check:

- the premise: with TFN_FLAG_FULL_BOUND (the bound computed as for every other kind) no pixel is
  ever flagged on qualifying FP16 frames, including adversarial ones built to make rho large
  (one-ulp steps just below a power of two, ramps of single-ulp increments, values across a binade
  boundary, the subnormal range, holes beside them) and the noisy scene batch;
- the promise: the kernel without the bound gives the same normals and masks, bit for bit, for the
  mean and the median, FP32 and FP16 output, the default and the short-item tile shapes;
- which kernel ran, by the names of the kernels a plan replays: a qualifying plan runs the form
  without the bound (its NOREF template argument true), the same plan with TFN_FLAG_FULL_BOUND the
  form with it, and so does a plan whose focal length is too short to qualify; for the median the
  bound form is also followed by the refinement kernel (the FD mean's kernel refines its own pixels);
- accuracy: the adversarial frames match the FP64 oracle under the usual 1e-3 degree rule.
"""
import numpy as np
import pytest

import scenes
from tests.parity import compare

pytestmark = pytest.mark.gpu

H, W = 480, 640
CAM = scenes.CAMERA  # f = 481.2: qualifies (7.8 < 11.7 for the mean, 6.0 < 19.1 for the median)


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


@pytest.fixture(scope="module")
def tfn(torch):
    import paper_2005_08165_gb300 as tfn
    return tfn


@pytest.fixture(scope="module")
def ctx(tfn):
    c = tfn.Context(0)
    yield c
    c.close()


def _holes(rng, z, frac=0.03):
    z = z.copy()
    z[rng.random(z.shape) < frac] = 0.0
    return z


def adversarial_frames(seed=0):
    """FP16 depth images that make |rho| large: neighbours one ulp apart where the ulp is smallest
    relative to the value."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    u = 2.0 ** -10  # ulp of binary16 in [1, 2)
    out = []
    # one-ulp noise just below 2 (rho up to about 2^11)
    z = 2.0 - u * (1 + rng.integers(0, 4, size=(H, W)))
    out.append(_holes(rng, z).astype(np.float16))
    # a ramp of single-ulp increments in both directions, tilted
    z = 1.25 + u * (xx // 3 + yy // 5)
    out.append(_holes(rng, z).astype(np.float16))
    # values on both sides of the binade boundary at 2 (spacing 2^-10 below, 2^-9 above)
    z = np.where((xx + yy) % 2 == 0, 2.0 - u, 2.0) + 2 * u * (rng.random((H, W)) < 0.3)
    out.append(_holes(rng, z).astype(np.float16))
    # the subnormal binary16 range (spacing 2^-24, values from 2^-16)
    z = 2.0 ** -15 + 2.0 ** -24 * rng.integers(0, 5, size=(H, W))
    out.append(_holes(rng, z).astype(np.float16))
    # a steep slope with one-ulp steps across it at depth 100 (ulp 2^-4)
    z = 100.0 + 2.0 ** -4 * ((7 * xx + yy) // 4 % 3)
    out.append(_holes(rng, z).astype(np.float16))
    return out


def to_dev(torch, tfn, img):
    t = tfn.empty_image(img.shape, torch.float16)
    t.copy_(torch.from_numpy(img))
    return t


def run(torch, tfn, ctx, ins, cam, *, phi, output, flags):
    ctx.refined_pixels()  # (reading the counter restarts it)
    n, m = ctx.normals_batch(ins, cam, grad="fd", phi=phi, output=output, flags=flags)
    torch.cuda.synchronize()
    return n, m, ctx.refined_pixels()


@pytest.mark.parametrize("phi", ["mean", "median"])
@pytest.mark.parametrize("output", ["f32", "f16"])
@pytest.mark.parametrize("batch", [1, 40])  # one frame: the short-item shape; 40: the default shape
def test_without_the_bound_same_bits_and_the_bound_never_fires(torch, tfn, ctx, phi, output, batch):
    adv = adversarial_frames(11)
    noisy = scenes.noisy_batch(max(0, batch - len(adv)) or 1, seed0=4000).astype(np.float16)
    imgs = (adv + list(noisy))[:batch]
    ins = [to_dev(torch, tfn, img) for img in imgs]
    n0, m0, r0 = run(torch, tfn, ctx, ins, CAM, phi=phi, output=output, flags=0)
    n1, m1, r1 = run(torch, tfn, ctx, ins, CAM, phi=phi, output=output, flags=tfn.TFN_FLAG_FULL_BOUND)
    assert r0 == 0
    assert r1 == 0, f"the bound flagged {r1} pixels of binary16 frames that qualify"
    for k in range(batch):
        assert torch.equal(m0[k], m1[k]), k
        assert torch.equal(n0[k], n1[k]), k
    assert ctx.device_status() == 0


@pytest.mark.parametrize("phi", ["mean", "median"])
def test_adversarial_frames_match_the_oracle(torch, tfn, ctx, phi):
    imgs = adversarial_frames(12)
    ins = [to_dev(torch, tfn, img) for img in imgs]
    n, m, _ = run(torch, tfn, ctx, ins, CAM, phi=phi, output="f32", flags=0)
    for k, img in enumerate(imgs):
        compare(n[k].cpu().numpy(), m[k].cpu().numpy(), img, CAM, grad="fd", phi=phi)


def _plan_kernels(torch, tfn, ctx, ins, cam, flags, phi="mean"):
    outs = [tfn.empty_normals(H, W, "f16") for _ in ins]
    masks = [tfn.empty_image((H, W), torch.uint8) for _ in ins]
    plan = ctx.plan(ins, cam, grad="fd", phi=phi, output="f16", normals=outs, masks=masks, flags=flags)
    try:
        k = plan.kernel_names()
        plan.launch()
        torch.cuda.synchronize()
    finally:
        plan.close()
    return k, outs, masks


def _forms(names):
    # per kernel: "noref" (normals_kernel<..., NOREF = true>), "bound" (NOREF = false) or "refine"
    out = []
    for nm in names:
        if "normals_kernel" in nm:
            assert ("Lb1EEEv" in nm) != ("Lb0EEEv" in nm), nm
            out.append("noref" if "Lb1EEEv" in nm else "bound")
        else:
            assert "refine_kernel" in nm, nm
            out.append("refine")
    return out


@pytest.mark.parametrize("phi", ["mean", "median"])
def test_which_kernel_runs(torch, tfn, ctx, phi):
    imgs = scenes.noisy_batch(40, seed0=4100).astype(np.float16)
    ins = [to_dev(torch, tfn, img) for img in imgs]
    bound = ["bound"] if phi == "mean" else ["bound", "refine"]  # (the FD mean refines in its own kernel)
    k0, n0, m0 = _plan_kernels(torch, tfn, ctx, ins, CAM, 0, phi)
    k1, n1, m1 = _plan_kernels(torch, tfn, ctx, ins, CAM, tfn.TFN_FLAG_FULL_BOUND, phi)
    assert (_forms(k0), _forms(k1)) == (["noref"], bound)
    assert all(torch.equal(a, b) for a, b in zip(n0, n1)) and all(torch.equal(a, b) for a, b in zip(m0, m1))
    # a focal length too short for the proof (1.84 x 2049 / 150 = 25 > the threshold): the bound kernel runs
    short = dict(CAM, fx=150.0, fy=150.0)
    ks, _, _ = _plan_kernels(torch, tfn, ctx, ins, short, 0, phi)
    assert _forms(ks) == bound
    # FP32 depth never qualifies
    d32 = [tfn.empty_image((H, W), torch.float32) for _ in range(40)]
    for t, img in zip(d32, imgs):
        t.copy_(torch.from_numpy(img.astype(np.float32)))
    outs = [tfn.empty_normals(H, W, "f32") for _ in d32]
    masks = [tfn.empty_image((H, W), torch.uint8) for _ in d32]
    plan = ctx.plan(d32, CAM, grad="fd", phi=phi, normals=outs, masks=masks)
    assert _forms(plan.kernel_names()) == bound and plan.kernels() == len(bound)
    plan.close()


def test_short_focal_length_frames_still_refine_correctly(torch, tfn, ctx):
    # the same adversarial depths seen through a short lens: the bound kernel runs and refines
    short = dict(CAM, fx=120.0, fy=120.0)
    imgs = adversarial_frames(13)
    ins = [to_dev(torch, tfn, img) for img in imgs]
    n, m, refined = run(torch, tfn, ctx, ins, short, phi="mean", output="f32", flags=0)
    for k, img in enumerate(imgs):
        compare(n[k].cpu().numpy(), m[k].cpu().numpy(), img, short, grad="fd", phi="mean")
