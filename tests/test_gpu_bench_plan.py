"""Parity of the exact call the benchmark times.

bench.py's step replays a plan: the 256 noisy 480x640 frames, their
descriptors uploaded once, the kernels captured in a CUDA graph.  At that size
the launch takes the default tile shape.  For the FD mean (the benchmark's
method) normals_kernel refines its flagged pixels itself, through a per-warp
queue that must start empty on every replay; for the Sobel median the
refinement kernel runs inside the graph and its list's count must be reset
between replays (the kernel's last block does it).  Each replay is checked
against the FP64 oracle on sampled frames and bit for bit against
tfn_normals_batch on every frame.
"""
import numpy as np
import pytest

import scenes
from tests.parity import compare

pytestmark = pytest.mark.gpu

N = 256
H, W = 480, 640


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


@pytest.fixture(scope="module")
def batch(torch):
    import paper_2005_08165_gb300 as tfn
    depth = scenes.noisy_batch(N)
    d = tfn.empty_image(depth.shape, torch.float32)
    d.copy_(torch.from_numpy(depth))
    return depth, d


@pytest.mark.parametrize("grad,phi", [("fd", "mean"), ("sobel", "median")])
def test_bench_plan_replays_match_oracle_and_batch(torch, batch, grad, phi):
    import paper_2005_08165_gb300 as tfn
    depth, d = batch
    cam = scenes.CAMERA
    with tfn.Context(0) as ctx:
        normals = tfn.empty_normals(H, W, "f32", lead=(N,))
        masks = tfn.empty_image((N, H, W), torch.uint8)
        ins = [d[k] for k in range(N)]
        plan = ctx.plan(ins, cam, grad=grad, phi=phi, normals=[normals[k] for k in range(N)],
                        masks=[masks[k] for k in range(N)])
        ref_n, ref_m = ctx.normals_batch(ins, cam, grad=grad, phi=phi)
        ref_n = torch.stack(ref_n)
        ref_m = torch.stack(ref_m)
        ctx.refined_pixels()
        refined = []
        for replay in range(3):
            normals.fill_(7.0)  # a replay must write every output again
            masks.fill_(7)
            plan.launch()
            torch.cuda.synchronize()
            refined.append(ctx.refined_pixels())
            assert torch.equal(masks, ref_m), f"replay {replay}: masks differ from tfn_normals_batch"
            assert torch.equal(normals, ref_n), f"replay {replay}: normals differ from tfn_normals_batch"
            n_np = normals.cpu().numpy()
            m_np = masks.cpu().numpy()
            for k in (0, 97, 255):
                compare(n_np[k], m_np[k], depth[k], cam, grad=grad, phi=phi)
        plan.close()
        assert ctx.device_status() == 0
        # every replay refines the same pixels (the list is reset between replays)
        assert refined[0] == refined[1] == refined[2]
        if phi == "mean":
            assert refined[0] > 0, "the noisy batch flags pixels for the double-float path"
    np.testing.assert_equal(refined[0], refined[2])
