"""tfn_normals_noalloc, the entry point for callers that may not allocate.

Some callers run under a fixed device-memory plan (a host framework that owns
every device byte, or a latency-critical loop where cudaMalloc could stall
the device) and cannot create a context.  This checks, through the C ABI,
that the allocation-free entry point gives the same normals and masks as
tfn_normals_batch on two calls in a row (the second must not see the first
call's leftovers in the shared scratch array), and that it refuses more
frames than its fixed scratch holds.  The file is named so that pytest runs
it last.
"""
import ctypes

import numpy as np
import pytest

import scenes
from tests.parity import TOL_DEG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def _frames(torch, tfn, seed, sizes):
    out = []
    for k, (H, W) in enumerate(sizes):
        f = 481.2 * W / 640
        r = scenes.Recipe(H=H, W=W, fx=f, fy=f, u0=(W - 1) / 2, v0=(H - 1) / 2, noise_k=0.0012, hole_frac=0.03)
        d = tfn.empty_image((H, W), torch.float32)
        d.copy_(torch.from_numpy(scenes.render(seed + k, r)))
        out.append((d, r.camera))
    return out


def _noalloc(torch, tfn, frames, grad, phi):
    normals = [tfn.empty_normals(d.shape[0], d.shape[1]) for d, _ in frames]
    masks = [tfn.empty_image(tuple(d.shape), torch.uint8) for d, _ in frames]
    arr = (tfn.tfn_frame * len(frames))(*[tfn.make_frame(d, n, m, cam) for (d, cam), n, m in
                                           zip(frames, normals, masks)])
    meth = tfn.make_method(grad, phi)
    st = tfn.tfn_normals_noalloc(arr, len(frames), ctypes.byref(meth),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == tfn.TFN_OK, tfn.tfn_status_string(st)
    torch.cuda.synchronize()
    return normals, masks


def _angle_deg(a, b):
    a = a.double().numpy()
    b = b.double().numpy()
    cr = np.cross(a, b, axis=0)
    return np.degrees(np.arctan2(np.sqrt((cr ** 2).sum(0)), (a * b).sum(0)))


@pytest.mark.parametrize("grad,phi", [("fd", "mean"), ("scharr", "median")])
def test_noalloc_matches_batch_on_two_calls(torch, grad, phi):
    import paper_2005_08165_gb300 as tfn
    with tfn.Context(0) as ctx:
        for call, seed in enumerate((7100, 7200)):
            frames = _frames(torch, tfn, seed, [(67, 131), (480, 640), (33, 64)] if call == 0 else [(120, 96)] * 5)
            n_ref, m_ref = ctx.normals_batch([d for d, _ in frames], [c for _, c in frames], grad=grad, phi=phi)
            n_na, m_na = _noalloc(torch, tfn, frames, grad, phi)
            for a, b, ma, mb in zip(n_na, n_ref, m_na, m_ref):
                assert torch.equal(ma, mb)
                v = mb.bool().cpu()
                ang = _angle_deg(a.cpu(), b.cpu())
                assert (ang[v.numpy()] <= TOL_DEG).all()
                assert (a.cpu()[:, ~v] == 0).all()


def test_noalloc_rejects_more_frames_than_its_scratch(torch):
    import paper_2005_08165_gb300 as tfn
    d = tfn.empty_image((8, 8), torch.float32)
    d.fill_(1.0)
    n = tfn.empty_normals(8, 8)
    m = tfn.empty_image((8, 8), torch.uint8)
    count = tfn.TFN_NOALLOC_MAX_FRAMES + 1
    arr = (tfn.tfn_frame * count)(*[tfn.make_frame(d, n, m, dict(fx=5.0, fy=5.0, u0=4.0, v0=4.0))] * count)
    meth = tfn.make_method()
    assert tfn.tfn_normals_noalloc(arr, count, ctypes.byref(meth), None) == tfn.TFN_ERR_INVALID_ARG
