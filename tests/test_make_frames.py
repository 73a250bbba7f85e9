"""The binding's batch descriptors: a stack (a leading frame dimension) must give the same tfn_frame
bytes as the list of its per-frame views, for every output layout, with and without the fused point
cloud, with one camera or one per frame.  Host-side only (CPU tensors; no kernel runs)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
tfn = pytest.importorskip("paper_2005_08165_gb300")


def _bytes(frames, n, ptr):
    size = n * ctypes.sizeof(tfn.tfn_frame)
    if isinstance(frames, np.ndarray):
        return ctypes.string_at(ctypes.cast(ptr, ctypes.c_void_p), size)
    return ctypes.string_at(ctypes.addressof(frames), size)


@pytest.mark.parametrize("output", ["f32", "f16", "bf16", "oct16", "f16x4", "bf16x4"])
@pytest.mark.parametrize("kind", ["depth_f32", "depth_f16", "disp_u16"])
def test_stack_matches_per_frame_views(output, kind):
    n, H, W = 5, 7, 13
    dt = {"depth_f32": torch.float32, "depth_f16": torch.float16, "disp_u16": torch.int16}[kind]
    disparity = kind == "disp_u16"
    inp = torch.zeros((n, H, 16), dtype=dt)[..., :W]  # a pitched stack
    nrm = tfn.empty_normals(H, W, output, "cpu", lead=(n,))
    msk = torch.zeros((n, H, W), dtype=torch.uint8)
    pts = tfn.empty_points(H, W, "cpu", lead=(n,))
    cams = [dict(fx=50.0 + k, fy=51.0 + k, u0=6.5, v0=3.25 + k, baseline=0.1 * (k + 1)) for k in range(n)]
    for cam in (dict(fx=48.0, fy=47.0, u0=6.0, v0=3.0), cams):
        for P in (None, pts):
            a, na, pa = tfn.make_frames(inp, nrm, msk, cam, disparity, 1.0 / 16, output, P)
            b, nb, pb = tfn.make_frames([inp[k] for k in range(n)], [nrm[k] for k in range(n)],
                                        [msk[k] for k in range(n)], cam, disparity, 1.0 / 16, output,
                                        None if P is None else [P[k] for k in range(n)])
            assert isinstance(a, np.ndarray) and not isinstance(b, np.ndarray)
            assert na == nb == n
            assert _bytes(a, na, pa) == _bytes(b, nb, pb)


def test_single_frame_and_mismatched_stacks_take_the_list_path():
    inp = torch.zeros((1, 4, 4), dtype=torch.float32)
    nrm = tfn.empty_normals(4, 4, "f32", "cpu", lead=(1,))
    msk = torch.zeros((1, 4, 4), dtype=torch.uint8)
    cam = dict(fx=4.0, fy=4.0, u0=1.5, v0=1.5)
    frames, n, _ = tfn.make_frames(inp, nrm, msk, cam)
    assert n == 1 and not isinstance(frames, np.ndarray)
    inp2 = torch.zeros((3, 4, 4), dtype=torch.float32)
    nrm2 = tfn.empty_normals(4, 4, "f32", "cpu", lead=(2,))  # one frame short
    msk2 = torch.zeros((3, 4, 4), dtype=torch.uint8)
    with pytest.raises(IndexError):
        tfn.make_frames(inp2, nrm2, msk2, cam)
