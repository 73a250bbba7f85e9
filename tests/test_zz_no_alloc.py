"""tfn_normals_noalloc, the entry point for callers that may not allocate.

Some callers run under a fixed device-memory plan (a host framework that owns
every device byte, or a loop that must not call cudaMalloc because it can
synchronise the device) and cannot create a context.  These tests check,
through the C ABI, that the allocation-free entry point gives exactly the
normals and masks of tfn_normals_batch on calls in a row (a later call must
not see an earlier call's leftovers in the shared scratch array), including a
call large enough to take the default tile shape (for the Scharr median the
refinement kernel and the scratch's refinement list, for the FD mean the
kernel's own refinement queue); that one of its frames matches the FP64
oracle; that it refuses more frames than its scratch holds; and that it
refuses to run while its stream is being captured.  The file is named so that
pytest runs it last.
"""
import ctypes

import pytest

import scenes
from tests.parity import compare

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
        img = scenes.render(seed + k, r)
        d = tfn.empty_image((H, W), torch.float32)
        d.copy_(torch.from_numpy(img))
        out.append((d, r.camera, img))
    return out


def _prepare(torch, tfn, frames, grad, phi):
    normals = [tfn.empty_normals(d.shape[0], d.shape[1]) for d, _, _ in frames]
    masks = [tfn.empty_image(tuple(d.shape), torch.uint8) for d, _, _ in frames]
    arr = (tfn.tfn_frame * len(frames))(*[tfn.make_frame(d, n, m, cam) for (d, cam, _), n, m in
                                           zip(frames, normals, masks)])
    return arr, tfn.make_method(grad, phi), normals, masks


def _call(tfn, arr, meth, stream):
    return tfn.tfn_normals_noalloc(arr, len(arr), ctypes.byref(meth), ctypes.c_void_p(stream.cuda_stream))


def _noalloc(torch, tfn, frames, grad, phi):
    arr, meth, normals, masks = _prepare(torch, tfn, frames, grad, phi)
    return _call(tfn, arr, meth, torch.cuda.current_stream()), normals, masks


# call 1: three small frames of mixed sizes (the short-item shape, refining in place);
# call 2: 40 full frames (the default shape; Scharr median: refinement kernel and the scratch's list);
# call 3: five small frames again, after the large call's list use
CALLS = [(7100, [(67, 131), (480, 640), (33, 64)]), (7200, [(480, 640)] * 40), (7300, [(120, 96)] * 5)]


@pytest.mark.parametrize("grad,phi", [("fd", "mean"), ("scharr", "median")])
def test_noalloc_matches_batch_bit_for_bit_on_calls_in_a_row(torch, grad, phi):
    import paper_2005_08165_gb300 as tfn
    with tfn.Context(0) as ctx:
        for seed, sizes in CALLS:
            frames = _frames(torch, tfn, seed, sizes)
            n_ref, m_ref = ctx.normals_batch([d for d, _, _ in frames], [c for _, c, _ in frames], grad=grad, phi=phi)
            st, n_na, m_na = _noalloc(torch, tfn, frames, grad, phi)
            assert st == tfn.TFN_OK, tfn.tfn_status_string(st)
            torch.cuda.synchronize()
            for a, b, ma, mb in zip(n_na, n_ref, m_na, m_ref):
                assert torch.equal(ma, mb)
                assert torch.equal(a, b)
            if len(frames) == 40:
                # one frame of the large call against the FP64 oracle
                k = 17
                compare(n_na[k].cpu().numpy(), m_na[k].cpu().numpy(), frames[k][2], frames[k][1], grad=grad, phi=phi)


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


def test_noalloc_refuses_a_capturing_stream(torch):
    import paper_2005_08165_gb300 as tfn
    frames = _frames(torch, tfn, 7400, [(64, 128)])
    assert _noalloc(torch, tfn, frames, "fd", "mean")[0] == tfn.TFN_OK  # the first call on the device: its set-up
    torch.cuda.synchronize()
    arr, meth, _, _ = _prepare(torch, tfn, frames, "fd", "mean")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    z = torch.zeros(1, device="cuda")
    with torch.cuda.graph(g, stream=s):
        z.add_(1.0)  # (a captured graph must not be empty)
        st = _call(tfn, arr, meth, s)
    assert st == tfn.TFN_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    # and the next ordinary call works
    st, n, m = _noalloc(torch, tfn, frames, "fd", "mean")
    assert st == tfn.TFN_OK
    torch.cuda.synchronize()
    compare(n[0].cpu().numpy(), m[0].cpu().numpy(), frames[0][2], frames[0][1], grad="fd", phi="mean")
