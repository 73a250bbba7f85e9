"""The device-side failure path: a bounded wait that runs out.

Every wait of the kernels on a TMA copy is bounded; when one gives up, the
warp sets a bit in the status word and leaves.  TFN_FLAG_TEST_WAIT_TIMEOUT
makes the first warp of a launch wait, before it issues any copy, on a
barrier that nothing completes, so the give-up path runs with no copy in
flight and no fault.  These tests check that such a launch returns, that the
status word reports the failed wait, that the context stays usable, and that
a server fails exactly the batch whose launch gave up while the next batch
succeeds.
"""
import numpy as np
import pytest

import scenes
from tests.parity import compare

pytestmark = pytest.mark.gpu

DEVERR_TMA_WAIT = 1


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def _frame(torch, tfn, seed, H=120, W=200):
    f = 481.2 * W / 640
    r = scenes.Recipe(H=H, W=W, fx=f, fy=f, u0=(W - 1) / 2, v0=(H - 1) / 2, noise_k=0.0012, hole_frac=0.03)
    img = scenes.render(seed, r)
    d = tfn.empty_image((H, W), torch.float32)
    d.copy_(torch.from_numpy(img))
    return img, d, r.camera


@pytest.mark.parametrize("grad,phi", [("fd", "mean"), ("sobel", "median")])
def test_failed_wait_is_reported_and_the_context_stays_usable(torch, grad, phi):
    import paper_2005_08165_gb300 as tfn
    img, d, cam = _frame(torch, tfn, 8100)
    with tfn.Context(0) as ctx:
        assert ctx.device_status() == 0
        ctx.normals_batch([d, d], cam, grad=grad, phi=phi, flags=tfn.TFN_FLAG_TEST_WAIT_TIMEOUT)
        torch.cuda.synchronize()
        assert ctx.device_status() == DEVERR_TMA_WAIT
        assert ctx.device_status() == 0, "reading the status word clears it"
        # the same context computes the next launch correctly
        n, m = ctx.normals(d, cam, grad=grad, phi=phi)
        torch.cuda.synchronize()
        assert ctx.device_status() == 0
        compare(n.cpu().numpy(), m.cpu().numpy(), img, cam, grad=grad, phi=phi)


def test_server_fails_only_the_batch_that_gave_up(torch):
    import paper_2005_08165_gb300 as tfn
    img, d, cam = _frame(torch, tfn, 8200)
    with tfn.Context(0) as ctx:
        n_ref, m_ref = ctx.normals(d, cam)
        torch.cuda.synchronize()
        with tfn.Server(ctx, grad="fd", phi="mean") as srv:
            outs = []
            for k, fl in enumerate((tfn.TFN_REQ_TEST_WAIT_TIMEOUT, 0, tfn.TFN_REQ_TEST_WAIT_TIMEOUT, 0)):
                n = tfn.empty_normals(img.shape[0], img.shape[1])
                m = tfn.empty_image(img.shape, torch.uint8)
                t = srv.submit(d, cam, n, m, flags=fl)
                # one request per batch: wait before submitting the next
                st = srv.wait(t, timeout_ms=10000)
                outs.append((st, n, m))
            stats = srv.stats()
        assert [st for st, _, _ in outs] == [tfn.TFN_ERR_DEVICE, tfn.TFN_OK] * 2
        assert stats["failed"] == 2 and stats["completed"] == 2
        for st, n, m in outs[1::2]:
            assert torch.equal(n, n_ref) and torch.equal(m, m_ref)
        assert ctx.device_status() == 0, "the server's batches report to their own status words"
    np.testing.assert_array_equal(m_ref.cpu().numpy() <= 1, True)
