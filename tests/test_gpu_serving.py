"""The serving form (request server with continuous batching and memory-budget
admission) and the tile-shape autotuner, through the C ABI."""
import ctypes
import os
import threading

import numpy as np
import pytest

import scenes
from tests.parity import compare

pytestmark = pytest.mark.gpu


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
    c.close()


def request_mix(n, seed):
    """Mixed resolutions, FP32/FP16 depth, per-request intrinsics (fx = fy = 481.2 W/640 x U(0.95, 1.05))."""
    rng = np.random.default_rng(seed)
    sizes = [(240, 320), (480, 640), (67, 131), (720, 1280)]
    out = []
    for k in range(n):
        H, W = sizes[rng.integers(len(sizes))]
        f = 481.2 * W / 640 * rng.uniform(0.95, 1.05)
        r = scenes.Recipe(H=H, W=W, fx=f, fy=f, u0=(W - 1) / 2, v0=(H - 1) / 2, noise_k=0.0012, hole_frac=0.03)
        img = scenes.render(seed * 1000 + k, r)
        if rng.integers(2):
            img = img.astype(np.float16)
        out.append((img, r.camera))
    return out


def host_image(torch, tfn, img):
    """Page-locked host copy (host requests need no row alignment)."""
    return torch.from_numpy(np.ascontiguousarray(img)).pin_memory()


def dev_image(torch, tfn, img):
    dt = torch.float16 if img.dtype == np.float16 else torch.float32
    t = tfn.empty_image(img.shape, dt)
    t.copy_(torch.from_numpy(img))
    return t


def submit_all(torch, tfn, srv, reqs, host_every=2):
    """Submits every request (alternately host and device buffers); returns [(ticket, normals, mask)]."""
    out = []
    for k, (img, cam) in enumerate(reqs):
        H, W = img.shape
        host = k % host_every == 0
        if host:
            inp = host_image(torch, tfn, img)
            n = torch.empty((3, H, W), dtype=torch.float32, pin_memory=True)
            m = torch.empty((H, W), dtype=torch.uint8, pin_memory=True)
        else:
            inp = dev_image(torch, tfn, img)
            n = tfn.empty_normals(H, W, "f32")
            m = tfn.empty_image((H, W), torch.uint8)
        t = srv.submit(inp, cam, n, m, host=host)
        out.append((t, n, m))
    return out


@pytest.mark.parametrize("graphs", [True, False])
def test_results_in_the_mix_equal_results_alone(torch, tfn, ctx, graphs):
    # (with graphs, a batch's kernels are replayed from a pipeline's CUDA graph, one per launch
    # structure, its kernel nodes updated to the batch; without, they are launched directly)
    reqs = request_mix(24, 11)
    with tfn.Server(ctx, grad="sobel", phi="median", max_batch=8, graphs=graphs) as srv:
        subs = submit_all(torch, tfn, srv, reqs)
        for t, _, _ in subs:
            assert srv.wait(t, 20000) == tfn.TFN_OK
        st = srv.stats()
    assert st["completed"] == 24 and st["failed"] == 0 and st["batches"] >= 3  # at most 8 per batch
    assert st["graph_launches"] == (st["batches"] if graphs else 0)
    assert 0 < st["latency_p50_us"] <= st["latency_p99_us"] <= st["latency_max_us"]
    torch.cuda.synchronize()
    for (img, cam), (_, n, m) in zip(reqs, subs):
        alone_n, alone_m = ctx.normals(dev_image(torch, tfn, img), cam, grad="sobel", phi="median")
        torch.cuda.synchronize()
        assert torch.equal(n.cpu(), alone_n.cpu()) and torch.equal(m.cpu(), alone_m.cpu())
    # and the served results are the estimator's (oracle parity on two of them)
    for k in (0, 1):
        img, cam = reqs[k]
        compare(subs[k][1].cpu().numpy(), subs[k][2].cpu().numpy(), img, cam, grad="sobel", phi="median")


def test_concurrent_clients(torch, tfn, ctx):
    reqs = request_mix(40, 12)
    results = {}
    with tfn.Server(ctx, grad="fd", phi="mean", pipelines=3, max_delay_us=200) as srv:
        def client(cid):
            mine = reqs[cid::4]
            subs = submit_all(torch, tfn, srv, mine, host_every=1 + cid % 2)
            results[cid] = [srv.wait(t, 20000) for t, _, _ in subs]

        threads = [threading.Thread(target=client, args=(c,)) for c in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        st = srv.stats(reset=True)
        st2 = srv.stats()
    assert all(s == tfn.TFN_OK for r in results.values() for s in r) and sum(map(len, results.values())) == 40
    assert st["completed"] == 40 and st["submitted"] == 40 and st["queued"] == 0 and st["in_flight"] == 0
    assert st["staging_bytes_in_use"] == 0 and st["mean_batch_frames"] >= 1
    assert st2["completed"] == 0 and st2["latency_samples"] == 0  # reset


def test_batches_overlap_on_the_device(torch, tfn, ctx):
    # continuous batching: requests that arrive while batches run are admitted into the next batch
    # before the running ones retire, several batches are in flight at once, and their kernels run
    # at the same time (each batch of two 1080x1920 frames fills less than half of the GPU)
    H, W = 1080, 1920
    f = 481.2 * W / 640
    r = scenes.Recipe(H=H, W=W, fx=f, fy=f, u0=(W - 1) / 2, v0=(H - 1) / 2, noise_k=0.0012, hole_frac=0.03)
    imgs = [scenes.render(6000 + k, r) for k in range(4)]
    ins = [dev_image(torch, tfn, img) for img in imgs]
    n_req = 24
    outs = [(tfn.empty_normals(H, W, "f32"), tfn.empty_image((H, W), torch.uint8)) for _ in range(n_req)]
    torch.cuda.synchronize()
    with tfn.Server(ctx, grad="fd", phi="mean", max_batch=2, pipelines=3) as srv:
        t0 = srv.submit(ins[0], r.camera, *outs[0])  # (warm-up: the pipelines' graphs)
        assert srv.wait(t0, 20000) == tfn.TFN_OK
        srv.stats(reset=True)
        tickets = [srv.submit(ins[k % 4], r.camera, *outs[k]) for k in range(n_req)]
        assert all(srv.wait(t, 20000) == tfn.TFN_OK for t in tickets)
        st = srv.stats()
    assert st["completed"] == n_req and st["batches"] >= n_req // 2
    assert st["max_batches_in_flight"] >= 2, st
    assert st["admitted_while_busy"] > 0, st
    assert st["device_overlaps"] > 0, st
    n_ref, m_ref = ctx.normals(ins[1], r.camera)
    torch.cuda.synchronize()
    assert torch.equal(outs[5][0], n_ref) and torch.equal(outs[5][1], m_ref)


def test_memory_budget_admission(torch, tfn, ctx):
    # 480x640 FP32 host requests stage about 5.3 MB each: a 16 MB budget admits three at a time
    reqs = [(scenes.render(500 + k, scenes.Recipe()), scenes.CAMERA) for k in range(9)]
    with tfn.Server(ctx, mem_budget=16 << 20, pipelines=4) as srv:
        subs = submit_all(torch, tfn, srv, reqs, host_every=1)
        for t, _, _ in subs:
            assert srv.wait(t, 20000) == tfn.TFN_OK
        st = srv.stats()
        assert st["staging_bytes_capacity"] == 16 << 20 and st["batches"] >= 3
        # a frame whose staging exceeds the whole budget can never be admitted
        big = np.full((1080, 1920), 2.0, np.float32)
        n = tfn.empty_normals(1080, 1920, "f32", "cpu")
        m = tfn.empty_image((1080, 1920), torch.uint8, "cpu")
        with pytest.raises(tfn.TfnError) as e:
            srv.submit(host_image(torch, tfn, big), scenes.CAMERA, n, m, host=True)
        assert e.value.status == tfn.TFN_ERR_OUT_OF_MEMORY
    img, cam = reqs[0]
    alone_n, alone_m = ctx.normals(dev_image(torch, tfn, img), cam)
    torch.cuda.synchronize()
    assert torch.equal(subs[0][1], alone_n.cpu()) and torch.equal(subs[0][2], alone_m.cpu())


def test_queue_limit_timeout_and_tickets(torch, tfn, ctx):
    big = np.full((4096, 4096), 3.0, np.float32)
    with tfn.Server(ctx, max_queue=2, pipelines=1) as srv:
        n = tfn.empty_normals(4096, 4096, "f32", "cpu")
        m = tfn.empty_image((4096, 4096), torch.uint8, "cpu")
        t_big = srv.submit(torch.from_numpy(big), scenes.CAMERA, n, m, host=True)  # pageable: a slow copy
        with pytest.raises(tfn.TfnError) as e:
            srv.wait(t_big, 0)  # polling right away: not done yet
        assert e.value.status == tfn.TFN_ERR_TIMEOUT
        small = [(scenes.render(600 + k, scenes.Recipe(H=48, W=64, fx=36.09, fy=36.09, u0=31.5, v0=23.5)),
                  dict(fx=36.09, fy=36.09, u0=31.5, v0=23.5)) for k in range(40)]
        accepted, busy = [], 0
        for img, cam in small:
            inp = dev_image(torch, tfn, img)
            nn = tfn.empty_normals(48, 64, "f32")
            mm = tfn.empty_image((48, 64), torch.uint8)
            try:
                accepted.append(srv.submit(inp, cam, nn, mm))
            except tfn.TfnError as err:
                assert err.status == tfn.TFN_ERR_BUSY
                busy += 1
        assert busy > 0 and srv.stats()["rejected"] == busy
        assert srv.wait(t_big, 60000) == tfn.TFN_OK
        for t in accepted:
            assert srv.wait(t, 20000) == tfn.TFN_OK
        with pytest.raises(tfn.TfnError) as e:
            srv.wait(t_big, 0)  # released by the first successful wait
        assert e.value.status == tfn.TFN_ERR_INVALID_ARG
        with pytest.raises(tfn.TfnError) as e:
            srv.wait(10 ** 9, 0)
        assert e.value.status == tfn.TFN_ERR_INVALID_ARG
    # constant depth: every evaluable pixel is [0, 0, -1]
    mk = m.numpy().astype(bool)
    assert mk[1:-1, 1:-1].all() and (n.numpy()[2][mk] == -1.0).all()


def test_invalid_requests_are_rejected_at_submit(torch, tfn, ctx):
    with tfn.Server(ctx) as srv:
        img = dev_image(torch, tfn, np.full((32, 32), 1.0, np.float32))
        n = tfn.empty_normals(32, 32, "f32")
        m = tfn.empty_image((32, 32), torch.uint8)
        with pytest.raises(tfn.TfnError) as e:
            srv.submit(img, dict(fx=-1.0, fy=1.0, u0=0, v0=0), n, m)
        assert e.value.status == tfn.TFN_ERR_INVALID_ARG
        base = torch.empty(32 * 40 + 1, dtype=torch.float32, device="cuda")
        odd = base[1:].view(32, 40)[:, :32]  # rows not on 16-byte boundaries
        with pytest.raises(tfn.TfnError) as e:
            srv.submit(odd, dict(fx=30.0, fy=30.0, u0=15.5, v0=15.5), n, m)
        assert e.value.status == tfn.TFN_ERR_MISALIGNED
        assert srv.stats()["submitted"] == 0


def test_autotune_table_and_cache_file(torch, tfn, ctx, tmp_path):
    imgs = [scenes.render(700 + k, scenes.Recipe()) for k in range(8)]
    inputs = [dev_image(torch, tfn, x) for x in imgs]
    with tfn.Context(0) as c:
        assert c.tuned_shape(tfn.TFN_DEPTH_F32) == -1
        ref_n, ref_m = c.normals_batch(inputs, scenes.CAMERA)
        torch.cuda.synchronize()
        ref = [x.cpu() for x in ref_n]
        best, ms = c.autotune(inputs, scenes.CAMERA, reps=3)
        assert 0 <= best < len(tfn.tile_shapes()) and len(ms) == len(tfn.tile_shapes())
        assert all(x > 0 for x in ms) and ms[best] == min(ms)
        assert c.tuned_shape(tfn.TFN_DEPTH_F32) == best
        assert c.tuned_shape(tfn.TFN_DEPTH_F16) == -1 and c.tuned_shape(tfn.TFN_DEPTH_F32, phi="median") == -1
        n2, m2 = c.normals_batch(inputs, scenes.CAMERA)  # runs with the tuned shape: same bits
        torch.cuda.synchronize()
        assert all(torch.equal(a.cpu(), b) for a, b in zip(n2, ref))
        path = str(tmp_path / "tune.txt")
        c.save_tune_cache(path)
    text = open(path).read().splitlines()
    assert text[0] == "tfn-tune 2" and text[1].startswith("device ") and len(text) == 3
    # the entry names the shape by its geometry: item size, then the CTA widths (3x3 filters, others)
    fields = text[2].split()
    shapes, warps = tfn.tile_shapes(), tfn.tile_shape_warps()
    assert tuple(map(int, fields[5:8])) == shapes[best] and tuple(map(int, fields[8:10])) == warps[best]
    # the tuner chooses CTA widths too: some heights are compiled with two widths
    assert len(set(zip(shapes, warps))) == len(shapes) > len(set(shapes))
    with tfn.Context(0) as c2:
        c2.load_tune_cache(path)
        assert c2.tuned_shape(tfn.TFN_DEPTH_F32) == best
        # a version 1 file (no CTA widths) loads as the shape of the default widths
        v1 = str(tmp_path / "v1.txt")
        with open(v1, "w") as f:
            f.write("\n".join(["tfn-tune 1", text[1], "entry 0 0 0 0 128 12 12 0.5"]) + "\n")
        c2.load_tune_cache(v1)
        assert c2.tuned_shape(tfn.TFN_DEPTH_F32) == 2 and warps[2] == (2, 4)
        c2.load_tune_cache(path)
        # another kind of device: nothing loaded
        other = str(tmp_path / "other.txt")
        with open(other, "w") as f:
            f.write("\n".join([text[0], "device Some_Other_GPU sms 7 cc 9.9"] + text[2:]) + "\n")
        with pytest.raises(tfn.TfnError) as e:
            c2.load_tune_cache(other)
        assert e.value.status == tfn.TFN_ERR_UNSUPPORTED
        bad = str(tmp_path / "bad.txt")
        with open(bad, "w") as f:
            f.write("\n".join(text[:2] + ["entry 0 0 0 0 64 32"]) + "\n")
        with pytest.raises(tfn.TfnError) as e:
            c2.load_tune_cache(bad)
        assert e.value.status == tfn.TFN_ERR_INVALID_ARG
        with pytest.raises(tfn.TfnError) as e:
            c2.load_tune_cache(str(tmp_path / "missing.txt"))
        assert e.value.status == tfn.TFN_ERR_IO
        # a forced shape overrides the table; -1 returns to it
        c2.set_tile_shape(len(tfn.tile_shapes()) - 1)
        c2.set_tile_shape(-1)
        with tfn.Server(c2) as srv:  # the server inherits the table
            n = tfn.empty_normals(480, 640, "f32")
            m = tfn.empty_image((480, 640), torch.uint8)
            assert srv.wait(srv.submit(inputs[0], scenes.CAMERA, n, m), 20000) == tfn.TFN_OK
            torch.cuda.synchronize()
            assert torch.equal(n.cpu(), ref[0])
