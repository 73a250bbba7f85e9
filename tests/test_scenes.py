"""The seeded input generator: determinism and the workload shapes it promises."""
import numpy as np

import scenes


def test_same_seed_same_bits_and_threads_agree():
    r = scenes.Recipe(noise_k=0.0012, hole_frac=0.03, H=60, W=80, u0=39.5, v0=29.5, fx=60.15, fy=60.15)
    a = scenes.render_batch(100, 5, r, threads=1)
    b = scenes.render_batch(100, 5, r, threads=4)
    assert a.tobytes() == b.tobytes()
    assert scenes.render(102, r).tobytes() == a[2].tobytes()
    assert a[0].tobytes() != a[1].tobytes()


def test_clean_scene_depth_range_and_truth():
    d, d64, prim, gt = scenes.render(1, with_truth=True)
    v = d > 0
    assert v.mean() > 0.9
    assert d[v].min() >= 0.5 and d[v].max() <= 10.0
    assert np.allclose(d[v], d64[v].astype(np.float32))
    assert ((prim >= 0) == v).all()
    assert np.allclose(np.sqrt((gt[:, v] ** 2).sum(0)), 1, atol=1e-6)


def test_noise_and_hole_statistics():
    r = scenes.Recipe(noise_k=0.0012, hole_frac=0.03)
    clean = scenes.render(1234, scenes.Recipe())
    noisy = scenes.render(1234, r)
    holes = (noisy == 0) & (clean > 0)
    assert 0.025 < holes.sum() / (clean > 0).sum() < 0.035
    both = (noisy > 0) & (clean > 0)
    z = clean[both].astype(np.float64)
    resid = (noisy[both] - clean[both]) / (0.0012 * z * z)
    assert abs(resid.mean()) < 0.01 and abs(resid.std() - 1) < 0.01


def test_disparity_workload_range():
    disp = scenes.disparity_batch(2)
    v = disp > 0
    assert disp[v].min() >= 16 and disp[v].max() <= 1536
    assert 0.04 < (disp == 0).mean() < 0.2
